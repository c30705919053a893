"""bench.py's reference arm is the CPU oracle timed on whole systems of the
headline batch; it needs no GPU, so its JSON line is checked here on a small
batch: the keys of the bench contract, the metric and workload of the GPU
arm, a value that is the oracle's own timing (no extrapolation), and an
end-to-end entry with no host-device traffic.  Under torchrun only rank 0
works and prints."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_contract", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


ARGS = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0", "--count", "32"]


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, *ARGS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def _lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_line_keeps_the_contract():
    bench = _bench_module()
    p = _run()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "solves/s at 2^-200 rel. error" and d["unit"] == "solves/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == bench.workload_name(32) and d["config"]["systems"] == 32
    assert bench.workload_name(bench.BATCH).startswith("mixed_batch_512_svd_n64-1024_kappa1e4-1e20")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # value x step time = the sampled systems that met the target (here the one
    # system a 32-system batch contributes): a timing, not an extrapolation
    assert abs(d["ms_per_step"] * 1e-3 * d["value"] - 1.0) < 1e-9


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0
    assert not [l for l in p.stdout.splitlines() if l.startswith("{")]


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_torchrun_prints_once_on_all_cores():
    single = _lines(_run().stdout)
    p = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), *ARGS, "--gpus", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _lines(p.stdout)
    assert len(lines) == 1 and len(single) == 1
    assert lines[0]["n_gpus"] == 2
    assert lines[0]["cpu_baseline"]["cores"] == single[0]["cpu_baseline"]["cores"]
