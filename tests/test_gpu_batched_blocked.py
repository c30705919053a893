"""Blocked batched LU (all systems advance one 64-column panel per step; one
trailing-update launch over the tiles of every active system) and the
batched refinement on top of it, through the C ABI.

Plain update: every system's factors, pivots, info, solutions and refined
solutions are bitwise identical to the CPU oracle's single-system results.
Split update (DD): per-system normwise backward error <= 1e-28 and pivots
that agree with the oracle's except at rare near-ties; refinement to
2^-200 checked exactly against x* = ones."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from parity_rules import check_pivots_near_tie
from paper_2107_12550_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_12550_gb300 import build as B
    B.build()


def api():
    from paper_2107_12550_gb300 import api as A
    return A


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _uniform_batch(w, n_list, seed):
    mats = [W.uniform_matrix(int(n), w, seed=W.system_seed(seed, s), lda=int(n)) for s, n in enumerate(n_list)]
    vecs = []
    for s, n in enumerate(n_list):
        v = np.zeros((w, int(n)))
        v[0] = W.uniform_matrix(int(n), 1, seed=W.system_seed(seed + 1, s), lda=int(n))[0, 0, :]
        vecs.append(v)
    return mats, vecs


# orders around the panel width and the tile edges, plus a ragged random mix
EDGE_N = [1, 2, 63, 64, 65, 127, 128, 129, 192, 257]


@pytest.mark.parametrize("w", [2, 3, 4])
def test_blocked_plain_bitwise(w):
    n_list = EDGE_N + [int(v) for v in W.batch_sizes(14, 1, 300, seed=40 + w)]
    mats, vecs = _uniform_batch(w, n_list, seed=20 * w)
    A = dev(api().pack_matrices(mats, w))
    b = dev(api().pack_vectors(vecs, w))
    LU, piv, info = api().ludecomp_batched_blocked(A, n_list, w, "plain")
    x = api().solve_batched(LU, piv, b, n_list, w)
    LUs = api().unpack_matrices(host(LU), n_list, w)
    xs = api().unpack_vectors(host(x), n_list, w)
    _, voff = api().batch_offsets(n_list)
    pv = host(piv)
    inf = host(info)
    for s, n in enumerate(n_list):
        LUo, pivo, infoo = oracle.lu(w, mats[s])
        assert np.array_equal(LUs[s], LUo[:, :, :n]), (s, n)
        assert np.array_equal(pv[voff[s]: voff[s] + n], pivo), (s, n)
        assert inf[s] == infoo
        assert np.array_equal(xs[s], oracle.solve(w, LUo, pivo, vecs[s])), (s, n)


def test_blocked_plain_equals_persistent():
    """Both batched LUs apply every element's updates in the same order."""
    w = 2
    n_list = [int(v) for v in W.batch_sizes(60, 1, 400, seed=5)]
    mats, _ = _uniform_batch(w, n_list, seed=77)
    A = dev(api().pack_matrices(mats, w))
    LUb, pivb, infob = api().ludecomp_batched_blocked(A, n_list, w, "plain")
    LUp, pivp, infop = api().ludecomp_batched(A, n_list, w)
    assert torch.equal(LUb, LUp) and torch.equal(pivb, pivp) and torch.equal(infob, infop)


def test_blocked_singular_member():
    w = 3
    n_list = [70, 130, 9, 200]
    mats, _ = _uniform_batch(w, n_list, seed=8)
    mats[1][:, 100, :] = 0.0          # zero column in the second panel
    mats[2][:, :, 3] = 0.0            # zero row
    A = dev(api().pack_matrices(mats, w))
    LU, piv, info = api().ludecomp_batched_blocked(A, n_list, w, "plain")
    inf = host(info)
    LUs = api().unpack_matrices(host(LU), n_list, w)
    for s in range(len(n_list)):
        LUo, _, infoo = oracle.lu(w, mats[s])
        assert inf[s] == infoo
        assert np.array_equal(LUs[s], LUo[:, :, :n_list[s]])
    assert inf[1] > 0 and inf[2] > 0 and inf[0] == 0 and inf[3] == 0


def _eta(A, b, x):
    n = x.shape[1]
    r = oracle.residual(A, b, x, 8)
    Ainf = np.max(np.sum(np.abs(A[0, :, :n]), axis=0))
    return np.max(np.abs(r[0])) / (Ainf * np.max(np.abs(x[0])) + np.max(np.abs(b[0])))


def test_blocked_split_dd_backward_error_and_pivots():
    n_list = [65, 200, 300, 129, 64, 1, 513, 128, 257]
    mats, vecs = _uniform_batch(2, n_list, seed=31)
    A = dev(api().pack_matrices(mats, 2))
    b = dev(api().pack_vectors(vecs, 2))
    LU, piv, info = api().ludecomp_batched_blocked(A, n_list, 2, "split")
    x = api().solve_batched(LU, piv, b, n_list, 2)
    xs = api().unpack_vectors(host(x), n_list, 2)
    _, voff = api().batch_offsets(n_list)
    pv = host(piv)
    assert int(host(info).max()) == 0
    for s, n in enumerate(n_list):
        eta = _eta(mats[s], vecs[s], xs[s])
        assert eta <= 1e-28, (s, n, eta)
        _, pivo, _ = oracle.lu(2, mats[s])
        check_pivots_near_tie(mats[s], 2, pv[voff[s]: voff[s] + n], pivo)


@pytest.mark.parametrize("leaf", [16, 32])
def test_blocked_split_leaf_widths(leaf):
    """Every leaf width the tuner may choose for the batched split panel
    (MW_TUNE_BATCH_SPLIT_LEAF; 8 is the default, tested above): each system
    keeps eta <= 1e-28 and pivots as the oracle's up to a near-tie."""
    from paper_2107_12550_gb300 import _lib as L
    lib = L.lib()
    prev = lib.mw_set_tuning(L.MW_TUNE_BATCH_SPLIT_LEAF, 2, leaf)
    try:
        n_list = [65, 200, 300, 129, 513, 128, 257]
        mats, vecs = _uniform_batch(2, n_list, seed=37)
        A = dev(api().pack_matrices(mats, 2))
        b = dev(api().pack_vectors(vecs, 2))
        LU, piv, info = api().ludecomp_batched_blocked(A, n_list, 2, "split")
        x = api().solve_batched(LU, piv, b, n_list, 2)
        xs = api().unpack_vectors(host(x), n_list, 2)
        _, voff = api().batch_offsets(n_list)
        pv = host(piv)
        for s, n in enumerate(n_list):
            assert _eta(mats[s], vecs[s], xs[s]) <= 1e-28, (leaf, s, n)
            _, pivo, _ = oracle.lu(2, mats[s])
            check_pivots_near_tie(mats[s], 2, pv[voff[s]: voff[s] + n], pivo)
    finally:
        lib.mw_set_tuning(L.MW_TUNE_BATCH_SPLIT_LEAF, 2, prev)


def test_blocked_split_close_to_plain_factors():
    """The batched split LU (U12 from the explicit inverse of L11 and both
    products on the tensor cores) stays within a few DD roundings of the
    plain factors: same pivots, entrywise |LU_split - LU_plain| <= 2^-90
    max|A| (uniform entries, moderate growth)."""
    n_list = [300, 129, 200]
    mats, _ = _uniform_batch(2, n_list, seed=55)
    A = dev(api().pack_matrices(mats, 2))
    LU, piv, _ = api().ludecomp_batched_blocked(A, n_list, 2, "split")
    LUs = api().unpack_matrices(host(LU), n_list, 2)
    _, voff = api().batch_offsets(n_list)
    pv = host(piv)
    for s, n in enumerate(n_list):
        LUo, pivo, _ = oracle.lu(2, mats[s])
        assert np.array_equal(pivo, pv[voff[s]: voff[s] + n])
        d = np.abs((LUs[s][0] - LUo[0, :, :n]) + (LUs[s][1] - LUo[1, :, :n]))
        assert d.max() <= 2.0 ** -90, (s, n, np.log2(d.max()))


@pytest.mark.parametrize("inner", [2, 3])
def test_refine_blocked_plain_bitwise(inner):
    n_list = [24, 5, 130, 70, 1, 47]
    systems = [W.svd_system(n, [4.0, 8.0, 12.0][s % 3], seed=300 + s) if n > 1 else
               W.System(np.array([[[3.0]]]), np.array([[1.0]] + [[0.0]] * 7), None) for s, n in enumerate(n_list)]
    A = dev(api().pack_matrices([s.A for s in systems], 4))
    b = dev(api().pack_vectors([s.b for s in systems], 8))
    x, stats = api().refine_batched_blocked(A, 4, b, 8, n_list, inner, "plain", 200)
    xs = api().unpack_vectors(host(x), n_list, 8)
    st = host(stats)
    for s, sysm in enumerate(systems):
        status, xo, corr, nres, info = oracle.refine(sysm.A, sysm.b, inner)
        assert (st[s, 0], st[s, 1], st[s, 2], st[s, 3]) == (corr, nres, info, status), s
        assert np.array_equal(xs[s], xo), s


def test_refine_blocked_split_reaches_target():
    """DD inner LU with the split update on kappa up to 1e20 (the mixed
    batched-refinement workload's range): every system converges and every
    sampled x_i equals x* = 1 to 2^-200 (exact check)."""
    n_list = [64, 150, 300, 97, 257]
    kap = [4.0, 20.0, 12.0, 16.0, 8.0]
    systems = [W.svd_system(n, kap[s], seed=500 + s) for s, n in enumerate(n_list)]
    A = dev(api().pack_matrices([s.A for s in systems], 4))
    b = dev(api().pack_vectors([s.b for s in systems], 8))
    x, stats = api().refine_batched_blocked(A, 4, b, 8, n_list, 2, "split", 200)
    xs = api().unpack_vectors(host(x), n_list, 8)
    st = host(stats)
    for s, n in enumerate(n_list):
        assert st[s, 3] == 0, (s, st[s])
        for i in range(0, n, 7):
            v = sum(Fraction(float(c)) for c in xs[s][:, i])
            assert abs(v - 1) <= Fraction(1, 2 ** 200), (s, i)


def test_batched_lu_and_solve_in_a_cuda_graph():
    """With resident plans, the blocked batched LU (split and plain) and the
    batched solve are captured in a CUDA graph; each replay reproduces the
    eager results bitwise."""
    n_list = [int(v) for v in W.batch_sizes(24, 1, 300, seed=71)]
    mats, vecs = _uniform_batch(2, n_list, seed=72)
    A = dev(api().pack_matrices(mats, 2))
    b = dev(api().pack_vectors(vecs, 2))
    from paper_2107_12550_gb300 import _lib as L
    prev = api().batch_plan_cache(True)
    try:
        for upd in ("plain", "split"):
            wk = api().batch_blocked_workspace(L.MW_OP_LUDECOMP, 2, upd, n_list)
            wks = api().batch_workspace(L.MW_OP_SOLVE, 2, n_list)
            LU = torch.empty_like(A)
            x = torch.empty_like(b)
            total_n = int(sum(n_list))
            piv = torch.empty(total_n, dtype=torch.int64, device="cuda")

            def step():
                LU.copy_(A)
                _, pv, _ = api().ludecomp_batched_blocked(LU, n_list, 2, upd, work=wk, inplace=True)
                piv.copy_(pv)
                api().solve_batched(LU, piv, b, n_list, 2, work=wks, out=x)

            step()                                   # uploads the plans
            torch.cuda.synchronize()
            LU_ref, x_ref = LU.clone(), x.clone()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                step()                               # warm on the capture stream
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step()
            LU.zero_()
            x.zero_()
            for _ in range(2):
                g.replay()
                torch.cuda.synchronize()
                assert torch.equal(LU, LU_ref) and torch.equal(x, x_ref), upd
    finally:
        api().batch_plan_cache(prev)


def test_mixed_batch_refine_full_range_exact():
    """The mixed-precision batched refinement at the workload's full ranges:
    the n and kappa of every 11th member of the 512-system workload plus
    its largest and most ill-conditioned ones (n up to 1024, kappa up to
    1e20), each system built with its seed in the workload: split DD inner LU, every
    system converges and every entry of every x equals x* = 1 to 2^-200
    (exact check)."""
    n_all, k_all = W.mixed_batch_spec(512, 64, 1024, 4.0, 20.0, seed=0)
    pick = sorted(set(list(range(0, 512, 11)) + [int(np.argmax(n_all)), int(np.argmax(k_all))]))
    n_list = [n_all[s] for s in pick]
    kap = [k_all[s] for s in pick]
    A_np, b_np = W.svd_batch(n_list, kap, seed=0, processes=4, system_ids=pick)
    x, stats = api().refine_batched_blocked(dev(A_np), 4, dev(b_np), 8, n_list, 2, "split", 200)
    st = host(stats)
    assert (st[:, 3] == 0).all(), st[st[:, 3] != 0]
    xs = api().unpack_vectors(host(x), n_list, 8)
    lim = Fraction(1, 2 ** 200)
    for s, n in enumerate(n_list):
        X = xs[s]
        for i in range(n):
            v = sum((Fraction(float(c)) for c in X[:, i]), Fraction(0))
            assert abs(v - 1) <= lim, (s, n, i)


@pytest.mark.parametrize("update", ["split", "plain"])
def test_batched_refinement_in_one_cuda_graph(update):
    """The whole batched refinement (blocked batched LU, substitution, and
    the refinement loop as a while node whose condition a kernel sets) is
    captured in one CUDA graph; each replay reproduces the eager call's x and
    per-system statistics bitwise, with no value read back in between."""
    n_all, k_all = W.mixed_batch_spec(512, 64, 1024, 4.0, 20.0, seed=0)
    pick = [s for s in range(512) if n_all[s] <= 320][:24]
    n_list = [n_all[s] for s in pick]
    kap = [k_all[s] for s in pick]
    A_np, b_np = W.svd_batch(n_list, kap, seed=0, processes=4, system_ids=pick)
    A, b = dev(A_np), dev(b_np)
    from paper_2107_12550_gb300 import _lib as L
    prev = api().batch_plan_cache(True)
    try:
        work = api().batch_blocked_workspace(L.MW_OP_REFINE, 2, update, n_list)
        x = torch.empty(8 * int(sum(n_list)), dtype=torch.float64, device="cuda")
        st = torch.empty((len(n_list), 4), dtype=torch.int64, device="cuda")

        def step():
            _, stats = api().refine_batched_blocked(A, 4, b, 8, n_list, 2, update, 200, work=work, out=x)
            st.copy_(stats)

        step()                                   # uploads the plans, outside the capture
        torch.cuda.synchronize()
        x_ref, st_ref = x.clone(), st.clone()
        assert (st_ref[:, 3] == 0).all()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
        for _ in range(2):
            x.zero_()
            st.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(x, x_ref) and torch.equal(st, st_ref), update
    finally:
        api().batch_plan_cache(prev)


@pytest.mark.parametrize("w,update", [(2, "plain"), (3, "plain"), (2, "split")])
def test_blocked_lookahead_bitwise_equal_to_serial(w, update):
    """With the look-ahead (MW_TUNE_LOOKAHEAD) the tiles holding the next
    panel's columns are updated first and that panel is factored on a second
    stream beside the other tiles; the factors, pivots and info are bit for
    bit those of the serial schedule (orders around the panel and tile
    edges, and a ragged mix up to 700)."""
    from paper_2107_12550_gb300 import _lib as L
    lib = L.lib()
    n_list = EDGE_N + [int(v) for v in W.batch_sizes(40, 1, 700, seed=90 + w)]
    mats, _ = _uniform_batch(w, n_list, seed=30 * w)
    prev = lib.mw_get_tuning(L.MW_TUNE_LOOKAHEAD, w)
    out = {}
    try:
        for la in (0, 1, 1):
            lib.mw_set_tuning(L.MW_TUNE_LOOKAHEAD, w, la)
            A = dev(api().pack_matrices(mats, w))
            LU, piv, info = api().ludecomp_batched_blocked(A, n_list, w, update)
            out.setdefault(la, []).append((host(LU), host(piv), host(info)))
    finally:
        lib.mw_set_tuning(L.MW_TUNE_LOOKAHEAD, w, prev)
    ref = out[0][0]
    for LU, piv, info in out[1]:
        assert np.array_equal(info, ref[2])
        assert np.array_equal(piv, ref[1])
        assert np.array_equal(LU.view(np.uint64), ref[0].view(np.uint64))
