// profile.cu -- optional per-phase CUDA-event timing of the library's kernel
// launches (off by default).  When enabled, every launch of a library kernel
// is bracketed by two events recorded on the launching stream; the totals per
// phase are read back by mw_profile_read.
#include <cuda_runtime.h>
#include <mutex>
#include <vector>

#include "mw_common.cuh"
#include "profile.cuh"

namespace mw {

namespace {
struct Entry {
  int phase;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Entry> g_entries;
std::vector<cudaEvent_t> g_pool;
long long g_counts[kNumPhases] = {0};

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

bool prof_enabled() { return g_on; }

void prof_count(int phase) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (phase >= 0 && phase < kNumPhases) g_counts[phase]++;
}

ProfScope::ProfScope(int phase, cudaStream_t s) : phase_(phase), s_(s), a_(nullptr) {
  prof_count(phase);
  if (!g_on) return;
  // inside a stream capture the events would become graph nodes that the
  // host never sees complete: count the launch only
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s_, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> lk(g_mu);
  a_ = take_event();
  cudaEventRecord(a_, s_);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, s_);
  g_entries.push_back({phase_, a_, b});
}

}  // namespace mw

extern "C" int mw_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(mw::g_mu);
  mw::g_on = on != 0;
  return MW_OK;
}

extern "C" int mw_profile_read(double* ms, long long* launches, int nphase, int reset) {
  if (nphase < 0) return -3;
  std::lock_guard<std::mutex> lk(mw::g_mu);
  std::vector<double> acc(mw::kNumPhases, 0.0);
  for (auto& e : mw::g_entries) {
    float t = 0.f;
    if (cudaEventSynchronize(e.b) != cudaSuccess) return MW_ECUDA;
    cudaEventElapsedTime(&t, e.a, e.b);
    acc[e.phase] += t;
  }
  for (int p = 0; p < nphase && p < mw::kNumPhases; ++p) {
    if (ms) ms[p] = acc[p];
    if (launches) launches[p] = mw::g_counts[p];
  }
  if (reset) {
    for (auto& e : mw::g_entries) {
      mw::g_pool.push_back(e.a);
      mw::g_pool.push_back(e.b);
    }
    mw::g_entries.clear();
    for (int p = 0; p < mw::kNumPhases; ++p) mw::g_counts[p] = 0;
  }
  return MW_OK;
}
