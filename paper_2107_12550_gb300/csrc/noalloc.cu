// noalloc.cu -- mw_solve_noalloc: forward/back substitution for callers
// that cannot hand the library a work buffer.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they need a solve: code running inside a framework that owns all device
// memory through its own pool and forbids outside allocations, plugins and
// hooks that are not allowed to allocate, and latency-critical loops that
// must not touch the allocator.  mw_solve asks for a caller-provided work
// buffer; this entry point instead uses a fixed scratch array that lives in
// the library's own device memory, so the caller only passes the factors,
// the right-hand side and the output.
//
// The scratch is kNoallocScratchBytes of file-scope __device__ memory.  Every
// GPU that loads the library holds it until the process exits.  Host code
// cannot use the array's name as a device address, so on the first call on
// each device (with that device current) the address is fetched with
// cudaGetSymbolAddress and cached.  The cache is keyed on the device index
// only: it does not survive cudaDeviceReset (the library's device memory,
// the scratch array included, is reloaded at a new address afterwards).
//
// Order bound: the largest order whose scratch fits at any precision is
// DD's 40320; orders above it are rejected before any size is computed, so
// no size arithmetic can overflow.
#include <cuda_runtime.h>
#include <cstdint>
#include <mutex>

#include "mw_common.cuh"
#include "lu_internal.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = MW_NOALLOC_SCRATCH_BYTES;
constexpr int64_t kNoallocMaxOrder = 40320;   // DD; TD and QD fit fewer
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array for the current device (set-up once)
int scratch_address(void** out) {
  int dev = 0;
  MW_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return MW_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    MW_CUDA_CHECK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MW_OK;
}

}  // namespace

extern "C" int mw_solve_noalloc(int prec, int64_t n, const double* LU, int64_t lda, const int64_t* piv,
                                const double* b, double* x, void* stream) {
  if (prec != MW_DD && prec != MW_TD && prec != MW_QD) return -1;
  if (n < 0 || n > kNoallocMaxOrder) return -2;                               // before any size arithmetic
  if (mw::solve_workspace_bytes(prec, n) > kNoallocScratchBytes) return -2;  // beyond the fixed scratch
  if (n > 0 && !LU) return -3;
  if (lda < (n > 1 ? n : 1) || lda > mw::kMaxOrder) return -4;
  if (n > 0 && !piv) return -5;
  if (n > 0 && !b) return -6;
  if (n > 0 && !x) return -7;
  if (n == 0) return MW_OK;
  void* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != MW_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(scratch);
  switch (prec) {
    case MW_DD: return mw::solve_launch<2>(n, LU, lda, piv, b, x, ws, kNoallocScratchBytes, s);
    case MW_TD: return mw::solve_launch<3>(n, LU, lda, piv, b, x, ws, kNoallocScratchBytes, s);
    default: return mw::solve_launch<4>(n, LU, lda, piv, b, x, ws, kNoallocScratchBytes, s);
  }
}

extern "C" int mw_solve_noalloc_status(void* stream) {
  void* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != MW_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mw::DeviceStatus st = {};
  MW_CUDA_CHECK(cudaMemcpyAsync(&st, static_cast<char*>(scratch) + mw::kWsStatus, sizeof(st),
                                cudaMemcpyDeviceToHost, s));
  MW_CUDA_CHECK(cudaStreamSynchronize(s));
  return st.timeout ? MW_ETIMEOUT : MW_OK;
}
