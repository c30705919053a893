// mw_common.cuh -- status codes, launch checks, the bounded-wait helpers and
// the cp.async wrappers shared by the library's kernels.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "../../include/mwlu.h"

namespace mw {

// Error word written by kernels that give up on a bounded wait.
struct DeviceStatus {
  unsigned int timeout;     // non-zero: a bounded spin-wait ran out
  unsigned int where;       // which wait (kernel-specific tag)
};

// The abort word shared by the CTAs of one cooperative launch.  Each of
// their waits spins at most a bounded number of times; a CTA whose wait
// gives up records the wait's tag in `status` and sets `abort`, and the
// waits of the other CTAs see it and leave as well.
struct GridAbort {
  unsigned int abort;
  unsigned int pad[3];
};

constexpr unsigned long long kSpinLimit = 1ull << 26;  // ~seconds at worst

// The poll limit that the host passes to the kernels whose waits it bounds
// (the substitution's ready-value polls, the panel's record waits, the
// batched substitution's flag waits): 0 (each kernel's own default) unless
// mw_set_wait_limit chose another (host function, capi.cu).
unsigned long long wait_limit();
__host__ __device__ constexpr unsigned long long pick_limit(unsigned long long given, unsigned long long dflt) {
  return given ? given : dflt;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const void* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(void* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? MW_OK : MW_ECUDA; }

// Raises a kernel's dynamic shared memory limit to at least `bytes` on the
// current device, once per (kernel, device) and size, when the dynamic bytes
// and the kernel's static shared memory (static_bytes) exceed the default
// 48 KB: the attribute belongs to the device's context, so every GPU a
// process uses needs its own call.  Safe for concurrent callers.  Returns a
// cudaError_t.
cudaError_t ensure_smem_limit(const void* kernel, size_t bytes, size_t static_bytes = 0);
template <typename K>
inline cudaError_t ensure_smem_limit(K* kernel, size_t bytes, size_t static_bytes = 0) {
  return ensure_smem_limit(reinterpret_cast<const void*>(kernel), bytes, static_bytes);
}

// the current device's SM count (cached per device; 1 if it cannot be read)
int device_sm_count();

#ifdef __CUDACC__
// 8-byte asynchronous copy global -> shared; ok == false fills zeros (no read)
__device__ __forceinline__ void cp_async8(void* smem_dst, const double* gsrc, bool ok) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(saddr), "l"(gsrc), "r"(ok ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
#endif

}  // namespace mw

// record the last CUDA error of the library for mw_last_cuda_error()
extern "C" void mw_internal_set_cuda_error(int e);

#define MW_CUDA_CHECK(expr)                                      \
  do {                                                           \
    cudaError_t _e = (expr);                                     \
    if (_e != cudaSuccess) {                                     \
      mw_internal_set_cuda_error((int)_e);                       \
      return MW_ECUDA;                                           \
    }                                                            \
  } while (0)

#define MW_LAUNCH_CHECK()                                        \
  do {                                                           \
    cudaError_t _e = cudaGetLastError();                         \
    if (_e != cudaSuccess) {                                     \
      mw_internal_set_cuda_error((int)_e);                       \
      return MW_ECUDA;                                           \
    }                                                            \
  } while (0)
