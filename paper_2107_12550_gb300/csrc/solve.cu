// solve.cu -- forward/back substitution with the factors of the blocked LU
// (Section 2, Listing 1: SolveTDLSPM).
//
// y = P b; y_i -= l_ij y_j (j ascending); x_j = y_j / u_jj and
// y_i -= u_ij x_j (j descending).  One cooperative launch runs a wavefront
// over block-rows of 32: each warp owns block-rows (lane = row) and keeps
// their values in registers.  For block-row I it waits, block by block, for
// the ready flag of every block J < I (forward) or J > I (back), applies that
// block's 32 updates in order with the published values, then solves its own
// diagonal block with shuffles, publishes the result and raises its flag.
// No grid-wide barrier is needed.  Each entry sees the same sequence of
// rounded multiply-subtract steps as the column-by-column algorithm, so the
// result is bitwise identical to it.
#include <algorithm>
#include <cuda_runtime.h>

#include "mw_arith.cuh"
#include "mw_common.cuh"
#include "lu_internal.cuh"
#include "profile.cuh"

namespace mw {

constexpr int kSolveBlock = 32;
constexpr int kSolveMaxOwned = 8;              // block-rows per warp kept in registers
constexpr int64_t kPermSmemMax = 26 * 1024;   // pivots handled in shared memory up to here

// solve work buffer: [status | perm (int32 n) | ready flags (int32 per block) | y (w planes of n)]
constexpr size_t kSolveWsPerm = 256;
__host__ __device__ inline size_t solve_ws_flags(int64_t n) {
  return (kSolveWsPerm + 4 * (size_t)n + 255) & ~(size_t)255;
}
__host__ __device__ inline int64_t solve_nblk(int64_t n) { return (n + kSolveBlock - 1) / kSolveBlock; }
__host__ __device__ inline size_t solve_ws_y(int64_t n) {
  return solve_ws_flags(n) + ((4 * (size_t)solve_nblk(n) + 255) & ~(size_t)255);
}

size_t solve_workspace_bytes(int w, int64_t n) {
  return solve_ws_y(n) + align256(sizeof(double) * (size_t)w * (size_t)(n > 0 ? n : 1));
}

// perm[i] = index of b that lands in row i after the swaps piv[0..n-1]
__global__ void __launch_bounds__(1024) k_perm(int64_t n, const int64_t* __restrict__ piv,
                                               int* __restrict__ perm) {
  extern __shared__ int sp[];
  const bool in_smem = n <= kPermSmemMax;
  int* pm = in_smem ? sp : perm;
  int* pv = in_smem ? sp + n : nullptr;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    pm[i] = (int)i;
    if (in_smem) pv[i] = (int)piv[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int64_t k = 0; k < n; ++k) {
      const int64_t p = in_smem ? pv[k] : piv[k];
      if (p != k) {
        const int t = pm[k];
        pm[k] = pm[p];
        pm[p] = t;
      }
    }
  }
  __syncthreads();
  if (in_smem)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) perm[i] = pm[i];
}

template <int W>
__device__ __forceinline__ val<W> shfl_val(const val<W>& v, int src) {
  val<W> z;
#pragma unroll
  for (int c = 0; c < W; ++c) z.v[c] = __shfl_sync(0xffffffffu, v.v[c], src);
  return z;
}

__device__ __forceinline__ int ld_acquire_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_i32(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// lane 0 waits (bounded) until flags[J] >= level; false if it gave up
__device__ __forceinline__ bool wait_flag(const int* flags, int64_t J, int level, DeviceStatus* status, int tag) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    unsigned long long spins = 0;
    while (ld_acquire_i32(flags + J) < level) {
      if (++spins > kSpinLimit) {
        atomicExch(&status->timeout, 1u);
        atomicExch(&status->where, (unsigned)tag);
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  return ok != 0;
}

// One warp per CTA; warp b owns block-rows b, b + G, b + 2G, ...
template <int W>
__global__ void __launch_bounds__(32)
k_solve(const double* __restrict__ LU, int64_t lda, int64_t plane, int64_t n,
        const double* b, double* x, char* __restrict__ ws) {
  DeviceStatus* status = reinterpret_cast<DeviceStatus*>(ws + kWsStatus);
  const int* perm = reinterpret_cast<const int*>(ws + kSolveWsPerm);
  int* flags = reinterpret_cast<int*>(ws + solve_ws_flags(n));
  double* y = reinterpret_cast<double*>(ws + solve_ws_y(n));
  const int lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  const int64_t nblk = solve_nblk(n);

  // gather y = P b for every owned block-row (before any flag is raised, so
  // b may alias x)
  val<W> yr[kSolveMaxOwned];
#pragma unroll
  for (int q = 0; q < kSolveMaxOwned; ++q) {
    const int64_t I = blockIdx.x + q * G;
    const int64_t i = I * kSolveBlock + lane;
#pragma unroll
    for (int c = 0; c < W; ++c) yr[q].v[c] = 0.0;
    if (I < nblk && i < n) {
      const int src = perm[i];
#pragma unroll
      for (int c = 0; c < W; ++c) yr[q].v[c] = b[c * n + src];
    }
  }

  // forward: unit lower L, block-rows in increasing order
#pragma unroll
  for (int q = 0; q < kSolveMaxOwned; ++q) {
    const int64_t I = blockIdx.x + q * G;
    if (I >= nblk) break;
    const int64_t i = I * kSolveBlock + lane;
    const bool row_ok = i < n;
    val<W> acc = yr[q];
    for (int64_t J = 0; J < I; ++J) {
      if (!wait_flag(flags, J, 1, status, 21)) return;
      const val<W> yJ = load_cg<W>(y, n, J * kSolveBlock + lane);
      for (int jj = 0; jj < kSolveBlock; ++jj) {
        const val<W> yj = shfl_val<W>(yJ, jj);
        if (row_ok) {
          const val<W> l = load_ro<W>(LU, plane, (J * kSolveBlock + jj) * lda + i);
          acc = msub<W>(acc, l, yj);
        }
      }
    }
    const int jb = (int)((n - I * kSolveBlock < kSolveBlock) ? n - I * kSolveBlock : kSolveBlock);
    for (int jj = 0; jj < jb; ++jj) {
      const val<W> yj = shfl_val<W>(acc, jj);
      if (lane > jj && lane < jb) {
        const val<W> l = load_ro<W>(LU, plane, (I * kSolveBlock + jj) * lda + i);
        acc = msub<W>(acc, l, yj);
      }
    }
    if (row_ok) store_cg<W>(y, n, i, acc);
    yr[q] = acc;
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release_i32(flags + I, 1);
  }

  // back: upper U, block-rows in decreasing order
#pragma unroll
  for (int q = kSolveMaxOwned - 1; q >= 0; --q) {
    const int64_t I = blockIdx.x + q * G;
    if (I >= nblk) continue;
    const int64_t i = I * kSolveBlock + lane;
    const bool row_ok = i < n;
    val<W> acc = yr[q];
    for (int64_t J = nblk - 1; J > I; --J) {
      if (!wait_flag(flags, J, 2, status, 22)) return;
      const int jbJ = (int)((n - J * kSolveBlock < kSolveBlock) ? n - J * kSolveBlock : kSolveBlock);
      val<W> xJ;
      if (lane < jbJ) xJ = load_cg<W>(y, n, J * kSolveBlock + lane);
      else {
#pragma unroll
        for (int c = 0; c < W; ++c) xJ.v[c] = 0.0;
      }
      for (int jj = jbJ - 1; jj >= 0; --jj) {
        const val<W> xj = shfl_val<W>(xJ, jj);
        if (row_ok) {
          const val<W> u = load_ro<W>(LU, plane, (J * kSolveBlock + jj) * lda + i);
          acc = msub<W>(acc, u, xj);
        }
      }
    }
    const int jb = (int)((n - I * kSolveBlock < kSolveBlock) ? n - I * kSolveBlock : kSolveBlock);
    for (int jj = jb - 1; jj >= 0; --jj) {
      if (lane == jj) {
        const val<W> ujj = load_ro<W>(LU, plane, (I * kSolveBlock + jj) * lda + i);
        acc = div<W>(acc, ujj);
      }
      const val<W> xj = shfl_val<W>(acc, jj);
      if (lane < jj) {
        const val<W> u = load_ro<W>(LU, plane, (I * kSolveBlock + jj) * lda + i);
        acc = msub<W>(acc, u, xj);
      }
    }
    if (row_ok) store_cg<W>(y, n, i, acc);
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release_i32(flags + I, 2);
    if (row_ok) {
#pragma unroll
      for (int c = 0; c < W; ++c) x[c * n + i] = acc.v[c];
    }
  }
}

static int sm_count_solve() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

int perm_launch(int64_t n, const int64_t* piv, int* perm, cudaStream_t s) {
  ProfScope ps(kPhPerm, s);
  const size_t shmem = (n <= kPermSmemMax) ? 8 * (size_t)n : 0;
  if (shmem > 48 * 1024) {
    MW_CUDA_CHECK(cudaFuncSetAttribute(k_perm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem));
  }
  k_perm<<<1, 1024, shmem, s>>>(n, piv, perm);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

// The permutation must already be in the work buffer (perm_launch).
template <int W>
int solve_with_perm(int64_t n, const double* LU, int64_t lda, const double* b, double* x,
                    char* ws, cudaStream_t s) {
  const int64_t plane = lda * n;
  ProfScope ps(kPhSolve, s);
  const int64_t nblk = solve_nblk(n);
  int64_t G = std::min<int64_t>(nblk, 4 * (int64_t)sm_count_solve());
  if (nblk > G * kSolveMaxOwned) return MW_EUNSUPPORTED;
  G = std::max<int64_t>(G, (nblk + kSolveMaxOwned - 1) / kSolveMaxOwned);
  MW_CUDA_CHECK(cudaMemsetAsync(ws, 0, kSolveWsPerm, s));
  MW_CUDA_CHECK(cudaMemsetAsync(ws + solve_ws_flags(n), 0, 4 * (size_t)nblk, s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MW_CUDA_CHECK(cudaLaunchKernelEx(&cfg, k_solve<W>, LU, lda, plane, n, b, x, ws));
  return MW_OK;
}

template <int W>
int solve_launch(int64_t n, const double* LU, int64_t lda, const int64_t* piv, const double* b,
                 double* x, char* ws, size_t ws_bytes, cudaStream_t s) {
  if (n == 0) return MW_OK;
  if (ws_bytes < solve_workspace_bytes(W, n)) return -9;
  int rc = perm_launch(n, piv, reinterpret_cast<int*>(ws + kSolveWsPerm), s);
  if (rc) return rc;
  return solve_with_perm<W>(n, LU, lda, b, x, ws, s);
}

template int solve_launch<2>(int64_t, const double*, int64_t, const int64_t*, const double*, double*, char*, size_t, cudaStream_t);
template int solve_launch<3>(int64_t, const double*, int64_t, const int64_t*, const double*, double*, char*, size_t, cudaStream_t);
template int solve_launch<4>(int64_t, const double*, int64_t, const int64_t*, const double*, double*, char*, size_t, cudaStream_t);
template int solve_with_perm<2>(int64_t, const double*, int64_t, const double*, double*, char*, cudaStream_t);
template int solve_with_perm<3>(int64_t, const double*, int64_t, const double*, double*, char*, cudaStream_t);
template int solve_with_perm<4>(int64_t, const double*, int64_t, const double*, double*, char*, cudaStream_t);

}  // namespace mw
