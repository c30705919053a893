// solve.cu -- forward/back substitution with the factors of the blocked LU
// (Section 2, Listing 1: SolveTDLSPM).
//
// y = P b; y_i -= l_ij y_j (j ascending); d_j = 1 / u_jj for every j (a
// parallel prologue), then x_j = y_j d_j and y_i -= u_ij x_j (j
// descending).  One cooperative launch runs a row-granular wavefront over
// block-rows of 32: each warp owns block-rows (lane = row) and keeps their
// values in registers.  A row's value is published to a work buffer the moment
// it is final; the buffers start filled with a NaN sentinel that no
// computation produces, so a consumer knows a published value by its bits
// alone and applies rows as soon as they appear.  The critical path is one
// multiply-subtract per row.  Each entry sees the same sequence of rounded
// steps as the column-by-column algorithm, so the result is bitwise
// identical to it.
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
constexpr unsigned long long kSentinel = 0x7FF4DEADBEEF5EA1ull;   // a NaN payload no operation produces

// solve work buffer: [status | perm (int32 n) | y | x | d], y/x/d: w planes of n
constexpr size_t kSolveWsPerm = 256;
__host__ __device__ inline size_t solve_ws_y(int64_t n) {
  return (kSolveWsPerm + 4 * (size_t)n + 255) & ~(size_t)255;
}
__host__ __device__ inline size_t solve_vec_bytes(int w, int64_t n) {
  return (sizeof(double) * (size_t)w * (size_t)(n > 0 ? n : 1) + 255) & ~(size_t)255;
}
__host__ __device__ inline int64_t solve_nblk(int64_t n) { return (n + kSolveBlock - 1) / kSolveBlock; }

// n <= kMaxOrder (checked by every entry point before sizes are computed)
size_t solve_workspace_bytes(int w, int64_t n) { return solve_ws_y(n) + 3 * solve_vec_bytes(w, n); }

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

// reciprocals of the diagonal and the sentinel fill of the y/x buffers
template <int W>
__global__ void k_solve_prep(const double* __restrict__ LU, int64_t lda, int64_t plane, int64_t n,
                             char* __restrict__ ws) {
  double* y = reinterpret_cast<double*>(ws + solve_ws_y(n));
  double* xb = y + solve_vec_bytes(W, n) / sizeof(double);
  double* d = xb + solve_vec_bytes(W, n) / sizeof(double);
  const double sent = __longlong_as_double((long long)kSentinel);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    val<W> one;
#pragma unroll
    for (int c = 0; c < W; ++c) one.v[c] = 0.0;
    one.v[0] = 1.0;
    const val<W> dj = div<W, false>(one, load_ro<W>(LU, plane, q * lda + q));
    store<W>(d, n, q, dj);
#pragma unroll
    for (int c = 0; c < W; ++c) {
      y[c * n + q] = sent;
      xb[c * n + q] = sent;
    }
  }
}

__device__ __forceinline__ bool is_sent(double v) {
  return (unsigned long long)__double_as_longlong(v) == kSentinel;
}

// lanes [lo, hi) load a published value; returns the ballot of ready lanes
template <int W>
__device__ __forceinline__ unsigned poll_block(const double* buf, int64_t n, int64_t base, int lo, int hi, val<W>& v) {
  const int lane = threadIdx.x & 31;
  bool ok = false;
  if (lane >= lo && lane < hi) {
    ok = true;
#pragma unroll
    for (int c = 0; c < W; ++c) {
      v.v[c] = __ldcv(buf + c * n + base + lane);
      ok = ok && !is_sent(v.v[c]);
    }
  }
  return __ballot_sync(0xffffffffu, ok);
}

__device__ __forceinline__ bool spin_backoff(unsigned long long& spins, unsigned long long limit,
                                             DeviceStatus* status, int tag) {
  if (++spins > pick_limit(limit, kSpinLimit)) {
    if ((threadIdx.x & 31) == 0) {
      atomicExch(&status->timeout, 1u);
      atomicExch(&status->where, (unsigned)tag);
    }
    return false;
  }
  __nanosleep(32);
  return true;
}

// One warp per CTA; warp b owns block-rows b, b + G, b + 2G, ...
template <int W>
__global__ void __launch_bounds__(32)
k_solve(const double* __restrict__ LU, int64_t lda, int64_t plane, int64_t n,
        const double* b, double* x, char* __restrict__ ws, unsigned long long spin_limit) {
  DeviceStatus* status = reinterpret_cast<DeviceStatus*>(ws + kWsStatus);
  const int* perm = reinterpret_cast<const int*>(ws + kSolveWsPerm);
  double* y = reinterpret_cast<double*>(ws + solve_ws_y(n));
  double* xb = y + solve_vec_bytes(W, n) / sizeof(double);
  const double* d = xb + solve_vec_bytes(W, n) / sizeof(double);
  const int lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  const int64_t nblk = solve_nblk(n);

  // gather y = P b for every owned block-row (before anything is published,
  // so b may alias x)
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
      int done = 0;
      unsigned long long spins = 0;
      while (done < kSolveBlock) {
        val<W> v;
        const unsigned mask = poll_block<W>(y, n, J * kSolveBlock, done, kSolveBlock, v);
        const unsigned notready = ~(mask >> done);
        const int k = notready ? __ffs(notready) - 1 : kSolveBlock - done;
        if (k == 0) {
          if (!spin_backoff(spins, spin_limit, status, 31)) return;
          continue;
        }
        for (int jj = done; jj < done + k; ++jj) {
          const val<W> yj = shfl_val<W>(v, jj);
          if (row_ok) acc = msub<W, false>(acc, load_ro<W>(LU, plane, (J * kSolveBlock + jj) * lda + i), yj);
        }
        done += k;
      }
    }
    const int jb = (int)((n - I * kSolveBlock < kSolveBlock) ? n - I * kSolveBlock : kSolveBlock);
    for (int jj = 0; jj < jb; ++jj) {
      if (lane == jj) {
#pragma unroll
        for (int c = 0; c < W; ++c) __stcg(y + c * n + i, acc.v[c]);
      }
      const val<W> yj = shfl_val<W>(acc, jj);
      if (lane > jj && lane < jb) acc = msub<W, false>(acc, load_ro<W>(LU, plane, (I * kSolveBlock + jj) * lda + i), yj);
    }
    yr[q] = acc;
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
      const int jbJ = (int)((n - J * kSolveBlock < kSolveBlock) ? n - J * kSolveBlock : kSolveBlock);
      int done = jbJ;   // rows [0, done) of block J still to apply, from done-1 down
      unsigned long long spins = 0;
      while (done > 0) {
        val<W> v;
        const unsigned mask = poll_block<W>(xb, n, J * kSolveBlock, 0, done, v);
        const unsigned top = (done == 32) ? mask : (mask << (32 - done));
        int k = __clz(~top);
        if (k > done) k = done;
        if (k == 0) {
          if (!spin_backoff(spins, spin_limit, status, 32)) return;
          continue;
        }
        for (int jj = done - 1; jj >= done - k; --jj) {
          const val<W> xj = shfl_val<W>(v, jj);
          if (row_ok) acc = msub<W, false>(acc, load_ro<W>(LU, plane, (J * kSolveBlock + jj) * lda + i), xj);
        }
        done -= k;
      }
    }
    const int jb = (int)((n - I * kSolveBlock < kSolveBlock) ? n - I * kSolveBlock : kSolveBlock);
    for (int jj = jb - 1; jj >= 0; --jj) {
      if (lane == jj) {
        acc = mul<W, false>(acc, load_ro<W>(d, n, i));
#pragma unroll
        for (int c = 0; c < W; ++c) __stcg(xb + c * n + i, acc.v[c]);
      }
      const val<W> xj = shfl_val<W>(acc, jj);
      if (lane < jj) acc = msub<W, false>(acc, load_ro<W>(LU, plane, (I * kSolveBlock + jj) * lda + i), xj);
    }
    if (row_ok) {
#pragma unroll
      for (int c = 0; c < W; ++c) x[c * n + i] = acc.v[c];
    }
  }
}

int perm_launch(int64_t n, const int64_t* piv, int* perm, cudaStream_t s) {
  ProfScope ps(kPhPerm, s);
  const size_t shmem = (n <= kPermSmemMax) ? 8 * (size_t)n : 0;
  if (shmem > 48 * 1024) {
    MW_CUDA_CHECK(ensure_smem_limit(k_perm, shmem));
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
  int64_t G = std::min<int64_t>(nblk, 4 * (int64_t)device_sm_count());
  if (nblk > G * kSolveMaxOwned) return MW_EUNSUPPORTED;
  G = std::max<int64_t>(G, (nblk + kSolveMaxOwned - 1) / kSolveMaxOwned);
  MW_CUDA_CHECK(cudaMemsetAsync(ws, 0, kSolveWsPerm, s));
  {
    const int pg = (int)std::min<int64_t>((n + 255) / 256, 4 * (int64_t)device_sm_count());
    k_solve_prep<W><<<std::max(pg, 1), 256, 0, s>>>(LU, lda, plane, n, ws);
    MW_LAUNCH_CHECK();
  }
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
  MW_CUDA_CHECK(cudaLaunchKernelEx(&cfg, k_solve<W>, LU, lda, plane, n, b, x, ws, wait_limit()));
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
