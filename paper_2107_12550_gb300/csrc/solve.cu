// solve.cu -- forward/back substitution with the factors of the blocked LU
// (Section 2, Listing 1: SolveTDLSPM).
//
// y = P b; y_i -= l_ij y_j (j ascending); x_j = y_j / u_jj and
// y_i -= u_ij x_j (j descending).  One cooperative launch walks the columns
// in blocks of 32: warp 0 of CTA 0 solves the 32 x 32 diagonal block with
// shuffles, then every CTA applies the block's 32 updates, in order, to the
// rows below (forward) or above (back) it.  Each entry sees the same
// sequence of rounded multiply-subtract steps as the column-by-column
// algorithm, so the result is bitwise identical to it.
#include <algorithm>
#include <cuda_runtime.h>

#include "mw_arith.cuh"
#include "mw_common.cuh"
#include "lu_internal.cuh"
#include "profile.cuh"

namespace mw {

constexpr int kSolveThreads = 256;
constexpr int kSolveBlock = 32;
constexpr int64_t kPermSmemMax = 26 * 1024;   // pivots handled in shared memory up to here

// solve work buffer: [barrier | status | perm (int32 n) | y (w planes of n)]
constexpr size_t kSolveWsPerm = 256;
__host__ __device__ inline size_t solve_ws_y(int64_t n) {
  return (kSolveWsPerm + 4 * (size_t)n + 255) & ~(size_t)255;
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

template <int W>
__global__ void __launch_bounds__(kSolveThreads)
k_solve(const double* __restrict__ LU, int64_t lda, int64_t plane, int64_t n,
        const double* b, double* x, char* __restrict__ ws) {
  GridBarrier* bar = reinterpret_cast<GridBarrier*>(ws + kWsBarrier);
  DeviceStatus* status = reinterpret_cast<DeviceStatus*>(ws + kWsStatus);
  const int* perm = reinterpret_cast<const int*>(ws + kSolveWsPerm);
  double* y = reinterpret_cast<double*>(ws + solve_ws_y(n));
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double sblk[W][kSolveBlock];

  // y = P b
  for (int64_t i = gtid; i < n; i += gthreads) {
    const int src = perm[i];
#pragma unroll
    for (int c = 0; c < W; ++c) __stcg(y + c * n + i, b[c * n + src]);
  }
  if (!grid_sync(bar, status, 11)) return;

  // forward: unit lower L
  for (int64_t J0 = 0; J0 < n; J0 += kSolveBlock) {
    const int jb = (int)((n - J0 < kSolveBlock) ? n - J0 : kSolveBlock);
    if (blockIdx.x == 0 && warp == 0) {
      const int64_t i = J0 + lane;
      val<W> yv;
      if (lane < jb) yv = load_cg<W>(y, n, i);
      else {
#pragma unroll
        for (int c = 0; c < W; ++c) yv.v[c] = 0.0;
      }
      for (int jj = 0; jj < jb; ++jj) {
        const val<W> yj = shfl_val<W>(yv, jj);
        if (lane > jj && lane < jb) {
          const val<W> l = load_ro<W>(LU, plane, (J0 + jj) * lda + i);
          yv = msub<W>(yv, l, yj);
        }
      }
      if (lane < jb) store_cg<W>(y, n, i, yv);
    }
    if (!grid_sync(bar, status, 12)) return;
    const int64_t below = J0 + jb;
    if (below < n) {
      for (int e = threadIdx.x; e < W * jb; e += blockDim.x)
        sblk[e / jb][e % jb] = __ldcg(y + (e / jb) * n + J0 + (e % jb));
      __syncthreads();
      for (int64_t i = below + gtid; i < n; i += gthreads) {
        val<W> acc = load_cg<W>(y, n, i);
        for (int jj = 0; jj < jb; ++jj) {
          val<W> yj;
#pragma unroll
          for (int c = 0; c < W; ++c) yj.v[c] = sblk[c][jj];
          const val<W> l = load_ro<W>(LU, plane, (J0 + jj) * lda + i);
          acc = msub<W>(acc, l, yj);
        }
        store_cg<W>(y, n, i, acc);
      }
      __syncthreads();
      if (!grid_sync(bar, status, 13)) return;
    }
  }

  // back: upper U
  for (int64_t J1 = n; J1 > 0;) {
    const int64_t J0 = (J1 > kSolveBlock) ? J1 - kSolveBlock : 0;
    const int jb = (int)(J1 - J0);
    if (blockIdx.x == 0 && warp == 0) {
      const int64_t i = J0 + lane;
      val<W> yv;
      if (lane < jb) yv = load_cg<W>(y, n, i);
      else {
#pragma unroll
        for (int c = 0; c < W; ++c) yv.v[c] = 0.0;
      }
      for (int jj = jb - 1; jj >= 0; --jj) {
        if (lane == jj) {
          const val<W> ujj = load_ro<W>(LU, plane, (J0 + jj) * lda + i);
          yv = div<W>(yv, ujj);
        }
        const val<W> xj = shfl_val<W>(yv, jj);
        if (lane < jj) {
          const val<W> u = load_ro<W>(LU, plane, (J0 + jj) * lda + i);
          yv = msub<W>(yv, u, xj);
        }
      }
      if (lane < jb) store_cg<W>(y, n, i, yv);
    }
    if (!grid_sync(bar, status, 14)) return;
    if (J0 > 0) {
      for (int e = threadIdx.x; e < W * jb; e += blockDim.x)
        sblk[e / jb][e % jb] = __ldcg(y + (e / jb) * n + J0 + (e % jb));
      __syncthreads();
      for (int64_t i = gtid; i < J0; i += gthreads) {
        val<W> acc = load_cg<W>(y, n, i);
        for (int jj = jb - 1; jj >= 0; --jj) {
          val<W> xj;
#pragma unroll
          for (int c = 0; c < W; ++c) xj.v[c] = sblk[c][jj];
          const val<W> u = load_ro<W>(LU, plane, (J0 + jj) * lda + i);
          acc = msub<W>(acc, u, xj);
        }
        store_cg<W>(y, n, i, acc);
      }
      __syncthreads();
      if (!grid_sync(bar, status, 15)) return;
    }
    J1 = J0;
  }

  for (int64_t i = gtid; i < n; i += gthreads) {
#pragma unroll
    for (int c = 0; c < W; ++c) x[c * n + i] = __ldcg(y + c * n + i);
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
  int G = (int)std::min<int64_t>((n + kSolveThreads - 1) / kSolveThreads, sm_count_solve());
  G = std::max(G, 1);
  MW_CUDA_CHECK(cudaMemsetAsync(ws, 0, kSolveWsPerm, s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kSolveThreads);
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
