// residual.cu -- the exact long residual, the exact solution update and the
// mixed precision iterative refinement loop (Section 2, Listing 1; stopping
// test Eq. (2)).
//
// Exact accumulation: a value is a signed fixed-point integer held as NL
// digits of 32 bits in 64-bit shared-memory slots (digit k weighs
// 2^(kLow + 32 k)).  Every binary64 word and every product of two words lies
// on this grid (the lowest bit of a product of subnormals is 2^-2148 and the
// highest below 2^2048), so deposits -- 64-bit shared-memory atomic adds of
// the digits of the shifted 106-bit integer product -- are exact, and the
// order in which threads deposit does not matter.  A slot absorbs 2^31
// deposits before it could overflow.  Reading back is greedy
// round-to-nearest (ties to even, subnormals and overflow as IEEE binary64):
// c_0 = RN(S), c_1 = RN(S - c_0), ... -- the unique canonical expansion.
#include <algorithm>
#include <cmath>
#include <cuda_runtime.h>

#include "mw_arith.cuh"
#include "mw_common.cuh"
#include "lu_internal.cuh"
#include "profile.cuh"
#include "exact_acc.cuh"

namespace mw {

// ---------------------------------------------------------------------------
// r = b - A x (exact), rounded greedily to r_words words
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kResThreads)
k_residual(int64_t n, const double* __restrict__ A, int64_t lda, int64_t plane, int a_words,
           const double* __restrict__ b, int b_words, const double* __restrict__ x, int x_words,
           double* __restrict__ r, int r_words) {
  __shared__ u64 acc[kRowsPerCta][kNL];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * kRowsPerCta;
  const int64_t i = i0 + lane;
  const bool row_ok = i < n;
  for (int e = threadIdx.x; e < kRowsPerCta * kNL; e += blockDim.x) (&acc[0][0])[e] = 0ull;
  __syncthreads();
  if (warp < b_words && row_ok) deposit_double(acc[lane], b[warp * n + i], 0, false);
  constexpr int NWARP = kResThreads / 32;
  for (int64_t j = warp; j < n; j += NWARP) {
    double xv[MW_LONG_WORDS];
#pragma unroll
    for (int d = 0; d < MW_LONG_WORDS; ++d) xv[d] = (d < x_words) ? __ldg(x + d * n + j) : 0.0;
    if (!row_ok) continue;
    for (int c = 0; c < a_words; ++c) {
      const double a = __ldg(A + c * plane + j * lda + i);
      if (zero_bits(a)) continue;
#pragma unroll
      for (int d = 0; d < MW_LONG_WORDS; ++d)
        if (d < x_words && !zero_bits(xv[d])) deposit_product(acc[lane], a, xv[d], 0, true);
    }
  }
  __syncthreads();
  if (warp == 0 && row_ok) {
    for (int c = 0; c < r_words; ++c) r[c * n + i] = acc_take(acc[lane]);
  }
}

int residual_launch(int64_t n, const double* A, int64_t lda, int a_words, const double* b,
                    int b_words, const double* x, int x_words, double* r, int r_words,
                    cudaStream_t s) {
  if (n == 0) return MW_OK;
  const int64_t plane = lda * n;
  ProfScope ps(kPhResidual, s);
  dim3 grid((unsigned)((n + kRowsPerCta - 1) / kRowsPerCta));
  k_residual<<<grid, kResThreads, 0, s>>>(n, A, lda, plane, a_words, b, b_words, x, x_words, r,
                                          r_words);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

// ---------------------------------------------------------------------------
// refinement helpers
// ---------------------------------------------------------------------------
struct RefineState {
  int er;            // exponent of max |r_0|
  int done;          // 1 converged, 2 stagnated, 0 continue
  double prev_corr;  // previous correction size (stop mode 1)
  double nA;         // ||A||_F from the leading words (stop mode 0)
  double last_corr;
  int rzero;         // residual exactly zero
  int pad;
};

__device__ double block_max_abs(const double* v, int64_t n) {
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(v[i]));
  for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
    red[0] = mm;
  }
  __syncthreads();
  const double res = red[0];
  __syncthreads();
  return res;
}

// ldexp(sqrt(RN(sum (v_i 2^-e)^2)), e) with e = ilogb(max|v_i|): exact sum
__device__ double block_norm2(const double* v, int64_t n, int64_t stride, u64* acc) {
  __shared__ double mx_s;
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(v[i * stride]));
  for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  __shared__ double red[32];
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  for (int k = threadIdx.x; k < kNL; k += blockDim.x) acc[k] = 0ull;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
    mx_s = mm;
  }
  __syncthreads();
  const double mx = mx_s;
  if (mx == 0.0) return 0.0;
  const int e = ilogb_pos(mx);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double t = v[i * stride];
    deposit_product(acc, t, t, -2 * e, false);
  }
  __syncthreads();
  __shared__ double res_s;
  if (threadIdx.x == 0) res_s = scale2(__dsqrt_rn(acc_take(acc)), e);
  __syncthreads();
  return res_s;
}

// ||A||_F over the leading words of the n x n matrix (stop mode 0)
__global__ void __launch_bounds__(1024) k_normA(int64_t n, const double* __restrict__ A, int64_t lda,
                                                RefineState* st) {
  __shared__ u64 acc[kNL];
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t q = threadIdx.x; q < n * n; q += blockDim.x) m = fmax(m, fabs(A[(q / n) * lda + q % n]));
  for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  for (int k = threadIdx.x; k < kNL; k += blockDim.x) acc[k] = 0ull;
  __syncthreads();
  __shared__ double mx_s;
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
    mx_s = mm;
  }
  __syncthreads();
  if (mx_s == 0.0) {
    if (threadIdx.x == 0) st->nA = 0.0;
    return;
  }
  const int e = ilogb_pos(mx_s);
  for (int64_t q = threadIdx.x; q < n * n; q += blockDim.x) {
    const double t = A[(q / n) * lda + q % n];
    deposit_product(acc, t, t, -2 * e, false);
  }
  __syncthreads();
  if (threadIdx.x == 0) st->nA = scale2(__dsqrt_rn(acc_take(acc)), e);
}

// after a residual: exponent e of max|r_0|, the Eq. (2) test (mode 0), and
// r_hat = first `inner` words of 2^-e r
__global__ void __launch_bounds__(1024)
k_refine_check(int64_t n, const double* __restrict__ r, const double* __restrict__ x, int inner,
               double* __restrict__ rhat, int stop_mode, double rtol, double atol,
               RefineState* st) {
  __shared__ u64 acc[kNL];
  const double rmax = block_max_abs(r, n);
  if (rmax == 0.0) {
    if (threadIdx.x == 0) {
      st->rzero = 1;
      st->done = 1;
    }
    return;
  }
  const int er = ilogb_pos(rmax);
  if (stop_mode == MW_STOP_EQ2) {
    const double nr = block_norm2(r, n, 1, acc);
    const double nx = block_norm2(x, n, 1, acc);
    if (threadIdx.x == 0) {
      double rhs = __dmul_rn(__dsqrt_rn((double)n), rtol);
      rhs = __dmul_rn(rhs, st->nA);
      rhs = __dmul_rn(rhs, nx);
      rhs = __dadd_rn(rhs, atol);
      st->done = (nr <= rhs) ? 1 : 0;
    }
  }
  if (threadIdx.x == 0) {
    st->er = er;
    st->rzero = 0;
  }
  for (int64_t q = threadIdx.x; q < (int64_t)inner * n; q += blockDim.x) rhat[q] = scale2(r[q], -er);
}

// x = RN_xw(x + 2^e z) exactly, one thread per entry (accumulator in shared memory)
__global__ void __launch_bounds__(kRowsPerCta)
k_update(int64_t n, double* __restrict__ x, int x_words, const double* __restrict__ z, int inner,
         const RefineState* __restrict__ st) {
  __shared__ u64 acc[kRowsPerCta][kNL];
  const int64_t i = (int64_t)blockIdx.x * kRowsPerCta + threadIdx.x;
  u64* a = acc[threadIdx.x];
  for (int k = 0; k < kNL; ++k) a[k] = 0ull;
  if (i >= n) return;
  const int e = st->er;
  for (int c = 0; c < x_words; ++c) deposit_double(a, x[c * n + i], 0, false);
  for (int c = 0; c < inner; ++c) deposit_double(a, z[c * n + i], e, false);
  for (int c = 0; c < x_words; ++c) x[c * n + i] = acc_take(a);
}

// stop mode 1 after an update: correction size vs 2^-(tb+2) ||x||_inf
__global__ void __launch_bounds__(1024)
k_refine_check2(int64_t n, const double* __restrict__ z, const double* __restrict__ x, int target_bits,
                int corrections, RefineState* st) {
  const double zmax = block_max_abs(z, n);
  const double xmax = block_max_abs(x, n);
  if (threadIdx.x == 0) {
    const double corr = scale2(zmax, st->er);
    const double lim = scale2(xmax, -target_bits - 2);
    int done = 0;
    if (corr <= lim) done = 1;
    else if (corrections >= 2 && corr > __dmul_rn(0.5, st->prev_corr)) done = 2;
    st->prev_corr = corr;
    st->last_corr = corr;
    st->done = done;
  }
}

// x (x_words planes) = z (inner planes) padded with zero words
__global__ void k_promote(int64_t n, double* __restrict__ x, int x_words, const double* __restrict__ z, int inner) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)x_words * n) return;
  const int c = (int)(q / n);
  x[q] = (c < inner) ? z[q] : 0.0;
}

// first `inner` planes of a (src_words planes, lda x n) into dst (inner planes)
__global__ void k_take_words_mat(int64_t n, const double* __restrict__ src, int64_t lda, int src_words,
                                 double* __restrict__ dst, int inner) {
  const int64_t plane = lda * n;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= plane) return;
  for (int c = 0; c < inner; ++c) dst[c * plane + q] = (c < src_words) ? src[c * plane + q] : 0.0;
}

__global__ void k_take_words_vec(int64_t n, const double* __restrict__ src, int src_words,
                                 double* __restrict__ dst, int inner) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)inner * n) return;
  const int c = (int)(q / n);
  dst[q] = (c < src_words) ? src[q] : 0.0;
}

// ---------------------------------------------------------------------------
// refine driver
// ---------------------------------------------------------------------------
int perm_launch(int64_t n, const int64_t* piv, int* perm, cudaStream_t s);
template <int W>
int solve_with_perm(int64_t n, const double* LU, int64_t lda, const double* b, double* x,
                    char* ws, cudaStream_t s);

struct RefineMap {
  size_t lu_ws, solve_ws, lu, piv, info, r, z, rhat, state, total;
};

static RefineMap refine_map(int inner, int update, int64_t n, int64_t lda) {
  RefineMap m;
  size_t off = 0;
  m.lu_ws = off;
  off += align256(lu_workspace_bytes(update, n));
  m.solve_ws = off;
  off += align256(solve_workspace_bytes(inner, n));
  m.lu = off;
  off += align256(sizeof(double) * (size_t)inner * (size_t)lda * (size_t)(n > 0 ? n : 1));
  m.piv = off;
  off += align256(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  m.info = off;
  off += 256;
  m.r = off;
  off += align256(sizeof(double) * MW_LONG_WORDS * (size_t)(n > 0 ? n : 1));
  m.z = off;
  off += align256(sizeof(double) * (size_t)inner * (size_t)(n > 0 ? n : 1));
  m.rhat = off;
  off += align256(sizeof(double) * (size_t)inner * (size_t)(n > 0 ? n : 1));
  m.state = off;
  off += 256;
  m.total = off;
  return m;
}

size_t refine_workspace_bytes(int inner, int update, int64_t n) {
  // the LU copy uses lda = n
  return refine_map(inner, update, n, n > 0 ? n : 1).total;
}

template <int W>
static int refine_impl(int64_t n, const double* A, int64_t lda, int a_words, const double* b, int b_words,
                       int update, int target_bits, int max_iter, int stop_mode, double rtol, double atol,
                       double* x, int x_words, int64_t* stats, char* ws, size_t ws_bytes, cudaStream_t s) {
  const int64_t ldl = n;
  const RefineMap m = refine_map(W, update, n, ldl);
  if (ws_bytes < m.total) return -17;
  double* LU = reinterpret_cast<double*>(ws + m.lu);
  int64_t* piv = reinterpret_cast<int64_t*>(ws + m.piv);
  int64_t* info_d = reinterpret_cast<int64_t*>(ws + m.info);
  double* r = reinterpret_cast<double*>(ws + m.r);
  double* z = reinterpret_cast<double*>(ws + m.z);
  double* rhat = reinterpret_cast<double*>(ws + m.rhat);
  RefineState* st = reinterpret_cast<RefineState*>(ws + m.state);
  char* solve_ws = ws + m.solve_ws;
  stats[0] = stats[1] = stats[2] = 0;
  stats[3] = MW_OK;
  if (n == 0) return MW_OK;
  // LU copy (lda = n) of the first W words of A
  if (lda == n) {
    prof_count(kPhRefineAux);
  k_take_words_mat<<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(n, A, lda, a_words, LU, W);
    MW_LAUNCH_CHECK();
  } else {
    for (int c = 0; c < W; ++c) {
      if (c < a_words) {
        MW_CUDA_CHECK(cudaMemcpy2DAsync(LU + (size_t)c * n * n, sizeof(double) * n, A + (size_t)c * lda * n,
                                        sizeof(double) * lda, sizeof(double) * n, n, cudaMemcpyDeviceToDevice, s));
      } else {
        MW_CUDA_CHECK(cudaMemsetAsync(LU + (size_t)c * n * n, 0, sizeof(double) * n * n, s));
      }
    }
  }
  MW_CUDA_CHECK(cudaMemsetAsync(st, 0, sizeof(RefineState), s));
  const int nb = (update == MW_UPDATE_SPLIT) ? kDefaultNb : tune_get(MW_TUNE_PANEL_WIDTH, W);
  int rc = lu_blocked<W>(update, n, LU, ldl, piv, info_d, ws + m.lu_ws, m.solve_ws - m.lu_ws, nb, s);
  if (rc) return rc;
  int64_t info = 0;
  DeviceStatus lu_st[2] = {};
  MW_CUDA_CHECK(cudaMemcpyAsync(&info, info_d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  MW_CUDA_CHECK(cudaMemcpyAsync(&lu_st[0], ws + m.lu_ws + kWsStatus, sizeof(DeviceStatus), cudaMemcpyDeviceToHost, s));
  if (update == MW_UPDATE_SPLIT)
    MW_CUDA_CHECK(cudaMemcpyAsync(&lu_st[1], ws + m.lu_ws + kWsSplit + kWsStatus, sizeof(DeviceStatus),
                                  cudaMemcpyDeviceToHost, s));
  MW_CUDA_CHECK(cudaStreamSynchronize(s));
  stats[2] = info;
  if (lu_st[0].timeout || lu_st[1].timeout) {   // a bounded wait of the LU gave up
    stats[3] = MW_ETIMEOUT;
    return MW_ETIMEOUT;
  }
  if (info != 0) {
    stats[3] = MW_ESINGULAR;
    return MW_ESINGULAR;
  }
  rc = perm_launch(n, piv, reinterpret_cast<int*>(solve_ws + 256), s);
  if (rc) return rc;
  prof_count(kPhRefineAux);
  k_take_words_vec<<<(unsigned)((W * n + 255) / 256), 256, 0, s>>>(n, b, b_words, rhat, W);
  MW_LAUNCH_CHECK();
  rc = solve_with_perm<W>(n, LU, ldl, rhat, z, solve_ws, s);
  if (rc) return rc;
  prof_count(kPhRefineAux);
  k_promote<<<(unsigned)((x_words * n + 255) / 256), 256, 0, s>>>(n, x, x_words, z, W);
  MW_LAUNCH_CHECK();
  if (stop_mode == MW_STOP_EQ2) {
    prof_count(kPhRefineAux);
  k_normA<<<1, 1024, 0, s>>>(n, A, lda, st);
    MW_LAUNCH_CHECK();
  }
  int corrections = 0, residuals = 0, status = MW_ENOTCONV;
  RefineState h;
  DeviceStatus sv = {};
  for (;;) {
    rc = residual_launch(n, A, lda, a_words, b, b_words, x, x_words, r, x_words, s);
    if (rc) return rc;
    residuals++;
    prof_count(kPhRefineAux);
  k_refine_check<<<1, 1024, 0, s>>>(n, r, x, W, rhat, stop_mode, rtol, atol, st);
    MW_LAUNCH_CHECK();
    MW_CUDA_CHECK(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
    MW_CUDA_CHECK(cudaMemcpyAsync(&sv, solve_ws + kWsStatus, sizeof(sv), cudaMemcpyDeviceToHost, s));
    MW_CUDA_CHECK(cudaStreamSynchronize(s));
    if (sv.timeout) {   // the last substitution's bounded wait gave up
      status = MW_ETIMEOUT;
      break;
    }
    if (h.rzero || (stop_mode == MW_STOP_EQ2 && h.done == 1)) {
      status = MW_OK;
      break;
    }
    if (corrections >= max_iter) break;
    rc = solve_with_perm<W>(n, LU, ldl, rhat, z, solve_ws, s);
    if (rc) return rc;
    prof_count(kPhRefineAux);
  k_update<<<(unsigned)((n + kRowsPerCta - 1) / kRowsPerCta), kRowsPerCta, 0, s>>>(n, x, x_words, z, W, st);
    MW_LAUNCH_CHECK();
    corrections++;
    if (stop_mode == MW_STOP_BITS) {
      prof_count(kPhRefineAux);
  k_refine_check2<<<1, 1024, 0, s>>>(n, z, x, target_bits, corrections, st);
      MW_LAUNCH_CHECK();
      MW_CUDA_CHECK(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
      MW_CUDA_CHECK(cudaMemcpyAsync(&sv, solve_ws + kWsStatus, sizeof(sv), cudaMemcpyDeviceToHost, s));
      MW_CUDA_CHECK(cudaStreamSynchronize(s));
      if (sv.timeout) {
        status = MW_ETIMEOUT;
        break;
      }
      if (h.done == 1) {
        status = MW_OK;
        break;
      }
      if (h.done == 2) break;
    }
  }
  stats[0] = corrections;
  stats[1] = residuals;
  stats[3] = status;
  return status;
}

int refine_dispatch(int64_t n, const double* A, int64_t lda, int a_words, const double* b, int b_words,
                    int inner, int update, int target_bits, int max_iter, int stop_mode, double rtol,
                    double atol, double* x, int x_words, int64_t* stats, char* ws, size_t ws_bytes,
                    cudaStream_t s) {
  switch (inner) {
    case 2: return refine_impl<2>(n, A, lda, a_words, b, b_words, update, target_bits, max_iter, stop_mode, rtol, atol, x, x_words, stats, ws, ws_bytes, s);
    case 3: return refine_impl<3>(n, A, lda, a_words, b, b_words, update, target_bits, max_iter, stop_mode, rtol, atol, x, x_words, stats, ws, ws_bytes, s);
    case 4: return refine_impl<4>(n, A, lda, a_words, b, b_words, update, target_bits, max_iter, stop_mode, rtol, atol, x, x_words, stats, ws, ws_bytes, s);
  }
  return -7;
}

}  // namespace mw
