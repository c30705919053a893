// lu.cu -- blocked right-looking LU decomposition with partial pivoting in
// DD/TD/QD (Section 2, Listing 1: TDLUdecompPM).
//
// For each panel of nb columns starting at k0:
//   1. k_panel  (cooperative): for each column k of the panel, a warp-shuffle
//      argmax of |a_ik| over rows i >= k across all CTAs, the row swap inside
//      the panel, the multipliers l_ik = a_ik / a_kk and the in-panel
//      updates a_ij -= l_ik u_kj.
//   2. the panel's row swaps on the columns left of it (one gather, k_swap_plan
//      and k_swap_apply), and k_trsm on the columns
//      right of it: the panel's row swaps, then U12 = L11^-1 A12.
//   3. the trailing update A22 -= L21 U12, either the plain multiword GEMM
//      on the FP64 pipe (k_gemm_plain, here) or the split-precision
//      tensor-core form (ozaki.cu).
// Every element a_ij receives its updates a_ij -= l_it u_tj in ascending t
// exactly as unblocked right-looking elimination applies them, with the same
// rounded multiply and subtraction, so the plain form is bitwise identical
// to unblocked elimination.
#include <algorithm>
#include <mutex>
#include <cuda_runtime.h>

#include "mw_arith.cuh"
#include "mw_common.cuh"
#include "lu_internal.cuh"
#include "profile.cuh"

namespace mw {

// ---------------------------------------------------------------------------
// panel factorisation
// ---------------------------------------------------------------------------
template <int W>
struct Cand {
  val<W> v;
  long long idx;  // -1: no candidate
};

template <int W>
__device__ __forceinline__ bool better(const val<W>& a, long long ia, const val<W>& b, long long ib) {
  if (ia < 0) return false;
  if (ib < 0) return true;
  const int c = cmp_abs<W>(a, b);
  return c > 0 || (c == 0 && ia < ib);
}

template <int W>
__device__ __forceinline__ void warp_argmax(val<W>& v, long long& idx) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    val<W> ov;
#pragma unroll
    for (int c = 0; c < W; ++c) ov.v[c] = __shfl_xor_sync(0xffffffffu, v.v[c], off);
    const long long oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (better<W>(ov, oi, v, idx)) {
      v = ov;
      idx = oi;
    }
  }
}

// Candidate record (in the work buffer, per column parity and CTA):
//   [0]             ready tag: k + 1 once the record of column k is complete
//   [1, 1+W)        candidate value words
//   [1+W]           candidate row index (as int64 bits)
//   [2+W, 2+W+W*nb) the candidate's whole panel row, word-major
// A CTA writes its record (and, if it owns row k, row k's old values after
// the records), then -- after a fence -- the tag with release semantics.
// Thread q of every CTA waits (bounded) for CTA q's tag with acquire
// semantics and reads its candidate: the tags are the column's only grid
// synchronisation.  A CTA writes the records of column k + 2 (same parity)
// only after reading every record of column k, and it reads them only after
// every CTA has written its column k + 1 record, so no record is overwritten
// while it is still being read.  Every CTA takes the pivot row from the
// winner's record, so it never has to be read from the matrix while its
// owner may be rewriting it; the owner of row k writes the pivot row into
// row k and the owner of the pivot row moves the old row k into its row.
//
// Each CTA owns the rows [r0, r1) of the panel.  With RES the CTA keeps its
// rows of all nb panel columns in shared memory from the first column to the
// last (read once, written back once); otherwise it works on them in global
// memory.  Every entry receives the same operations in the same order either
// way.
template <int W, bool RES>
struct PanelRows {
  double* A;
  int64_t lda, plane, k0, r0, chunk;
  double* sp;   // RES: [W][nb][chunk]
  int nb;
  __device__ __forceinline__ val<W> get(int64_t i, int j) const {
    val<W> v;
    if (RES) {
#pragma unroll
      for (int c = 0; c < W; ++c) v.v[c] = sp[((int64_t)c * nb + j) * chunk + (i - r0)];
    } else {
      v = load_cg<W>(A, plane, (k0 + j) * lda + i);
    }
    return v;
  }
  __device__ __forceinline__ double get1(int64_t i, int j, int c) const {
    if (RES) return sp[((int64_t)c * nb + j) * chunk + (i - r0)];
    return __ldcg(A + c * plane + (k0 + j) * lda + i);
  }
  __device__ __forceinline__ void put(int64_t i, int j, const val<W>& v) const {
    if (RES) {
#pragma unroll
      for (int c = 0; c < W; ++c) sp[((int64_t)c * nb + j) * chunk + (i - r0)] = v.v[c];
    } else {
      store_cg<W>(A, plane, (k0 + j) * lda + i, v);
    }
  }
};

template <int W>
struct CandC {
  val<W> v;
  long long idx;
  int cta;
};

template <int W, bool RES>
__global__ void __launch_bounds__(kPanelThreads)
k_panel(double* __restrict__ A, int64_t lda, int64_t plane, int64_t n, int64_t k0, int nb,
        int64_t* __restrict__ piv, int64_t* __restrict__ info, char* __restrict__ ws,
        unsigned long long spin_limit) {
  GridAbort* bar = reinterpret_cast<GridAbort*>(ws + kWsAbort);
  DeviceStatus* status = reinterpret_cast<DeviceStatus*>(ws + kWsStatus);

  const int G = gridDim.x;
  const int cta = blockIdx.x;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int64_t rows = n - k0;
  const int64_t chunk = (rows + G - 1) / G;
  const int64_t r0 = k0 + (int64_t)cta * chunk;
  const int64_t r1 = (r0 + chunk < n) ? r0 + chunk : n;
  const int64_t nown = (r1 > r0) ? r1 - r0 : 0;

  extern __shared__ double smem[];
  double* su = smem;                 // [W][nb]  pivot row u_kj (all panel columns)
  double* sl = smem + W * nb;        // [W][chunk]  multipliers of owned rows
  const PanelRows<W, RES> pr{A, lda, plane, k0, r0, chunk, sl + W * chunk, nb};
  __shared__ CandC<W> wred[kPanelThreads / 32];
  __shared__ long long s_piv;
  __shared__ int s_zero, s_wcta;
  constexpr int kRecVal = 1, kRecIdx = 1 + W, kRecRow = 2 + W;

  if (RES) {
    const int64_t per = (int64_t)nb * nown;
    for (int64_t e = tid; e < W * per; e += kPanelThreads) {
      const int c = (int)(e / per);
      const int64_t rem = e % per;
      const int j = (int)(rem / nown);
      const int64_t il = rem % nown;
      pr.sp[((int64_t)c * nb + j) * chunk + il] = __ldcg(A + c * plane + (k0 + j) * lda + r0 + il);
    }
    __syncthreads();
  }

  for (int kk = 0; kk < nb; ++kk) {
    const int64_t k = k0 + kk;
    double* rec_base = reinterpret_cast<double*>(ws + kWsCand + (size_t)(kk & 1) * kCandParity);
    double* rec = rec_base + (size_t)cta * (kCandStride / 8);
    double* oldk = rec_base + (size_t)kMaxPanelCtas * (kCandStride / 8);
    // (a) local argmax over owned rows i >= k
    val<W> bv;
#pragma unroll
    for (int c = 0; c < W; ++c) bv.v[c] = 0.0;
    long long bi = -1;
    for (int64_t i = (r0 > k ? r0 : k) + tid; i < r1; i += kPanelThreads) {
      const val<W> v = pr.get(i, kk);
      if (better<W>(v, i, bv, bi)) {
        bv = v;
        bi = i;
      }
    }
    warp_argmax<W>(bv, bi);
    if (lane == 0) {
      wred[warp].v = bv;
      wred[warp].idx = bi;
    }
    __syncthreads();
    // every thread combines the warps' candidates (integer comparisons), so
    // the row copy needs no second barrier
    long long brow;
    {
      CandC<W> b = wred[0];
      for (int w = 1; w < kPanelThreads / 32; ++w)
        if (better<W>(wred[w].v, wred[w].idx, b.v, b.idx)) b = wred[w];
      if (tid == 0) {
#pragma unroll
        for (int c = 0; c < W; ++c) __stcg(rec + kRecVal + c, b.v.v[c]);
        __stcg(reinterpret_cast<long long*>(rec + kRecIdx), b.idx);
      }
      brow = b.idx;
    }
    // publish the candidate's whole panel row, and old row k if this CTA owns it
    {
      const bool own_k = (k >= r0 && k < r1);
      for (int e = tid; e < W * nb; e += kPanelThreads) {
        const int c = e / nb, j = e % nb;
        if (brow >= 0) __stcg(rec + kRecRow + e, pr.get1(brow, j, c));
        if (own_k) __stcg(oldk + e, pr.get1(k, j, c));
      }
    }
    __syncthreads();
    // the barrier orders the CTA's record stores before tid 0's release
    // store, which is cumulative over them (gpu scope)
    const unsigned long long tag = (unsigned long long)k + 1ull;
    if (tid == 0) st_release_u64(rec, tag);
    // (b) global argmax: thread q waits for CTA q's record and reads its
    // candidate (every CTA computes the same)
    {
      val<W> gv;
#pragma unroll
      for (int c = 0; c < W; ++c) gv.v[c] = 0.0;
      long long gi = -1;
      int gc = -1;
      int failed = 0;
      if (tid < G) {
        const double* rq = rec_base + (size_t)tid * (kCandStride / 8);
        unsigned long long spins = 0;
        while (ld_acquire_u64(rq) != tag) {
          if (++spins > pick_limit(spin_limit, kSpinLimit) || ld_acquire_u32(&bar->abort)) {
            failed = 1;
            break;
          }
          if (spins > 64) __nanosleep(32);
        }
        if (!failed) {
#pragma unroll
          for (int c = 0; c < W; ++c) gv.v[c] = __ldcg(rq + kRecVal + c);
          gi = __ldcg(reinterpret_cast<const long long*>(rq + kRecIdx));
          gc = tid;
        }
      }
      if (__syncthreads_or(failed)) {
        if (tid == 0) {
          atomicExch(&bar->abort, 1u);
          atomicExch(&status->timeout, 1u);
          atomicExch(&status->where, 1u);
        }
        return;
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        val<W> ov;
#pragma unroll
        for (int c = 0; c < W; ++c) ov.v[c] = __shfl_xor_sync(0xffffffffu, gv.v[c], off);
        const long long oi = __shfl_xor_sync(0xffffffffu, gi, off);
        const int oc = __shfl_xor_sync(0xffffffffu, gc, off);
        if (better<W>(ov, oi, gv, gi)) {
          gv = ov;
          gi = oi;
          gc = oc;
        }
      }
      if (lane == 0) {
        wred[warp].v = gv;
        wred[warp].idx = gi;
        wred[warp].cta = gc;
      }
      __syncthreads();
      if (tid == 0) {
        CandC<W> b = wred[0];
        for (int w = 1; w < kPanelThreads / 32; ++w)
          if (better<W>(wred[w].v, wred[w].idx, b.v, b.idx)) b = wred[w];
        s_piv = b.idx;
        s_wcta = b.cta;
        s_zero = is_zero<W>(b.v) ? 1 : 0;
      }
      __syncthreads();
    }
    const int64_t p = s_piv;
    if (cta == 0 && tid == 0) {
      piv[k] = p;
      if (s_zero && *info == 0) *info = k + 1;
    }
    // (c) pivot row from the winner's record; swap rows k and p
    {
      const double* wrec = rec_base + (size_t)s_wcta * (kCandStride / 8) + kRecRow;
      for (int e = tid; e < W * nb; e += kPanelThreads) su[e] = __ldcg(wrec + e);
      __syncthreads();
      if (p != k) {
        const bool own_k = (k >= r0 && k < r1);
        const bool own_p = (p >= r0 && p < r1);
        for (int j = tid; j < nb; j += kPanelThreads) {
          val<W> vk, vp;
#pragma unroll
          for (int c = 0; c < W; ++c) {
            vk.v[c] = su[c * nb + j];
            vp.v[c] = __ldcg(oldk + c * nb + j);
          }
          if (own_k) pr.put(k, j, vk);
          if (own_p) pr.put(p, j, vp);
        }
      }
      __syncthreads();
    }
    // (d) multipliers and in-panel update of owned rows i > k
    val<W> akk;
#pragma unroll
    for (int c = 0; c < W; ++c) akk.v[c] = su[c * nb + kk];
    const bool zero = is_zero<W>(akk);
    const int64_t ilo = (r0 > k + 1) ? r0 : k + 1;
    for (int64_t i = ilo + tid; i < r1; i += kPanelThreads) {
      val<W> a = pr.get(i, kk);
      if (!zero) {
        a = div<W, false>(a, akk);
        pr.put(i, kk, a);
      }
#pragma unroll
      for (int c = 0; c < W; ++c) sl[c * chunk + (i - r0)] = a.v[c];
    }
    __syncthreads();
    const int64_t nrows = r1 - ilo;
    const int ncols = nb - kk - 1;
    if (nrows > 0 && ncols > 0) {
      const int64_t items = nrows * ncols;
      for (int64_t q = tid; q < items; q += kPanelThreads) {
        const int64_t i = ilo + q % nrows;
        const int j = kk + 1 + (int)(q / nrows);
        val<W> l, u;
#pragma unroll
        for (int c = 0; c < W; ++c) {
          l.v[c] = sl[c * chunk + (i - r0)];
          u.v[c] = su[c * nb + j];
        }
        val<W> a = pr.get(i, j);
        a = msub<W, false>(a, l, u);
        pr.put(i, j, a);
      }
    }
    __syncthreads();
  }
  if (RES) {
    const int64_t per = (int64_t)nb * nown;
    for (int64_t e = tid; e < W * per; e += kPanelThreads) {
      const int c = (int)(e / per);
      const int64_t rem = e % per;
      const int j = (int)(rem / nown);
      const int64_t il = rem % nown;
      __stcg(A + c * plane + (k0 + j) * lda + r0 + il, pr.sp[((int64_t)c * nb + j) * chunk + il]);
    }
  }
}

// ---------------------------------------------------------------------------
// row interchanges as a gather (SwapPlan): one warp composes the swaps
// (k0 + kk, piv[k0 + kk]), kk in [lo, hi), in order into the contents of the
// block rows [k0 + lo, k0 + hi) and of the rows below them that the swaps
// reach; then one warp per column and word loads every source and stores
// every destination.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void build_swap_plan(const int64_t* __restrict__ pv, int k0, int lo, int hi,
                                                SwapPlan* __restrict__ plan) {
  __shared__ int blk[kMaxNb], orow[kMaxNb], ocont[kMaxNb];
  const int lane = threadIdx.x & 31;
  const int nbk = hi - lo;
  const int base = k0 + lo;
  for (int q = lane; q < nbk; q += 32) blk[q] = base + q;
  __syncwarp();
  int m = 0;
  for (int kk = 0; kk < nbk; ++kk) {
    const int p = (int)pv[base + kk];
    if (p < base + nbk) {
      if (lane == 0 && p != base + kk) {
        const int t = blk[kk];
        blk[kk] = blk[p - base];
        blk[p - base] = t;
      }
    } else {
      int found = -1;
      for (int e = lane; e < m; e += 32)
        if (orow[e] == p) found = e;
      const unsigned hit = __ballot_sync(0xffffffffu, found >= 0);
      const int idx = hit ? __shfl_sync(0xffffffffu, found, __ffs(hit) - 1) : -1;
      if (lane == 0) {
        if (idx >= 0) {
          const int t = blk[kk];
          blk[kk] = ocont[idx];
          ocont[idx] = t;
        } else {
          orow[m] = p;
          ocont[m] = blk[kk];
          blk[kk] = p;
        }
      }
      if (idx < 0) ++m;
    }
    __syncwarp();
  }
  for (int q = lane; q < nbk; q += 32) plan->pairs[q] = make_int2(base + q, blk[q]);
  for (int e = lane; e < m; e += 32) plan->pairs[nbk + e] = make_int2(orow[e], ocont[e]);
  if (lane == 0) plan->count = nbk + m;
}

__device__ __forceinline__ void apply_swap_plan(double* __restrict__ col, const SwapPlan* __restrict__ plan) {
  constexpr int Q = 2 * kMaxNb / 32;
  const int lane = threadIdx.x & 31;
  const int cnt = plan->count;
  double v[Q];
  int dst[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int e = lane + 32 * q;
    if (e < cnt) {
      const int2 pr = plan->pairs[e];
      v[q] = col[pr.y];
      dst[q] = pr.x;
    }
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int e = lane + 32 * q;
    if (e < cnt) col[dst[q]] = v[q];
  }
}

__global__ void __launch_bounds__(32)
k_swap_plan(const int64_t* __restrict__ piv, int k0, int nb, SwapPlan* __restrict__ plan) {
  build_swap_plan(piv, k0, 0, nb, plan);
}

// 8 columns per CTA (one warp each), blockIdx.y = word
template <int W>
__global__ void __launch_bounds__(256)
k_swap_apply(double* __restrict__ A, int64_t lda, int64_t plane, int64_t c_begin, int64_t c_end,
             const SwapPlan* __restrict__ plan) {
  const int64_t j = c_begin + (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= c_end) return;   // uniform per warp
  apply_swap_plan(A + blockIdx.y * plane + j * lda, plan);
}

static int swap_gather(double* A, int64_t lda, int64_t plane, int W, int64_t n, int64_t k0, int kb,
                       const int64_t* piv, char* ws, bool left, bool right, cudaStream_t s);

// ---------------------------------------------------------------------------
// row interchanges + U12 = L11^-1 A12 on 8 columns per CTA.
// Thread (c, g): column j = j0 + c (c = tid % 8), rows r = q * 32 + g
// (g = tid / 8).  Step t: the owner of row t publishes u_tj through shared
// memory; every thread then updates its rows r > t.
// ---------------------------------------------------------------------------
template <int W, int NB, bool I = true>
__device__ __forceinline__ void trsm_cols(double* __restrict__ A, int64_t lda, int64_t plane, int64_t n,
                                          int64_t k0, const int64_t* __restrict__ piv, int64_t cblock) {
  constexpr int TC = 8;
  constexpr int NG = 256 / TC;
  constexpr int RPT = (NB + NG - 1) / NG;
  const int c = threadIdx.x % TC, g = threadIdx.x / TC;
  const int64_t j = k0 + NB + cblock * TC + c;
  const bool active = j < n;
  __shared__ double su[2][W][TC];
  if (active && g < W) {
    double* col = A + g * plane + j * lda;
    for (int kk = 0; kk < NB; ++kk) {
      const int64_t k = k0 + kk;
      const int64_t p = piv[k];
      if (p != k) {
        const double a = col[k];
        col[k] = col[p];
        col[p] = a;
      }
    }
  }
  __syncthreads();
  val<W> a[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int r = q * NG + g;
    if (active && r < NB) a[q] = load<W>(A, plane, j * lda + k0 + r);
    else {
#pragma unroll
      for (int cc = 0; cc < W; ++cc) a[q].v[cc] = 0.0;
    }
  }
#pragma unroll
  for (int qt = 0; qt < RPT; ++qt) {
    for (int gg = 0; gg < NG; ++gg) {
      const int t = qt * NG + gg;
      if (t >= NB) break;
      const int buf = t & 1;
      if (g == gg) {
#pragma unroll
        for (int cc = 0; cc < W; ++cc) su[buf][cc][c] = a[qt].v[cc];
      }
      __syncthreads();
      val<W> u;
#pragma unroll
      for (int cc = 0; cc < W; ++cc) u.v[cc] = su[buf][cc][c];
      const int64_t lcol = (k0 + t) * lda + k0;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = q * NG + g;
        if (q >= qt && r > t && r < NB) {
          const val<W> l = load_ro<W>(A, plane, lcol + r);
          a[q] = msub<W, I>(a[q], l, u);
        }
      }
    }
  }
  if (active) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int r = q * NG + g;
      if (r < NB) store<W>(A, plane, j * lda + k0 + r, a[q]);
    }
  }
}

template <int W, int NB>
__global__ void __launch_bounds__(256)
k_trsm(double* __restrict__ A, int64_t lda, int64_t plane, int64_t n, int64_t k0,
       const int64_t* __restrict__ piv) {
  trsm_cols<W, NB, false>(A, lda, plane, n, k0, piv, blockIdx.x);
}

// ---------------------------------------------------------------------------
// batched blocked LU: the same panel / laswp / TRSM / trailing-update steps,
// for every system of a batch that is still active at panel step k0
// ---------------------------------------------------------------------------

// one CTA per active system: columns [k0, k0+kb) of rows [k0, n), column by
// column (argmax, swap inside the panel, multipliers, in-panel update)
// dynamic shared memory: pivot row [W][kBatchNb] and multipliers [W][nmax]
template <int W>
__global__ void __launch_bounds__(kPanelThreads, 4)
k_bpanel(BatchView bv, int nmax, int kp, int width, double* __restrict__ A, int64_t* __restrict__ piv,
         int64_t* __restrict__ info) {
  extern __shared__ double bsm[];
  double* su = bsm;                  // [W][kBatchNb]
  double* sl = bsm + W * kBatchNb;   // [W][nmax], rows relative to k0
  __shared__ Cand<W> wred[kPanelThreads / 32];
  __shared__ long long s_p;
  __shared__ int s_zero;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sys = bv.order[blockIdx.x];
  const int n = bv.n[sys];
  const int k0 = kp;                  // first column (and row) of this panel
  const int kb = min(width, n - k0);
  if (kb <= 0) return;                // uniform per CTA
  double* a = A + (int64_t)W * bv.moff[sys];
  const int64_t plane = (int64_t)n * n;
  int64_t* pv = piv + bv.voff[sys];
  int64_t inf = (k0 == 0) ? 0 : info[sys];
  for (int kk = 0; kk < kb; ++kk) {
    const int k = k0 + kk;
    const int64_t colk = (int64_t)k * n;
    val<W> bvv;
#pragma unroll
    for (int c = 0; c < W; ++c) bvv.v[c] = 0.0;
    long long bi = -1;
    for (int i = k + tid; i < n; i += kPanelThreads) {
      const val<W> v = load<W>(a, plane, colk + i);
      if (better<W>(v, i, bvv, bi)) {
        bvv = v;
        bi = i;
      }
    }
    warp_argmax<W>(bvv, bi);
    if (lane == 0) {
      wred[warp].v = bvv;
      wred[warp].idx = bi;
    }
    __syncthreads();
    if (tid == 0) {
      Cand<W> b = wred[0];
      for (int w = 1; w < kPanelThreads / 32; ++w)
        if (better<W>(wred[w].v, wred[w].idx, b.v, b.idx)) b = wred[w];
      s_p = b.idx;
      s_zero = is_zero<W>(b.v) ? 1 : 0;
      pv[k] = b.idx;
    }
    __syncthreads();
    const int p = (int)s_p;
    if (s_zero && inf == 0) inf = k + 1;
    // swap rows k and p inside the panel; cache the new row k
    for (int e = tid; e < W * kb; e += kPanelThreads) {
      const int c = e / kb, j = e % kb;
      double* col = a + c * plane + (int64_t)(k0 + j) * n;
      const double x = col[k];
      const double y = col[p];
      if (p != k) {
        col[k] = y;
        col[p] = x;
      }
      su[c * kBatchNb + j] = (p != k) ? y : x;
    }
    __syncthreads();
    val<W> akk;
#pragma unroll
    for (int c = 0; c < W; ++c) akk.v[c] = su[c * kBatchNb + kk];
    const bool zero = is_zero<W>(akk);
    for (int i = k + 1 + tid; i < n; i += kPanelThreads) {
      val<W> l = load<W>(a, plane, colk + i);
      if (!zero) {
        l = div<W>(l, akk);
        store<W>(a, plane, colk + i, l);
      }
#pragma unroll
      for (int c = 0; c < W; ++c) sl[c * nmax + (i - k0)] = l.v[c];
    }
    __syncthreads();
    const int rows = n - k - 1;
    const int cols = kb - kk - 1;
    if (rows > 0 && cols > 0) {
      const int items = rows * cols;
      for (int q = tid; q < items; q += kPanelThreads) {
        const int i = k + 1 + q % rows;
        const int j = kk + 1 + q / rows;
        const int64_t idx = (int64_t)(k0 + j) * n + i;
        val<W> l, u;
#pragma unroll
        for (int c = 0; c < W; ++c) {
          l.v[c] = sl[c * nmax + (i - k0)];
          u.v[c] = su[c * kBatchNb + j];
        }
        val<W> x = load<W>(a, plane, idx);
        x = msub<W>(x, l, u);
        store<W>(a, plane, idx, x);
      }
    }
    __syncthreads();
  }
  if (tid == 0) info[sys] = inf;
}

// row swaps k0 + [sw_lo, min(sw_hi, kb)) on the columns
// [max(0, k0 + c_lo), min(n, k0 + c_hi)): CTA (pos, word, block of 128 columns)
template <int W>
__global__ void __launch_bounds__(128)
k_bswap(BatchView bv, int k0, int sw_lo, int sw_hi, int c_lo, int c_hi, double* __restrict__ A,
        const int64_t* __restrict__ piv) {
  const int sys = bv.order[blockIdx.x];
  const int n = bv.n[sys];
  const int kb = min(kBatchNb, n - k0);
  const int j0 = max(0, k0 + c_lo);
  const int j1 = min(n, k0 + c_hi);
  const int64_t j = (int64_t)j0 + (int64_t)blockIdx.z * blockDim.x + threadIdx.x;
  if (j >= j1) return;
  const int64_t plane = (int64_t)n * n;
  const int64_t* pv = piv + bv.voff[sys];
  double* col = A + (int64_t)W * bv.moff[sys] + blockIdx.y * plane + j * n;
  const int hi = min(sw_hi, kb);
  for (int kk = sw_lo; kk < hi; ++kk) {
    const int k = k0 + kk;
    const int p = (int)pv[k];
    if (p != k) {
      const double t = col[k];
      col[k] = col[p];
      col[p] = t;
    }
  }
}

// batched swap plans: one warp per active system
__global__ void __launch_bounds__(32)
k_bswap_plan(BatchView bv, int k0, int sw_lo, int sw_hi, const int64_t* __restrict__ piv,
             SwapPlan* __restrict__ plans) {
  const int sys = bv.order[blockIdx.x];
  const int n = bv.n[sys];
  const int kb = min(kBatchNb, n - k0);
  build_swap_plan(piv + bv.voff[sys], k0, sw_lo, max(sw_lo, min(sw_hi, kb)), plans + blockIdx.x);
}

// CTA (pos, word, block of 8 columns), one warp per column
template <int W>
__global__ void __launch_bounds__(256)
k_bswap_apply(BatchView bv, int k0, int c_lo, int c_hi, double* __restrict__ A, const SwapPlan* __restrict__ plans) {
  const int sys = bv.order[blockIdx.x];
  const int n = bv.n[sys];
  const int j0 = max(0, k0 + c_lo);
  const int j1 = min(n, k0 + c_hi);
  const int64_t j = (int64_t)j0 + (int64_t)blockIdx.z * 8 + (threadIdx.x >> 5);
  if (j >= j1) return;   // uniform per warp
  const int64_t plane = (int64_t)n * n;
  apply_swap_plan(A + (int64_t)W * bv.moff[sys] + blockIdx.y * plane + j * n, plans + blockIdx.x);
}

// inside the panel, block of 2H columns at column c0 = k0 + c_off: the top H
// rows of its right half get the swaps of the left half, then the unit
// lower H x H solve; CTA (pos, block of 8 columns)
template <int W, int H>
__global__ void __launch_bounds__(256)
k_btrsm_sub(BatchView bv, int c0, double* __restrict__ A, const int64_t* __restrict__ piv) {
  const int sys = bv.order[blockIdx.x];
  const int n = bv.n[sys];
  if (n - c0 - H <= 0) return;        // no right half: uniform per CTA
  // columns c0 + H + blockIdx.y * 8 + c < min(n, c0 + 2H) (trsm_cols checks the bound)
  trsm_cols<W, H>(A + (int64_t)W * bv.moff[sys], n, (int64_t)n * n, min(n, c0 + 2 * H), c0, piv + bv.voff[sys],
                  blockIdx.y);
}

// swaps + U12 = L11^-1 A12 on 8 columns: CTA (pos, column block)
template <int W>
__global__ void __launch_bounds__(256)
k_btrsm(BatchView bv, int k0, double* __restrict__ A, const int64_t* __restrict__ piv) {
  const int sys = bv.order[blockIdx.x];
  const int n = bv.n[sys];
  if ((int64_t)blockIdx.y * 8 >= (int64_t)n - k0 - kBatchNb) return;   // uniform per CTA
  trsm_cols<W, kBatchNb>(A + (int64_t)W * bv.moff[sys], n, (int64_t)n * n, n, k0, piv + bv.voff[sys],
                         blockIdx.y);
}


// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
template <int W>
int launch_panel(double* A, int64_t lda, int64_t plane, int64_t n, int64_t k0, int nb,
                 int64_t* piv, int64_t* info, char* ws, cudaStream_t s) {
  const int64_t rows = n - k0;
  const int rpc = std::max(1, tune_get(MW_TUNE_PANEL_ROWS_PER_CTA, W));
  int G = (int)std::min<int64_t>((rows + rpc - 1) / rpc, device_sm_count());
  G = std::max(1, std::min(G, kMaxPanelCtas));
  const int64_t chunk = (rows + G - 1) / G;
  // the CTA's rows of the panel stay in shared memory when they fit
  const size_t shmem_res = sizeof(double) * (size_t)W * ((size_t)nb + (size_t)chunk + (size_t)nb * (size_t)chunk);
  const bool res = shmem_res <= kPanelResidentMax;
  const size_t shmem = res ? shmem_res : sizeof(double) * (size_t)W * ((size_t)nb + (size_t)chunk);
  auto kern = res ? k_panel<W, true> : k_panel<W, false>;
  if (shmem > 48 * 1024) {
    MW_CUDA_CHECK(ensure_smem_limit(kern, shmem));
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kPanelThreads);
  cfg.dynamicSmemBytes = shmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MW_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, A, lda, plane, n, k0, nb, piv, info, ws, wait_limit()));
  return MW_OK;
}

template <int W>
static int launch_trsm(double* A, int64_t lda, int64_t plane, int64_t n, int64_t k0, int nb,
                       const int64_t* piv, cudaStream_t s) {
  const int64_t ncols = n - k0 - nb;
  if (ncols <= 0) return MW_OK;
  dim3 grid((unsigned)((ncols + 7) / 8));
  switch (nb) {
    case 32: k_trsm<W, 32><<<grid, 256, 0, s>>>(A, lda, plane, n, k0, piv); break;
    case 64: k_trsm<W, 64><<<grid, 256, 0, s>>>(A, lda, plane, n, k0, piv); break;
    case 128: k_trsm<W, 128><<<grid, 256, 0, s>>>(A, lda, plane, n, k0, piv); break;
    default: return MW_EUNSUPPORTED;
  }
  MW_LAUNCH_CHECK();
  return MW_OK;
}

// ---------------------------------------------------------------------------
// split-update DD LU of one system: per 64-column panel, the cooperative
// panel kernel, the swaps left and right of the panel, M = -(L11^-1)
// strictly lower (column-parallel), then U12 -= M U12 and A22 -= L21 U12 as
// split tensor-core products.  (The batched split path also factors the
// panel recursively; for one system the panel is bound by its per-column
// latency, and the extra launches and small products of the recursion cost
// more than the FP64 work they move.)
// ---------------------------------------------------------------------------
// the swaps piv[sk0 .. sk0 + ns) on the columns [c0, c1), as one gather
static int swap_gather_range(double* A, int64_t lda, int64_t plane, int64_t sk0, int ns, int64_t c0, int64_t c1,
                             const int64_t* piv, char* ws, cudaStream_t s) {
  if (ns <= 0 || c1 <= c0) return MW_OK;
  ProfScope ps(kPhLaswp, s);
  SwapPlan* plan = reinterpret_cast<SwapPlan*>(ws + kWsSwapPlan);
  k_swap_plan<<<1, 32, 0, s>>>(piv, (int)sk0, ns, plan);
  MW_LAUNCH_CHECK();
  dim3 grid((unsigned)((c1 - c0 + 7) / 8), 2);
  k_swap_apply<2><<<grid, 256, 0, s>>>(A, lda, plane, c0, c1, plan);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

// the panel [kp, kp + w) of the split LU, recursively: left half, the right
// half's top rows solved with the left half's unit lower triangle (and its
// swaps), its rows below updated by a split product (K = half width), right
// half, then the right half's swaps on the left half; leaves of `leaf`
// columns on the cooperative panel kernel
static int split_panel_rec(double* A, int64_t lda, int64_t plane, int64_t n, int64_t kp, int w, int leaf,
                           int64_t* piv, int64_t* info, char* ws, char* sws, size_t sbytes, cudaStream_t s) {
  w = (int)std::min<int64_t>(w, n - kp);
  if (w <= 0) return MW_OK;
  if (w <= leaf) {
    ProfScope ps(kPhPanel, s);
    return launch_panel<2>(A, lda, plane, n, kp, w, piv, info, ws, s);
  }
  const int h = (w > 32) ? 32 : (w > 16 ? 16 : 8);   // halves of 64 -> 32 -> 16 -> 8
  int rc = split_panel_rec(A, lda, plane, n, kp, h, leaf, piv, info, ws, sws, sbytes, s);
  if (rc) return rc;
  const int64_t lim = kp + w;   // right half: columns [kp + h, lim)
  {
    ProfScope ps(kPhPanel, s);
    dim3 grid((unsigned)((lim - kp - h + 7) / 8));
    switch (h) {
      case 32: k_trsm<2, 32><<<grid, 256, 0, s>>>(A, lda, plane, lim, kp, piv); break;
      case 16: k_trsm<2, 16><<<grid, 256, 0, s>>>(A, lda, plane, lim, kp, piv); break;
      default: k_trsm<2, 8><<<grid, 256, 0, s>>>(A, lda, plane, lim, kp, piv); break;
    }
    MW_LAUNCH_CHECK();
  }
  SplitOperands o;
  o.L = A + kp * lda + kp + h;
  o.lrs = 1;
  o.lks = lda;
  o.planeL = plane;
  o.U = A + (kp + h) * lda + kp;
  o.uks = 1;
  o.ujs = lda;
  o.planeU = plane;
  o.C = A + (kp + h) * lda + kp + h;
  o.crs = 1;
  o.cjs = lda;
  o.planeC = plane;
  o.m = n - kp - h;
  o.N = lim - kp - h;
  o.K = h;
  rc = split_product_dd(o, sws, sbytes, kPhPanelInner, s);
  if (rc) return rc;
  rc = split_panel_rec(A, lda, plane, n, kp + h, w - h, leaf, piv, info, ws, sws, sbytes, s);
  if (rc) return rc;
  return swap_gather_range(A, lda, plane, kp + h, (int)(lim - kp - h), kp, kp + h, piv, ws, s);
}

// Blocked look-ahead: once panel k's block row U12 is known, the next
// panel's columns are updated first; that panel is then factored on the
// side stream while the caller's stream updates the rest of the trailing
// matrix, and the caller's stream waits for the panel before the next row
// swaps.  The panel only touches its own columns (and the pivots, the
// candidate records and its own split product area), the trailing update
// only the columns right of it, and every entry receives the same
// operations in the same order as in the serial schedule, so the result is
// bitwise the same.  The side stream's priority places the panel's CTAs
// ahead of the update's queued CTAs; the panel's grid-wide waits are bounded
// like every other wait.
namespace {
struct SideSlot {
  std::mutex mu;
  cudaStream_t s2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kSideDevices = 64;
SideSlot g_side[kSideDevices];
}  // namespace

int SideStream::open(cudaStream_t s, bool* ready) {
  *ready = false;
  s_ = s;
  MW_CUDA_CHECK(cudaGetDevice(&dev_));
  if (dev_ < 0 || dev_ >= kSideDevices) return MW_OK;
  SideSlot& slot = g_side[dev_];
  slot.mu.lock();
  if (!slot.s2) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      slot.mu.unlock();
      dev_ = -1;
      if (e != cudaSuccess) MW_CUDA_CHECK(e);
      return MW_OK;
    }
    int lo = 0, hi = 0;
    cudaError_t ce = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&slot.s2, cudaStreamNonBlocking, hi);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&slot.fork, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&slot.join, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
      if (slot.fork) cudaEventDestroy(slot.fork);
      if (slot.s2) cudaStreamDestroy(slot.s2);
      slot.s2 = nullptr;
      slot.fork = nullptr;
      slot.join = nullptr;
      slot.mu.unlock();
      dev_ = -1;
      MW_CUDA_CHECK(ce);
    }
  }
  s2_ = slot.s2;
  fork_ = slot.fork;
  join_ = slot.join;
  *ready = true;
  return MW_OK;
}

int SideStream::fork(cudaStream_t* s2) {
  MW_CUDA_CHECK(cudaEventRecord(fork_, s_));
  MW_CUDA_CHECK(cudaStreamWaitEvent(s2_, fork_, 0));
  open_ = true;
  *s2 = s2_;
  return MW_OK;
}

int SideStream::join() {
  open_ = false;
  MW_CUDA_CHECK(cudaEventRecord(join_, s2_));
  MW_CUDA_CHECK(cudaStreamWaitEvent(s_, join_, 0));
  return MW_OK;
}

SideStream::~SideStream() {
  if (open_) {
    cudaEventRecord(join_, s2_);
    cudaStreamWaitEvent(s_, join_, 0);
  }
  if (dev_ >= 0 && s2_) g_side[dev_].mu.unlock();
}

size_t lu_workspace_bytes(int update, int64_t n) {
  if (update != MW_UPDATE_SPLIT) return kWsSplit;
  return kWsSplit + split_workspace_bytes(n, kDefaultNb) + split_product_bytes(n, kDefaultNb);
}

static int lu_split_dd(int64_t n, double* A, int64_t lda, int64_t* piv, int64_t* info, char* ws, size_t ws_bytes,
                       cudaStream_t s) {
  const int64_t plane = lda * n;
  char* sws = ws + kWsSplit;
  const size_t sbytes = ws_bytes > kWsSplit ? ws_bytes - kWsSplit : 0;
  if (sbytes < split_workspace_bytes(n, kDefaultNb)) return MW_EUNSUPPORTED;
  // the look-ahead panel's own product area, after the trailing update's
  char* pws = sws + split_workspace_bytes(n, kDefaultNb);
  const size_t pbytes = split_product_bytes(n, kDefaultNb);
  SideStream la;
  bool ahead = false;
  if (ws_bytes >= lu_workspace_bytes(MW_UPDATE_SPLIT, n) && tune_get(MW_TUNE_LOOKAHEAD, 2) == 1) {
    int rc = la.open(s, &ahead);
    if (rc) return rc;
  }
  double* aux = split_aux(sws, n);
  MW_CUDA_CHECK(cudaMemsetAsync(ws, 0, kWsCand + 2 * kCandParity, s));
  MW_CUDA_CHECK(cudaMemsetAsync(sws, 0, 256, s));
  if (ahead) MW_CUDA_CHECK(cudaMemsetAsync(pws, 0, 256, s));
  MW_CUDA_CHECK(cudaMemsetAsync(info, 0, sizeof(int64_t), s));
  constexpr int NB = kDefaultNb;
  const int leaf = tune_get(MW_TUNE_SPLIT_PANEL_LEAF, 2);
  auto panel = [&](int64_t kp, int w, char* xws, size_t xbytes, cudaStream_t st) -> int {
    if (leaf > 0) return split_panel_rec(A, lda, plane, n, kp, w, leaf, piv, info, ws, xws, xbytes, st);
    ProfScope ps(kPhPanel, st);
    return launch_panel<2>(A, lda, plane, n, kp, w, piv, info, ws, st);
  };
  int rc = panel(0, (int)std::min<int64_t>(NB, n), sws, sbytes, s);
  if (rc) return rc;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int kb = (int)std::min<int64_t>(NB, n - k0);
    rc = swap_gather(A, lda, plane, 2, n, k0, kb, piv, ws, k0 > 0, k0 + kb < n, s);
    if (rc) return rc;
    if (k0 + kb >= n) break;
    rc = split_inv_l11(A, lda, plane, k0, aux, s);
    if (rc) return rc;
    const int64_t r0 = k0 + NB;
    SplitOperands o;                 // U12 -= M U12, transposed: rows = the columns of U12
    o.L = A + r0 * lda + k0;
    o.lrs = lda;
    o.lks = 1;
    o.planeL = plane;
    o.U = aux;
    o.uks = NB;
    o.ujs = 1;
    o.planeU = (int64_t)NB * NB;
    o.C = A + r0 * lda + k0;
    o.crs = lda;
    o.cjs = 1;
    o.planeC = plane;
    o.m = n - r0;
    o.N = NB;
    o.K = NB;
    rc = split_product_dd(o, sws, sbytes, kPhTrsm, s);
    if (rc) return rc;
    const int kb1 = (int)std::min<int64_t>(NB, n - r0);   // the next panel
    const int64_t rest = n - r0 - kb1;                     // columns right of it
    if (ahead && rest > 0) {
      rc = split_update_dd(A, lda, plane, r0, n - r0, r0, kb1, k0, NB, sws, sbytes, s);
      if (rc) return rc;
      cudaStream_t s2;
      rc = la.fork(&s2);
      if (rc) return rc;
      rc = panel(r0, kb1, pws, pbytes, s2);
      if (rc) return rc;
      rc = split_update_dd(A, lda, plane, r0, n - r0, r0 + kb1, rest, k0, NB, sws, sbytes, s);
      if (rc) return rc;
      rc = la.join();
    } else {
      rc = split_update_dd(A, lda, plane, r0, n - r0, r0, n - r0, k0, NB, sws, sbytes, s);
      if (rc) return rc;
      rc = panel(r0, kb1, sws, sbytes, s);
    }
    if (rc) return rc;
  }
  return MW_OK;
}

template <int W>
int lu_blocked(int update, int64_t n, double* A, int64_t lda, int64_t* piv, int64_t* info,
               char* ws, size_t ws_bytes, int nb, cudaStream_t s) {
  if (update == MW_UPDATE_SPLIT && W == 2) return lu_split_dd(n, A, lda, piv, info, ws, ws_bytes, s);
  const int64_t plane = lda * n;
  MW_CUDA_CHECK(cudaMemsetAsync(ws, 0, kWsCand + 2 * kCandParity, s));
  MW_CUDA_CHECK(cudaMemsetAsync(info, 0, sizeof(int64_t), s));
  if (n <= 0) return MW_OK;
  SideStream la;
  bool ahead = false;
  if (tune_get(MW_TUNE_LOOKAHEAD, W) == 1) {
    int rc = la.open(s, &ahead);
    if (rc) return rc;
  }
  auto panel = [&](int64_t kp, int w, cudaStream_t st) -> int {
    ProfScope ps(kPhPanel, st);
    return launch_panel<W>(A, lda, plane, n, kp, w, piv, info, ws, st);
  };
  auto gemm = [&](int64_t r0, int64_t c0, int64_t N, int64_t k0, int kb) -> int {
    ProfScope ps(kPhGemmPlain, s);
    return launch_gemm_plain<W>(A, lda, plane, r0, n - r0, c0, N, k0, kb, s);
  };
  int rc = panel(0, (int)std::min<int64_t>(nb, n), s);
  if (rc) return rc;
  for (int64_t k0 = 0; k0 < n; k0 += nb) {
    const int kb = (int)std::min<int64_t>(nb, n - k0);
    if (k0 > 0) {
      rc = swap_gather(A, lda, plane, W, n, k0, kb, piv, ws, true, false, s);
      if (rc) return rc;
    }
    if (k0 + kb >= n) break;
    {
      ProfScope ps(kPhTrsm, s);
      rc = launch_trsm<W>(A, lda, plane, n, k0, kb, piv, s);
    }
    if (rc) return rc;
    const int64_t r0 = k0 + kb;
    const int kb1 = (int)std::min<int64_t>(nb, n - r0);   // the next panel
    const int64_t rest = n - r0 - kb1;                     // columns right of it
    if (ahead && rest > 0) {
      rc = gemm(r0, r0, kb1, k0, kb);
      if (rc) return rc;
      cudaStream_t s2;
      rc = la.fork(&s2);
      if (rc) return rc;
      rc = panel(r0, kb1, s2);
      if (rc) return rc;
      rc = gemm(r0, r0 + kb1, rest, k0, kb);
      if (rc) return rc;
      rc = la.join();
    } else {
      rc = gemm(r0, r0, n - r0, k0, kb);
      if (rc) return rc;
      rc = panel(r0, kb1, s);
    }
    if (rc) return rc;
  }
  return MW_OK;
}

template int lu_blocked<2>(int, int64_t, double*, int64_t, int64_t*, int64_t*, char*, size_t, int, cudaStream_t);
template int lu_blocked<3>(int, int64_t, double*, int64_t, int64_t*, int64_t*, char*, size_t, int, cudaStream_t);
template int lu_blocked<4>(int, int64_t, double*, int64_t, int64_t*, int64_t*, char*, size_t, int, cudaStream_t);

// the panel's swaps on the columns left of it (left) and right of it (right)
static int swap_gather(double* A, int64_t lda, int64_t plane, int W, int64_t n, int64_t k0, int kb,
                       const int64_t* piv, char* ws, bool left, bool right, cudaStream_t s) {
  if (!left && !right) return MW_OK;
  ProfScope ps(kPhLaswp, s);
  SwapPlan* plan = reinterpret_cast<SwapPlan*>(ws + kWsSwapPlan);
  k_swap_plan<<<1, 32, 0, s>>>(piv, (int)k0, kb, plan);
  MW_LAUNCH_CHECK();
  auto apply = [&](int64_t c0, int64_t c1) -> int {
    const int64_t nc = c1 - c0;
    if (nc <= 0) return MW_OK;
    dim3 grid((unsigned)((nc + 7) / 8), W);
    switch (W) {
      case 2: k_swap_apply<2><<<grid, 256, 0, s>>>(A, lda, plane, c0, c1, plan); break;
      case 3: k_swap_apply<3><<<grid, 256, 0, s>>>(A, lda, plane, c0, c1, plan); break;
      default: k_swap_apply<4><<<grid, 256, 0, s>>>(A, lda, plane, c0, c1, plan); break;
    }
    MW_LAUNCH_CHECK();
    return MW_OK;
  };
  int rc = left ? apply(0, k0) : MW_OK;
  if (rc) return rc;
  return right ? apply(k0 + kb, n) : MW_OK;
}

// ---- batched launchers ------------------------------------------------------
int launch_bswap_plan(const BatchView& bv, int act, int k0, int sw_lo, int sw_hi, const int64_t* piv,
                      SwapPlan* plans, cudaStream_t s) {
  if (act <= 0) return MW_OK;
  ProfScope ps(kPhLaswp, s);
  k_bswap_plan<<<act, 32, 0, s>>>(bv, k0, sw_lo, sw_hi, piv, plans);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

template <int W>
int launch_bswap_apply(const BatchView& bv, int act, int k0, int c_lo, int c_hi, int max_cols, double* A,
                       const SwapPlan* plans, cudaStream_t s) {
  if (act <= 0 || max_cols <= 0) return MW_OK;
  ProfScope ps(kPhLaswp, s);
  k_bswap_apply<W><<<dim3((unsigned)act, W, (unsigned)((max_cols + 7) / 8)), 256, 0, s>>>(bv, k0, c_lo, c_hi, A,
                                                                                         plans);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

template <int W>
int launch_bpanel(const BatchView& bv, int act, int nmax, int k0, int c_off, int width, double* A, int64_t* piv,
                  int64_t* info, cudaStream_t s) {
  if (act <= 0) return MW_OK;
  if (width < 1 || width > kBatchNb) return MW_EUNSUPPORTED;
  const size_t shmem = sizeof(double) * (size_t)W * ((size_t)kBatchNb + (size_t)nmax);
  if (shmem > 48 * 1024)
    MW_CUDA_CHECK(ensure_smem_limit(k_bpanel<W>, shmem));
  ProfScope ps(kPhPanel, s);
  k_bpanel<W><<<act, kPanelThreads, shmem, s>>>(bv, nmax, k0 + c_off, width, A, piv, info);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

template <int W>
int launch_bswap(const BatchView& bv, int act, int k0, int sw_lo, int sw_hi, int c_lo, int c_hi, int max_cols,
                 double* A, const int64_t* piv, cudaStream_t s) {
  if (act <= 0 || max_cols <= 0 || sw_hi <= sw_lo) return MW_OK;
  ProfScope ps(kPhLaswp, s);
  k_bswap<W><<<dim3((unsigned)act, W, (unsigned)((max_cols + 127) / 128)), 128, 0, s>>>(bv, k0, sw_lo, sw_hi, c_lo,
                                                                                       c_hi, A, piv);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

template <int W>
int launch_btrsm_sub(const BatchView& bv, int act, int k0, int c_off, int h, double* A, const int64_t* piv,
                     cudaStream_t s) {
  if (act <= 0) return MW_OK;
  ProfScope ps(kPhPanel, s);
  switch (h) {
    case 8: k_btrsm_sub<W, 8><<<dim3((unsigned)act, 1), 256, 0, s>>>(bv, k0 + c_off, A, piv); break;
    case 16: k_btrsm_sub<W, 16><<<dim3((unsigned)act, 2), 256, 0, s>>>(bv, k0 + c_off, A, piv); break;
    case 32: k_btrsm_sub<W, 32><<<dim3((unsigned)act, 4), 256, 0, s>>>(bv, k0 + c_off, A, piv); break;
    default: return MW_EUNSUPPORTED;
  }
  MW_LAUNCH_CHECK();
  return MW_OK;
}

template <int W>
int launch_btrsm(const BatchView& bv, int act, int max_cblocks, int k0, double* A, const int64_t* piv,
                 cudaStream_t s) {
  if (act <= 0 || max_cblocks <= 0) return MW_OK;
  ProfScope ps(kPhTrsm, s);
  k_btrsm<W><<<dim3((unsigned)act, (unsigned)max_cblocks), 256, 0, s>>>(bv, k0, A, piv);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

#define MW_BATCHED_INST(W)                                                                                   \
  template int launch_bpanel<W>(const BatchView&, int, int, int, int, int, double*, int64_t*, int64_t*,        \
                                cudaStream_t);                                                                \
  template int launch_bswap<W>(const BatchView&, int, int, int, int, int, int, int, double*, const int64_t*,    \
                               cudaStream_t);                                                                 \
  template int launch_btrsm_sub<W>(const BatchView&, int, int, int, int, double*, const int64_t*, cudaStream_t); \
  template int launch_bswap_apply<W>(const BatchView&, int, int, int, int, int, double*, const SwapPlan*,          \
                                     cudaStream_t);                                                                 \
  template int launch_btrsm<W>(const BatchView&, int, int, int, double*, const int64_t*, cudaStream_t);
MW_BATCHED_INST(2)
MW_BATCHED_INST(3)
MW_BATCHED_INST(4)
#undef MW_BATCHED_INST

}  // namespace mw
