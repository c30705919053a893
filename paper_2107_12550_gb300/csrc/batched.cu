// batched.cu -- many independent systems of uneven order: LU with partial
// pivoting, substitution, and the refinement loop of the paper (Section 2,
// Listing 1), one launch per step for the whole batch.
//
// Layout of a batch (device arrays, caller-owned):
//   n[s]     order of system s;
//   moff[s]  sum_{s' < s} n[s']^2;  voff[s] = sum_{s' < s} n[s'];
//   order    a permutation of the systems: the processing order (largest
//            first balances the persistent CTAs);
//   a matrix of w words for system s lives at M + w*moff[s] (word c of
//   M_s(i,j) at M[w*moff[s] + c*n*n + j*n + i]); a vector of w words at
//   v + w*voff[s] (word c of v_s(i) at v[w*voff[s] + c*n + i]); pivots at
//   piv + voff[s].
//
// The LU and the substitution are persistent: each CTA takes the next system
// from an atomic counter and processes it alone, so no CTA waits for another.
// Within a system every entry receives exactly the operation sequence of the
// unblocked algorithms (right-looking k-j-i elimination; column-oriented
// substitution), so each system's results are bitwise identical to the
// single-system calls.
#include <algorithm>
#include <mutex>
#include <vector>
#include <cuda_runtime.h>

#include "mw_arith.cuh"
#include "mw_common.cuh"
#include "lu_internal.cuh"
#include "profile.cuh"
#include "exact_acc.cuh"

namespace mw {

constexpr int kBatchThreads = 256;
constexpr int kBatchMaxN = 1024;   // largest order in a batch (shared-memory caches)

// Head of a batched work buffer: the systems' counter of the persistent
// kernels, then the error word of the call (pad[0], pad[1] laid out as a
// DeviceStatus: non-zero pad[0] when a bounded wait gave up).
struct BatchCursor {
  unsigned int next;
  unsigned int pad[63];
};
__host__ __device__ inline DeviceStatus* cursor_status(BatchCursor* c) {
  return reinterpret_cast<DeviceStatus*>(&c->pad[0]);
}

struct BatchState {
  int er;            // exponent of max |r_0|
  int done;          // 0 running, 1 converged, 2 not converged, 3 singular
  int corrections;
  int residuals;
  double prev_corr;
};

template <int W>
struct BCand {
  val<W> v;
  int idx;
};

template <int W>
__device__ __forceinline__ bool bbetter(const val<W>& a, int ia, const val<W>& b, int ib) {
  if (ia < 0) return false;
  if (ib < 0) return true;
  const int c = cmp_abs<W>(a, b);
  return c > 0 || (c == 0 && ia < ib);
}

__device__ __forceinline__ int next_system(BatchCursor* cur, int count) {
  __shared__ int s_idx;
  if (threadIdx.x == 0) s_idx = (int)atomicAdd(&cur->next, 1u);
  __syncthreads();
  const int v = s_idx;
  __syncthreads();
  return v < count ? v : -1;
}

// system containing flat index e, given prefix offsets off[0..count] (off[count] = total)
__device__ __forceinline__ int find_system(const int64_t* off, int count, int64_t e) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// LU of one system per CTA (unblocked right-looking, LAPACK getf2 order).
// dynamic shared memory: pivot row and multipliers, 2 * W * nmax doubles
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kBatchThreads)
k_lu_batched(int count, int nmax, const int* __restrict__ order, const int* __restrict__ nn,
             const int64_t* __restrict__ moff, const int64_t* __restrict__ voff, double* __restrict__ A,
             int64_t* __restrict__ piv, int64_t* __restrict__ info, BatchCursor* cur) {
  extern __shared__ double bsm[];
  double* su = bsm;               // [W][nmax]
  double* sl = bsm + W * nmax;    // [W][nmax]
  __shared__ BCand<W> wred[kBatchThreads / 32];
  __shared__ int s_p;
  __shared__ int s_zero;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    const int pos = next_system(cur, count);
    if (pos < 0) break;
    const int s = order[pos];
    const int n = nn[s];
    double* a = A + (int64_t)W * moff[s];
    const int64_t plane = (int64_t)n * n;
    int64_t* pv = piv + voff[s];
    int64_t inf = 0;
    for (int k = 0; k < n; ++k) {
      val<W> bv;
#pragma unroll
      for (int c = 0; c < W; ++c) bv.v[c] = 0.0;
      int bi = -1;
      for (int i = k + tid; i < n; i += kBatchThreads) {
        const val<W> v = load<W>(a, plane, (int64_t)k * n + i);
        if (bbetter<W>(v, i, bv, bi)) {
          bv = v;
          bi = i;
        }
      }
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        val<W> ov;
#pragma unroll
        for (int c = 0; c < W; ++c) ov.v[c] = __shfl_xor_sync(0xffffffffu, bv.v[c], off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (bbetter<W>(ov, oi, bv, bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        wred[warp].v = bv;
        wred[warp].idx = bi;
      }
      __syncthreads();
      if (tid == 0) {
        BCand<W> b = wred[0];
        for (int w = 1; w < kBatchThreads / 32; ++w)
          if (bbetter<W>(wred[w].v, wred[w].idx, b.v, b.idx)) b = wred[w];
        s_p = b.idx;
        s_zero = is_zero<W>(b.v) ? 1 : 0;
        pv[k] = b.idx;
      }
      __syncthreads();
      const int p = s_p;
      if (s_zero && inf == 0) inf = k + 1;
      // swap rows k and p over all columns; cache the new row k (j >= k)
      for (int j = tid; j < n; j += kBatchThreads) {
#pragma unroll
        for (int c = 0; c < W; ++c) {
          double* col = a + c * plane + (int64_t)j * n;
          const double x = col[k];
          const double y = col[p];
          if (p != k) {
            col[k] = y;
            col[p] = x;
          }
          if (j >= k) su[c * nmax + j] = (p != k) ? y : x;
        }
      }
      __syncthreads();
      val<W> akk;
#pragma unroll
      for (int c = 0; c < W; ++c) akk.v[c] = su[c * nmax + k];
      const bool zero = is_zero<W>(akk);
      for (int i = k + 1 + tid; i < n; i += kBatchThreads) {
        val<W> l = load<W>(a, plane, (int64_t)k * n + i);
        if (!zero) {
          l = div<W, false>(l, akk);
          store<W>(a, plane, (int64_t)k * n + i, l);
        }
#pragma unroll
        for (int c = 0; c < W; ++c) sl[c * nmax + i] = l.v[c];
      }
      __syncthreads();
      const int m = n - k - 1;
      const int items = m * m;
      for (int q = tid; q < items; q += kBatchThreads) {
        const int i = k + 1 + q % m;
        const int j = k + 1 + q / m;
        val<W> l, u;
#pragma unroll
        for (int c = 0; c < W; ++c) {
          l.v[c] = sl[c * nmax + i];
          u.v[c] = su[c * nmax + j];
        }
        const int64_t idx = (int64_t)j * n + i;
        val<W> x = load<W>(a, plane, idx);
        x = msub<W, false>(x, l, u);
        store<W>(a, plane, idx, x);
      }
      __syncthreads();
    }
    if (tid == 0) info[s] = inf;
  }
}

// ---------------------------------------------------------------------------
// substitution of one system per CTA (x may alias b): y = P b, then
// y_i -= l_ij y_j (j ascending), d_j = 1 / u_jj for all j, then
// x_j = y_j d_j and y_i -= u_ij x_j (j descending), blocked by 32 rows, as a
// pipeline between warps that synchronise through shared-memory flags:
//  * the leader (warp 0) takes block b: it applies block b-1 (forward; b+1
//    backward) to block b's rows, with the rows in its lanes, once the
//    workers have applied every earlier block to them, then solves block
//    b's 32 x 32 triangle and publishes it;
//  * the 15 worker warps apply each published block to the rows two or
//    more blocks further on; each worker thread always owns the same rows.
// So every y_i still receives its updates in the order above, while the
// triangles overlap the workers' updates.  Each wait is bounded; a wait that
// runs out records an error word and makes all warps leave the system.
// Systems whose state is not "running" are skipped when st is given.
// dynamic shared memory: W * (2 nmax + 4096) doubles (y, the reciprocals,
// the leader's two tiles)
// ---------------------------------------------------------------------------
constexpr int kSolveBs = 32;
// The substitution's CTA: 512 threads, one per SM: warp 0 leads, warps
// 1 .. 15 work (measured: fewer workers were slower, 12 gave 77.2 ms and
// 15 gave 75.0 ms for a 512-system refinement, 8 gave 89 ms).  The
// leader's serial chain takes TwoSum's FP64 form, the workers' loops the
// integer form (63.2 ms; the other three combinations 75.0-86.3 ms).
constexpr int kSolveThreads = 512;
constexpr int kSolveWorkers = kSolveThreads / 32 - 1;                            // worker warps
constexpr int kSolveWGroups = (kBatchMaxN / 32 + kSolveWorkers - 1) / kSolveWorkers;  // row groups per worker
constexpr unsigned long long kSolveSpin = 1ull << 24;

template <int W>
__device__ __forceinline__ val<W> smem_val(const double* v, int nmax, int i) {
  val<W> r;
#pragma unroll
  for (int c = 0; c < W; ++c) r.v[c] = v[c * nmax + i];
  return r;
}

template <int W>
__device__ __forceinline__ void smem_put(double* v, int nmax, int i, const val<W>& r) {
#pragma unroll
  for (int c = 0; c < W; ++c) v[c * nmax + i] = r.v[c];
}

// bounded wait until pred() holds or the system is being abandoned
template <typename P>
__device__ __forceinline__ bool solve_wait(P pred, volatile int* abort_flag, BatchCursor* cur,
                                           unsigned long long limit) {
  unsigned long long spins = 0;
  while (!pred()) {
    if (*abort_flag) return false;
    if (++spins > pick_limit(limit, kSolveSpin)) {
      *abort_flag = 1;
      atomicExch(&cur->pad[0], 1u);   // error word: a solve wait ran out
      return false;
    }
    __nanosleep(32);
  }
  __threadfence_block();
  return true;
}

template <int W>
__global__ void __launch_bounds__(kSolveThreads, 1)
k_solve_batched(int count, int nmax, const int* __restrict__ order, const int* __restrict__ nn,
                const int64_t* __restrict__ moff, const int64_t* __restrict__ voff,
                const double* __restrict__ LU, const int64_t* __restrict__ piv, const double* b,
                double* x, const BatchState* __restrict__ st, BatchCursor* cur, unsigned long long spin_limit) {
  constexpr int NT = kSolveThreads;
  constexpr int kWorkers = kSolveWorkers;
  constexpr int kWRows = kSolveWGroups;
  extern __shared__ double bsm[];
  double* ysm = bsm;
  double* dsm = bsm + W * nmax;
  __shared__ int far_done[kBatchMaxN / kSolveBs + 2];
  __shared__ int tri_done;
  __shared__ int s_abort;
  volatile int* vfar = far_done;
  volatile int* vtri = &tri_done;
  volatile int* vab = &s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // Row group g (rows 32 g .. 32 g + 31, one per lane; the same as solve
  // block g) belongs to worker g mod kWorkers, so the groups still active in
  // any step (a contiguous range) are dealt round-robin; workers are
  // numbered in warp order.  Ownership is fixed for the whole call, so each
  // row's updates stay in program order on one warp.  wk < 0: not a worker.
  const int wk = warp - 1;   // worker index (-1: the leader)
  auto group_row = [&](int q) { return (wk + q * kWorkers) * 32 + lane; };
  // The leader's two 32 x 64 tiles of the factor (rows of its block, the 64
  // columns from c0), double-buffered in shared memory: tile bk goes to
  // buffer bk & 1, word c of column c0 + cc, row j0 + lane, at
  // [((buf * W + c) * 64 + cc) * 32 + lane].  Each lane copies and reads only
  // its own row, so its own cp.async wait orders them; rows and columns
  // outside the matrix are zero-filled (never read).
  double* ltile = dsm + (size_t)W * nmax;
  const double* a_cur = nullptr;
  int n_cur = 0;
  int64_t plane_cur = 0;
  auto fetch_tile = [&](int bk, int c0) {
    const int r = bk * kSolveBs + lane;
    const bool rok = r < n_cur;
    double* dst = ltile + (size_t)(bk & 1) * W * 64 * 32 + lane;
    for (int cc = 0; cc < 64; ++cc) {
      const int col = c0 + cc;
      if (col < 0 || col >= n_cur) continue;           // warp-uniform
#pragma unroll
      for (int c = 0; c < W; ++c)
        cp_async8(dst + (c * 64 + cc) * 32, a_cur + c * plane_cur + (int64_t)col * n_cur + (rok ? r : 0), rok);
    }
    cp_async_commit();
  };
  auto tile_val = [&](const double* tl, int cc) {
    val<W> v;
#pragma unroll
    for (int c = 0; c < W; ++c) v.v[c] = tl[(c * 64 + cc) * 32];
    return v;
  };
  for (;;) {
    const int pos = next_system(cur, count);
    if (pos < 0) break;
    const int s = order[pos];
    if (st && st[s].done) continue;
    const int n = nn[s];
    const int nb = (n + kSolveBs - 1) / kSolveBs;
    const double* a = LU + (int64_t)W * moff[s];
    const int64_t plane = (int64_t)n * n;
    a_cur = a;
    n_cur = n;
    plane_cur = plane;
    const int64_t* pv = piv + voff[s];
    const double* bs = b + (int64_t)W * voff[s];
    double* xs = x + (int64_t)W * voff[s];
    if (warp == 0) fetch_tile(0, -kSolveBs);   // the leader's first tile, during the set-up
    for (int i = tid; i < n; i += NT)
#pragma unroll
      for (int c = 0; c < W; ++c) ysm[c * nmax + i] = bs[c * n + i];
    // reciprocals of the diagonal, all j in parallel
    for (int j = tid; j < n; j += NT) {
      val<W> one;
#pragma unroll
      for (int c = 0; c < W; ++c) one.v[c] = 0.0;
      one.v[0] = 1.0;
      smem_put<W>(dsm, nmax, j, div<W>(one, load_ro<W>(a, plane, (int64_t)j * n + j)));
    }
    for (int q = tid; q < nb + 2; q += NT) far_done[q] = 0;
    if (tid == 0) {
      tri_done = -1;
      s_abort = 0;
    }
    __syncthreads();
    if (tid == 0) {
      for (int k = 0; k < n; ++k) {
        const int p = (int)pv[k];
        if (p != k)
#pragma unroll
          for (int c = 0; c < W; ++c) {
            const double t = ysm[c * nmax + k];
            ysm[c * nmax + k] = ysm[c * nmax + p];
            ysm[c * nmax + p] = t;
          }
      }
    }
    __syncthreads();
    // ---- forward: unit lower L ----
    if (warp == 0) {
      for (int bk = 0; bk < nb; ++bk) {
        const int j0 = bk * kSolveBs;
        const int bsz = min(kSolveBs, n - j0);
        // block bk + 1's tile streams in while block bk is worked on
        if (bk + 1 < nb) fetch_tile(bk + 1, j0);
        else cp_async_commit();
        if (bk >= 2 && !solve_wait([&] { return vfar[bk - 2] >= kWorkers; }, vab, cur, spin_limit)) break;
        cp_async_wait<1>();
        const double* tl = ltile + (size_t)(bk & 1) * W * 64 * 32 + lane;   // column cc of word c: tl[(c*64+cc)*32]
        const int i = j0 + lane;
        val<W> yi;
        if (lane < bsz) yi = smem_val<W>(ysm, nmax, i);
        else {
#pragma unroll
          for (int c = 0; c < W; ++c) yi.v[c] = 0.0;
        }
        if (bk >= 1 && lane < bsz) {
          const int jp = j0 - kSolveBs;
#pragma unroll 4
          for (int jj = 0; jj < kSolveBs; ++jj)
            yi = msub<W, false>(yi, tile_val(tl, jj), smem_val<W>(ysm, nmax, jp + jj));
        }
        for (int jj = 0; jj < bsz - 1; ++jj) {
          val<W> yj;
#pragma unroll
          for (int c = 0; c < W; ++c) yj.v[c] = __shfl_sync(0xffffffffu, yi.v[c], jj);
          if (lane > jj && lane < bsz)
            yi = msub<W, false>(yi, tile_val(tl, kSolveBs + jj), yj);
        }
        if (lane < bsz) smem_put<W>(ysm, nmax, i, yi);
        __threadfence_block();
        __syncwarp();
        if (lane == 0) *vtri = bk;
      }
      cp_async_wait<0>();
    } else {
      for (int bk = 0; bk < nb; ++bk) {
        if (!solve_wait([&] { return *vtri >= bk; }, vab, cur, spin_limit)) break;
        const int j0 = bk * kSolveBs;
        const int bsz = min(kSolveBs, n - j0);
        const int r0 = j0 + 2 * kSolveBs;
        // the thread's rows advance together, one column at a time, so their
        // independent multiply-subtract chains interleave (each row still
        // takes its updates in ascending column order)
        val<W> yq[kWRows];
        bool act[kWRows];
#pragma unroll
        for (int q = 0; q < kWRows; ++q) {
          const int i = group_row(q);
          act[q] = i >= r0 && i < n;
          if (act[q]) yq[q] = smem_val<W>(ysm, nmax, i);
        }
#pragma unroll 2
        for (int jj = 0; jj < bsz; ++jj) {
          const val<W> yj = smem_val<W>(ysm, nmax, j0 + jj);
#pragma unroll
          for (int q = 0; q < kWRows; ++q) {
            const int i = group_row(q);
            if (act[q]) yq[q] = msub<W>(yq[q], load_ro<W>(a, plane, (int64_t)(j0 + jj) * n + i), yj);
          }
        }
#pragma unroll
        for (int q = 0; q < kWRows; ++q)
          if (act[q]) smem_put<W>(ysm, nmax, group_row(q), yq[q]);
        __threadfence_block();
        __syncwarp();
        if (lane == 0) atomicAdd(&far_done[bk], 1);
      }
    }
    __syncthreads();
    for (int q = tid; q < nb + 2; q += NT) far_done[q] = 0;
    if (tid == 0) tri_done = nb;
    __syncthreads();
    // ---- backward: upper U with the reciprocals ----
    if (!*vab) {
      if (warp == 0) {
        fetch_tile(nb - 1, (nb - 1) * kSolveBs);
        for (int bk = nb - 1; bk >= 0; --bk) {
          const int j0 = bk * kSolveBs;
          const int bsz = min(kSolveBs, n - j0);
          if (bk >= 1) fetch_tile(bk - 1, j0 - kSolveBs);
          else cp_async_commit();
          if (bk <= nb - 3 && !solve_wait([&] { return vfar[bk + 2] >= kWorkers; }, vab, cur, spin_limit)) break;
          cp_async_wait<1>();
          const double* tl = ltile + (size_t)(bk & 1) * W * 64 * 32 + lane;
          const int i = j0 + lane;
          val<W> yi, di;
          if (lane < bsz) {
            yi = smem_val<W>(ysm, nmax, i);
            di = smem_val<W>(dsm, nmax, i);
          } else {
#pragma unroll
            for (int c = 0; c < W; ++c) yi.v[c] = di.v[c] = 0.0;
          }
          if (bk <= nb - 2 && lane < bsz) {
            const int jn = j0 + kSolveBs;
            const int bszn = min(kSolveBs, n - jn);
#pragma unroll 4
            for (int jj = bszn - 1; jj >= 0; --jj)
              yi = msub<W, false>(yi, tile_val(tl, kSolveBs + jj), smem_val<W>(ysm, nmax, jn + jj));
          }
          for (int jj = bsz - 1; jj >= 0; --jj) {
            if (lane == jj) yi = mul<W, false>(yi, di);   // x_j = y_j d_j
            val<W> xj;
#pragma unroll
            for (int c = 0; c < W; ++c) xj.v[c] = __shfl_sync(0xffffffffu, yi.v[c], jj);
            if (lane < jj)
              yi = msub<W, false>(yi, tile_val(tl, jj), xj);
          }
          if (lane < bsz) smem_put<W>(ysm, nmax, i, yi);
          __threadfence_block();
          __syncwarp();
          if (lane == 0) *vtri = bk;
        }
        cp_async_wait<0>();
      } else {
        for (int bk = nb - 1; bk >= 0; --bk) {
          if (!solve_wait([&] { return *vtri <= bk; }, vab, cur, spin_limit)) break;
          const int j0 = bk * kSolveBs;
          const int bsz = min(kSolveBs, n - j0);
          const int rend = j0 - kSolveBs;          // rows [0, rend): blocks <= bk - 2
          val<W> yq[kWRows];
          bool act[kWRows];
#pragma unroll
          for (int q = 0; q < kWRows; ++q) {
            const int i = group_row(q);
            act[q] = i < rend;
            if (act[q]) yq[q] = smem_val<W>(ysm, nmax, i);
          }
#pragma unroll 2
          for (int jj = bsz - 1; jj >= 0; --jj) {
            const val<W> xj = smem_val<W>(ysm, nmax, j0 + jj);
#pragma unroll
            for (int q = 0; q < kWRows; ++q) {
              const int i = group_row(q);
              if (act[q]) yq[q] = msub<W>(yq[q], load_ro<W>(a, plane, (int64_t)(j0 + jj) * n + i), xj);
            }
          }
#pragma unroll
          for (int q = 0; q < kWRows; ++q)
            if (act[q]) smem_put<W>(ysm, nmax, group_row(q), yq[q]);
          __threadfence_block();
          __syncwarp();
          if (lane == 0) atomicAdd(&far_done[bk], 1);
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < n; i += NT)
#pragma unroll
      for (int c = 0; c < W; ++c) xs[c * n + i] = ysm[c * nmax + i];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// refinement kernels (stop mode: correction below 2^-(tb+2) ||x||_inf)
// ---------------------------------------------------------------------------

// LU buffer (W words) <- first W words of A (a_words words), zero-padded
__global__ void k_bt_take_mat(int count, const int64_t* __restrict__ moff, const int* __restrict__ nn,
                              int64_t total, const double* __restrict__ A, int a_words, double* __restrict__ LU,
                              int W) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int s = find_system(moff, count, e);
  const int64_t loc = e - moff[s];
  const int64_t nn2 = (int64_t)nn[s] * nn[s];
  for (int c = 0; c < W; ++c)
    LU[W * moff[s] + c * nn2 + loc] = (c < a_words) ? A[a_words * moff[s] + c * nn2 + loc] : 0.0;
}

// dst (dw words) <- first dw words of src (sw words), zero-padded
__global__ void k_bt_take_vec(int count, const int64_t* __restrict__ voff, const int* __restrict__ nn,
                              int64_t total, const double* __restrict__ src, int sw, double* __restrict__ dst,
                              int dw) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int s = find_system(voff, count, e);
  const int64_t loc = e - voff[s];
  const int n = nn[s];
  for (int c = 0; c < dw; ++c) dst[dw * voff[s] + c * n + loc] = (c < sw) ? src[sw * voff[s] + c * n + loc] : 0.0;
}

__global__ void k_bt_init_state(int count, const int64_t* __restrict__ info, BatchState* __restrict__ st) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  BatchState z;
  z.er = 0;
  z.done = info[s] ? 3 : 0;
  z.corrections = 0;
  z.residuals = 0;
  z.prev_corr = 0.0;
  st[s] = z;
}

// r = b - A x exactly (running systems only); one CTA per 32-row block.
// Warp w takes the columns j = w, w + 8, ...  Each column's A words (one
// per lane's row) and x words are copied into a ring of kResStages stages
// of the warp's shared memory by cp.async, kResStages - 1 columns ahead, so
// the loads of later columns are in flight while a column's products are
// deposited (one column's loads at a time left the kernel bound by their
// latency).  dynamic shared memory: 8 warps x kResStages x
// (32 a_words + x_words) doubles (res_stage_bytes)
constexpr int kResStages = 3;
constexpr int kResWarps = kResThreads / 32;
inline size_t res_stage_bytes(int a_words, int x_words) {
  return sizeof(double) * (size_t)kResWarps * kResStages * (size_t)(32 * a_words + x_words);
}

__global__ void __launch_bounds__(kResThreads)
k_bt_residual(int count, const int* __restrict__ nn, const int64_t* __restrict__ moff,
              const int64_t* __restrict__ voff, const int64_t* __restrict__ rbstart, const double* __restrict__ A,
              int a_words, const double* __restrict__ b, int b_words, const double* __restrict__ x, int x_words,
              double* __restrict__ r, int r_words, const BatchState* __restrict__ st) {
  __shared__ u64 acc[kRowsPerCta][kNL];
  extern __shared__ double rstage[];
  const int s = find_system(rbstart, count, blockIdx.x);
  if (st[s].done) return;
  const int n = nn[s];
  const int64_t plane = (int64_t)n * n;
  const double* As = A + (int64_t)a_words * moff[s];
  const double* bs = b + (int64_t)b_words * voff[s];
  const double* xs = x + (int64_t)x_words * voff[s];
  double* rs = r + (int64_t)r_words * voff[s];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = (int)(blockIdx.x - rbstart[s]) * kRowsPerCta + lane;
  const bool row_ok = i < n;
  for (int e = threadIdx.x; e < kRowsPerCta * kNL; e += blockDim.x) (&acc[0][0])[e] = 0ull;
  __syncthreads();
  if (warp < b_words && row_ok) deposit_double(acc[lane], bs[warp * n + i], 0, false);
  const int per = 32 * a_words + x_words;                 // doubles per stage
  double* ring = rstage + (size_t)warp * kResStages * per;
  // column t of this warp (j = warp + 8 t) into stage t % kResStages; rows
  // beyond n are zero-filled (never used); always one commit group
  auto issue = [&](int t) {
    const int j = warp + t * kResWarps;
    if (j < n) {
      double* dst = ring + (t % kResStages) * per;
      for (int c = 0; c < a_words; ++c)
        cp_async8(dst + c * 32 + lane, As + c * plane + (int64_t)j * n + (row_ok ? i : 0), row_ok);
      if (lane < x_words) cp_async8(dst + 32 * a_words + lane, xs + (int64_t)lane * n + j, true);
    }
    cp_async_commit();
  };
  const int ncols = (n > warp) ? (n - warp + kResWarps - 1) / kResWarps : 0;
  for (int t = 0; t < kResStages - 1; ++t) issue(t);
  for (int t = 0; t < ncols; ++t) {
    issue(t + kResStages - 1);
    cp_async_wait<kResStages - 1>();
    __syncwarp();   // the x words copied by lanes 0 .. x_words-1 are visible to the warp
    const double* src = ring + (t % kResStages) * per;
    if (row_ok) {
      double xv[MW_LONG_WORDS];
#pragma unroll
      for (int d = 0; d < MW_LONG_WORDS; ++d) xv[d] = (d < x_words) ? src[32 * a_words + d] : 0.0;
      for (int c = 0; c < a_words; ++c) {
        const double a = src[c * 32 + lane];
        if (zero_bits(a)) continue;
#pragma unroll
        for (int d = 0; d < MW_LONG_WORDS; ++d)
          if (d < x_words && !zero_bits(xv[d])) deposit_product(acc[lane], a, xv[d], 0, true);
      }
    }
    __syncwarp();   // every lane is done with this stage before it is refilled
  }
  cp_async_wait<0>();
  __syncthreads();
  if (warp == 0 && row_ok) {
    for (int c = 0; c < r_words; ++c) rs[c * n + i] = acc_take(acc[lane]);
  }
}

// per system (one CTA each): residual count, zero residual, iteration limit,
// e = ilogb(max|r_0|) and r_hat = first W words of 2^-e r
__global__ void __launch_bounds__(256)
k_bt_check(int count, const int* __restrict__ nn, const int64_t* __restrict__ voff, const double* __restrict__ r,
           int r_words, double* __restrict__ rhat, int W, int max_iter, BatchState* __restrict__ st) {
  const int s = blockIdx.x;
  if (st[s].done) return;
  const int n = nn[s];
  const double* rs = r + (int64_t)r_words * voff[s];
  __shared__ double red[8];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(rs[i]));
  for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  double rmax = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) rmax = fmax(rmax, red[w]);
  __shared__ int s_go;
  if (threadIdx.x == 0) {
    BatchState q = st[s];
    q.residuals += 1;
    int go = 0;
    if (rmax == 0.0) q.done = 1;
    else if (q.corrections >= max_iter) q.done = 2;
    else {
      q.er = ilogb_pos(rmax);
      go = 1;
    }
    st[s] = q;
    s_go = go;
  }
  __syncthreads();
  if (!s_go) return;
  const int er = st[s].er;
  double* hs = rhat + (int64_t)W * voff[s];
  for (int q = threadIdx.x; q < W * n; q += blockDim.x) hs[q] = scale2(rs[q], -er);
}

// x = RN_xw(x + 2^e z) exactly, one thread per entry (running systems)
__global__ void __launch_bounds__(kRowsPerCta)
k_bt_update(int count, const int* __restrict__ nn, const int64_t* __restrict__ voff, int64_t total,
            double* __restrict__ x, int x_words, const double* __restrict__ z, int W,
            const BatchState* __restrict__ st) {
  __shared__ u64 acc[kRowsPerCta][kNL];
  u64* a = acc[threadIdx.x];
  for (int k = 0; k < kNL; ++k) a[k] = 0ull;
  const int64_t e = (int64_t)blockIdx.x * kRowsPerCta + threadIdx.x;
  if (e >= total) return;
  const int s = find_system(voff, count, e);
  if (st[s].done) return;
  const int n = nn[s];
  const int64_t i = e - voff[s];
  double* xs = x + (int64_t)x_words * voff[s];
  const double* zs = z + (int64_t)W * voff[s];
  const int er = st[s].er;
  for (int c = 0; c < x_words; ++c) deposit_double(a, xs[c * n + i], 0, false);
  for (int c = 0; c < W; ++c) deposit_double(a, zs[c * n + i], er, false);
  for (int c = 0; c < x_words; ++c) xs[c * n + i] = acc_take(a);
}

// per system after an update: correction size and the stopping tests
__global__ void __launch_bounds__(256)
k_bt_check2(int count, const int* __restrict__ nn, const int64_t* __restrict__ voff, const double* __restrict__ z,
            int W, const double* __restrict__ x, int x_words, int target_bits, BatchState* __restrict__ st) {
  const int s = blockIdx.x;
  if (st[s].done) return;
  const int n = nn[s];
  const double* zs = z + (int64_t)W * voff[s];
  const double* xs = x + (int64_t)x_words * voff[s];
  __shared__ double rz[8], rx[8];
  double mz = 0.0, mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    mz = fmax(mz, fabs(zs[i]));
    mx = fmax(mx, fabs(xs[i]));
  }
  for (int off = 16; off; off >>= 1) {
    mz = fmax(mz, __shfl_xor_sync(0xffffffffu, mz, off));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  }
  if ((threadIdx.x & 31) == 0) {
    rz[threadIdx.x >> 5] = mz;
    rx[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double zmax = 0.0, xmax = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      zmax = fmax(zmax, rz[w]);
      xmax = fmax(xmax, rx[w]);
    }
    BatchState q = st[s];
    q.corrections += 1;
    const double corr = scale2(zmax, q.er);
    const double lim = scale2(xmax, -target_bits - 2);
    if (corr <= lim) q.done = 1;
    else if (q.corrections >= 2 && corr > __dmul_rn(0.5, q.prev_corr)) q.done = 2;
    q.prev_corr = corr;
    st[s] = q;
  }
}

__global__ void k_bt_count_running(int count, const BatchState* __restrict__ st, int* __restrict__ running) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int c = 0;
  for (int s = threadIdx.x; s < count; s += blockDim.x) c += (st[s].done == 0);
  atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0) *running = cnt;
}

// per-system results; a bounded wait that gave up anywhere in the call
// (the cursor's error word) marks every system MW_ETIMEOUT
__global__ void k_bt_stats(int count, const BatchState* __restrict__ st, const int64_t* __restrict__ info,
                           const DeviceStatus* __restrict__ err, int64_t* __restrict__ stats) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  const BatchState q = st[s];
  stats[4 * s + 0] = q.corrections;
  stats[4 * s + 1] = q.residuals;
  stats[4 * s + 2] = info[s];
  stats[4 * s + 3] = err->timeout ? MW_ETIMEOUT
                                  : (q.done == 1 ? MW_OK : (q.done == 3 ? MW_ESINGULAR : MW_ENOTCONV));
}

// the number of systems still running, as the condition of the refinement's
// graph while node (capture mode)
__global__ void k_bt_running_cond(int count, const BatchState* __restrict__ st, cudaGraphConditionalHandle h) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int c = 0;
  for (int s = threadIdx.x; s < count; s += blockDim.x) c += (st[s].done == 0);
  atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(h, cnt > 0 ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename K>
static int set_smem(K kern, size_t bytes) {
  MW_CUDA_CHECK(ensure_smem_limit(kern, bytes));
  return MW_OK;
}

template <int W>
static int lu_batched_launch(int count, int nmax, const int* order, const int* nn, const int64_t* moff,
                             const int64_t* voff, double* A, int64_t* piv, int64_t* info, char* ws, cudaStream_t s) {
  if (count <= 0) return MW_OK;
  BatchCursor* cur = reinterpret_cast<BatchCursor*>(ws);
  MW_CUDA_CHECK(cudaMemsetAsync(&cur->next, 0, sizeof(cur->next), s));   // the error word stays
  const size_t shmem = sizeof(double) * 2 * W * (size_t)nmax;
  int rc = set_smem(k_lu_batched<W>, shmem);
  if (rc) return rc;
  ProfScope ps(kPhBatchLu, s);
  const int grid = std::min(count, std::max(1, tune_get(MW_TUNE_BATCH_CTAS_PER_SM, W)) * device_sm_count());
  k_lu_batched<W><<<grid, kBatchThreads, shmem, s>>>(count, nmax, order, nn, moff, voff, A, piv, info, cur);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

template <int W>
static int solve_batched_launch(int count, int nmax, const int* order, const int* nn, const int64_t* moff,
                                const int64_t* voff, const double* LU, const int64_t* piv, const double* b,
                                double* x, const void* st, char* ws, cudaStream_t s) {
  if (count <= 0) return MW_OK;
  BatchCursor* cur = reinterpret_cast<BatchCursor*>(ws);
  MW_CUDA_CHECK(cudaMemsetAsync(&cur->next, 0, sizeof(cur->next), s));   // the error word stays
  // y and the reciprocals (2 W nmax doubles), then the leader's two tiles
  const size_t shmem = sizeof(double) * W * (2 * (size_t)nmax + 2 * 64 * 32);
  const int grid = std::min(count, device_sm_count());
  const BatchState* bst = static_cast<const BatchState*>(st);
  int rc = set_smem(k_solve_batched<W>, shmem);
  if (rc) return rc;
  ProfScope ps(kPhBatchSolve, s);
  k_solve_batched<W><<<grid, kSolveThreads, shmem, s>>>(count, nmax, order, nn, moff, voff, LU, piv, b, x, bst, cur,
                                                        wait_limit());
  MW_LAUNCH_CHECK();
  return MW_OK;
}

// ---------------------------------------------------------------------------
// batch plan: n, offsets, processing order and residual row-block prefix,
// computed on the host from the host copy of n and uploaded into the work
// buffer at the start of every call
// ---------------------------------------------------------------------------
struct BatchPlanHost {
  std::vector<int> n, order;
  std::vector<int64_t> moff, voff, rb;
  int64_t sum_n = 0, sum_n2 = 0;
  int nmax = 0;
};

static bool make_plan(int count, const int* n_host, BatchPlanHost& p) {
  p.n.assign(n_host, n_host + count);
  p.moff.resize(count + 1);
  p.voff.resize(count + 1);
  p.rb.resize(count + 1);
  int64_t m = 0, v = 0, r = 0;
  p.nmax = 1;
  for (int s = 0; s < count; ++s) {
    if (p.n[s] < 1 || p.n[s] > kBatchMaxN) return false;
    p.moff[s] = m;
    p.voff[s] = v;
    p.rb[s] = r;
    m += (int64_t)p.n[s] * p.n[s];
    v += p.n[s];
    r += (p.n[s] + kRowsPerCta - 1) / kRowsPerCta;
    p.nmax = std::max(p.nmax, p.n[s]);
  }
  p.moff[count] = m;
  p.voff[count] = v;
  p.rb[count] = r;
  p.sum_n = v;
  p.sum_n2 = m;
  p.order.resize(count);
  for (int s = 0; s < count; ++s) p.order[s] = s;
  std::stable_sort(p.order.begin(), p.order.end(), [&](int a, int b) { return p.n[a] > p.n[b]; });
  return true;
}

struct BatchPlanDev {
  int* n;
  int64_t* moff;
  int64_t* voff;
  int* order;
  int64_t* rb;
};

// [cursor 256 | n | moff | voff | order | rb]
static size_t plan_bytes(int count) {
  return 256 + align256(sizeof(int) * count) + 2 * align256(sizeof(int64_t) * (count + 1)) +
         align256(sizeof(int) * count) + align256(sizeof(int64_t) * (count + 1));
}

// Plans already resident in work buffers: (device address, kind, hash of the
// batch).  Only while the caller has switched this on (mw_batch_plan_cache):
// then a call whose plan is already in place issues no host-to-device copy,
// so repeated calls on the same batch and work buffer can be captured in a
// CUDA graph.  The caller must keep those work buffers (a freed buffer's
// address can come back holding other data); mw_batch_plan_reset() or
// switching the cache off forgets every entry.
struct ResidentPlan {
  const void* addr;
  int kind;
  unsigned long long hash;
};
static std::mutex g_plan_mu;
static std::vector<ResidentPlan> g_plans;
static bool g_plan_cache_on = false;
constexpr size_t kMaxResidentPlans = 256;

static unsigned long long batch_hash(const std::vector<int>& n, int a, int b) {
  unsigned long long h = 1469598103934665603ull;   // FNV-1a
  auto mix = [&](unsigned long long v) {
    for (int i = 0; i < 8; ++i) {
      h ^= (v >> (8 * i)) & 0xffull;
      h *= 1099511628211ull;
    }
  };
  mix((unsigned long long)n.size());
  mix((unsigned long long)(unsigned)a);
  mix((unsigned long long)(unsigned)b);
  for (int v : n) mix((unsigned long long)(unsigned)v);
  return h;
}

// true if the plan is already resident; otherwise records it (the caller
// then uploads it)
static bool plan_resident(const void* addr, int kind, unsigned long long hash) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  if (!g_plan_cache_on) return false;
  for (auto& e : g_plans)
    if (e.addr == addr) {
      if (e.kind == kind && e.hash == hash) return true;
      e.kind = kind;
      e.hash = hash;
      return false;
    }
  if (g_plans.size() >= kMaxResidentPlans) g_plans.erase(g_plans.begin());
  g_plans.push_back(ResidentPlan{addr, kind, hash});
  return false;
}

static void plan_forget(const void* addr) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  for (size_t i = 0; i < g_plans.size(); ++i)
    if (g_plans[i].addr == addr) {
      g_plans.erase(g_plans.begin() + i);
      return;
    }
}

static int upload_plan(const BatchPlanHost& p, int count, char* ws, BatchPlanDev& d, cudaStream_t s) {
  // the cursor and its error word (a bounded wait that gave up) start clear
  // in every call
  MW_CUDA_CHECK(cudaMemsetAsync(ws, 0, sizeof(BatchCursor), s));
  size_t off = 256;
  d.n = reinterpret_cast<int*>(ws + off);
  off += align256(sizeof(int) * count);
  d.moff = reinterpret_cast<int64_t*>(ws + off);
  off += align256(sizeof(int64_t) * (count + 1));
  d.voff = reinterpret_cast<int64_t*>(ws + off);
  off += align256(sizeof(int64_t) * (count + 1));
  d.order = reinterpret_cast<int*>(ws + off);
  off += align256(sizeof(int) * count);
  d.rb = reinterpret_cast<int64_t*>(ws + off);
  if (plan_resident(ws, 0, batch_hash(p.n, 0, 0))) return MW_OK;
  cudaError_t e = cudaMemcpyAsync(d.n, p.n.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.moff, p.moff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.voff, p.voff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.order, p.order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.rb, p.rb.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    plan_forget(ws);
    MW_CUDA_CHECK(e);
  }
  return MW_OK;
}

// ---------------------------------------------------------------------------
// blocked batched LU: all systems advance one panel of kBatchNb columns per
// step.  Step k0 factors the panels of the systems with n > k0 (one CTA
// each), applies their swaps left of the panel, solves U12 = L11^-1 A12 and
// runs the trailing update A22 -= L21 U12 as one launch over a tile list
// that spans all active systems (plain multiword GEMM, or the split form for
// DD).  The plan below holds, per step, the active count, the grid extents
// and the tile lists; it is computed on the host from n and uploaded with
// the batch plan.
// ---------------------------------------------------------------------------
// one kind of trailing-update work per step: tiles over all active systems
struct GeomPlanHost {
  std::vector<int> max_mt, max_cb;   // per step: slicing grid extents (split)
  std::vector<int64_t> toff, boff;   // per step: first tile, first base (nsteps + 1 entries)
  std::vector<int64_t> tnext;        // trail, per step: tiles touching the next panel's 64 columns,
                                     // listed first among the step's tiles
  std::vector<TileEntry> tiles;
  std::vector<int2> bases;           // split: {first A-slice tile, first B-slice tile} per (step, pos)
  int64_t a_tiles = 0, b_tiles = 0;  // split: slice tiles of the largest step
};

struct BlockedPlanHost {
  int update = MW_UPDATE_PLAIN;
  int nsteps = 0;
  std::vector<int> act, max_cb_trsm, max_cols;
  GeomPlanHost trail;   // plain: BM x BN tiles; split: 128 x 16 tiles of A22
  GeomPlanHost tinv;    // split: 128 x 16 tiles of U12^T (the TRSM as a product with L11^-1)
  GeomPlanHost pinner[7];  // split: 128 x 16 tiles of the inner panel updates (kInner order)
};

// the inner updates of the recursive split panel: (column offset, half width)
// of the blocks 64 -> 32 + 32 -> 16 + 16
struct InnerSpec {
  int c_off, h;
};
constexpr int kNumInner = 7;
constexpr InnerSpec kInner[kNumInner] = {{0, 8}, {16, 8}, {0, 16}, {32, 8}, {48, 8}, {32, 16}, {0, 32}};

// tiles of an m x N product for every active system of one step
static void add_geom_step(GeomPlanHost& g, const BatchPlanHost& p, int act, bool split, int bm, int bn,
                          int (*dims)(int n, int k0, int c_off, int h, int* N), int k0, int c_off = 0,
                          int h = 0, bool next_first = false) {
  const size_t t_begin = g.tiles.size();
  int64_t at = 0, btl = 0;
  int max_m = 0, max_n = 0;
  for (int pos = 0; pos < act; ++pos) {
    int N = 0;
    const int m = dims(p.n[p.order[pos]], k0, c_off, h, &N);
    if (split) g.bases.push_back(make_int2((int)at, (int)btl));
    if (m <= 0 || N <= 0) continue;
    max_m = std::max(max_m, m);
    max_n = std::max(max_n, N);
    const int mt = (m + bm - 1) / bm, nt = (N + bn - 1) / bn;
    for (int tj = 0; tj < nt; ++tj)
      for (int ti = 0; ti < mt; ++ti) g.tiles.push_back(TileEntry{pos, ti, tj, 0});
    at += mt;
    btl += nt;
  }
  if (next_first) {
    // the tiles holding any of the first kBatchNb columns first (the next
    // panel's columns, updated before that panel is factored)
    auto mid = std::stable_partition(g.tiles.begin() + (std::ptrdiff_t)t_begin, g.tiles.end(),
                                     [&](const TileEntry& t) { return t.tj * bn < kBatchNb; });
    g.tnext.push_back((int64_t)(mid - (g.tiles.begin() + (std::ptrdiff_t)t_begin)));
  }
  g.max_mt.push_back((max_m + kSplitTileM - 1) / kSplitTileM);
  g.max_cb.push_back(((max_n + kSplitTileN - 1) / kSplitTileN * kSplitTileN + 127) / 128);
  if (split) {
    g.a_tiles = std::max(g.a_tiles, at);
    g.b_tiles = std::max(g.b_tiles, btl);
  }
  g.toff.push_back((int64_t)g.tiles.size());
  g.boff.push_back((int64_t)g.bases.size());
}

static int dims_trail(int n, int k0, int, int, int* N) {
  *N = n - k0 - kBatchNb;
  return n - k0 - kBatchNb;
}
static int dims_tinv(int n, int k0, int, int, int* N) {
  *N = kBatchNb;
  return n - k0 - kBatchNb;
}
static int dims_pinner(int n, int k0, int c_off, int h, int* N) {
  const int m = n - k0 - c_off - h;
  *N = std::min(h, m);
  return m;
}

static void make_blocked_plan(const BatchPlanHost& p, int W, int update, BlockedPlanHost& bp) {
  bp = BlockedPlanHost();
  bp.update = update;
  const bool split = update == MW_UPDATE_SPLIT;
  int bm = 0, bn = 0;
  gemm_plain_tile_shape(W, &bm, &bn);
  if (split) {
    bm = kSplitTileM;
    bn = kSplitTileN;
  }
  const int count = (int)p.n.size();
  for (GeomPlanHost* g : {&bp.trail, &bp.tinv}) {
    g->toff.push_back(0);
    g->boff.push_back(0);
  }
  for (auto& g : bp.pinner) {
    g.toff.push_back(0);
    g.boff.push_back(0);
  }
  if (count == 0) return;
  int act = count;
  for (int k0 = 0; k0 < p.nmax; k0 += kBatchNb) {
    while (act > 0 && p.n[p.order[act - 1]] <= k0) --act;   // order is largest first
    bp.act.push_back(act);
    const int m0 = p.n[p.order[0]] - k0 - kBatchNb;          // largest trailing order
    bp.max_cb_trsm.push_back(m0 > 0 ? (m0 + 7) / 8 : 0);
    bp.max_cols.push_back(std::max(m0, 0));
    add_geom_step(bp.trail, p, act, split, bm, bn, dims_trail, k0, 0, 0, true);
    if (split) {
      add_geom_step(bp.tinv, p, act, true, kSplitTileM, kSplitTileN, dims_tinv, k0);
      for (int q = 0; q < kNumInner; ++q)
        add_geom_step(bp.pinner[q], p, act, true, kSplitTileM, kSplitTileN, dims_pinner, k0, kInner[q].c_off,
                      kInner[q].h);
    }
    ++bp.nsteps;
  }
}

static size_t geom_bytes(const GeomPlanHost& g) {
  return align256(sizeof(TileEntry) * std::max<size_t>(1, g.tiles.size())) +
         align256(sizeof(int2) * std::max<size_t>(1, g.bases.size()));
}

static int64_t blocked_count(const BlockedPlanHost& bp) { return bp.act.empty() ? 0 : bp.act[0]; }

static int64_t max_a_tiles(const BlockedPlanHost& bp) {
  int64_t t = std::max(bp.trail.a_tiles, bp.tinv.a_tiles);
  for (const auto& g : bp.pinner) t = std::max(t, g.a_tiles);
  return t;
}
static int64_t max_b_tiles(const BlockedPlanHost& bp) {
  int64_t t = std::max(bp.trail.b_tiles, bp.tinv.b_tiles);
  for (const auto& g : bp.pinner) t = std::max(t, g.b_tiles);
  return t;
}

static int64_t inner_a_tiles(const BlockedPlanHost& bp) {
  int64_t t = 0;
  for (const auto& g : bp.pinner) t = std::max(t, g.a_tiles);
  return t;
}
static int64_t inner_b_tiles(const BlockedPlanHost& bp) {
  int64_t t = 0;
  for (const auto& g : bp.pinner) t = std::max(t, g.b_tiles);
  return t;
}

// [trail | tinv | pinner tiles and bases | swap plans | aux | split scratch |
//  the look-ahead panel's split scratch]
static size_t blocked_extra_bytes(const BlockedPlanHost& bp) {
  size_t b = geom_bytes(bp.trail) + geom_bytes(bp.tinv);
  for (const auto& g : bp.pinner) b += geom_bytes(g);
  b += align256(sizeof(SwapPlan) * (size_t)std::max<int64_t>(1, blocked_count(bp)));
  if (bp.update == MW_UPDATE_SPLIT) {
    b += align256(sizeof(double) * 2 * kBatchNb * kBatchNb * (size_t)std::max<int64_t>(1, blocked_count(bp)));
    b += split_batched_workspace_bytes(max_a_tiles(bp), max_b_tiles(bp));
    b += split_batched_workspace_bytes(inner_a_tiles(bp), inner_b_tiles(bp));   // the look-ahead panel's
  }
  return b;
}

struct GeomDev {
  TileEntry* tiles;
  int2* bases;
};

struct BlockedDev {
  GeomDev trail, tinv, pinner[kNumInner];
  SwapPlan* plans;   // one per active position
  double* aux;
  char* split_ws;
  size_t split_bytes;
  int64_t a_tiles, b_tiles;
  char* panel_ws;                  // the look-ahead panel's split scratch
  size_t panel_bytes;
  int64_t pa_tiles, pb_tiles;
  DeviceStatus* status;   // the call's error word (in the batch cursor)
};

static int upload_geom(const GeomPlanHost& g, char* base, size_t& off, GeomDev& d, cudaStream_t s,
                       bool resident) {
  d.tiles = reinterpret_cast<TileEntry*>(base + off);
  off += align256(sizeof(TileEntry) * std::max<size_t>(1, g.tiles.size()));
  d.bases = reinterpret_cast<int2*>(base + off);
  off += align256(sizeof(int2) * std::max<size_t>(1, g.bases.size()));
  if (resident) return MW_OK;
  if (!g.tiles.empty())
    MW_CUDA_CHECK(cudaMemcpyAsync(d.tiles, g.tiles.data(), sizeof(TileEntry) * g.tiles.size(),
                                  cudaMemcpyHostToDevice, s));
  if (!g.bases.empty())
    MW_CUDA_CHECK(cudaMemcpyAsync(d.bases, g.bases.data(), sizeof(int2) * g.bases.size(),
                                  cudaMemcpyHostToDevice, s));
  return MW_OK;
}

static int upload_blocked(const BlockedPlanHost& bp, const std::vector<int>& n, int prec, char* base,
                          BlockedDev& d, cudaStream_t s) {
  const bool resident = plan_resident(base, 1, batch_hash(n, prec, bp.update));
  size_t off = 0;
  int rc = upload_geom(bp.trail, base, off, d.trail, s, resident);
  if (rc) return rc;
  if (rc) {
    plan_forget(base);
    return rc;
  }
  rc = upload_geom(bp.tinv, base, off, d.tinv, s, resident);
  if (rc) {
    plan_forget(base);
    return rc;
  }
  for (int q = 0; q < kNumInner; ++q) {
    rc = upload_geom(bp.pinner[q], base, off, d.pinner[q], s, resident);
    if (rc) {
      plan_forget(base);
      return rc;
    }
  }
  d.plans = reinterpret_cast<SwapPlan*>(base + off);
  off += align256(sizeof(SwapPlan) * (size_t)std::max<int64_t>(1, blocked_count(bp)));
  d.aux = nullptr;
  d.split_ws = nullptr;
  d.split_bytes = 0;
  d.a_tiles = max_a_tiles(bp);
  d.b_tiles = max_b_tiles(bp);
  d.panel_ws = nullptr;
  d.panel_bytes = 0;
  d.pa_tiles = d.pb_tiles = 0;
  if (bp.update == MW_UPDATE_SPLIT) {
    d.aux = reinterpret_cast<double*>(base + off);
    off += align256(sizeof(double) * 2 * kBatchNb * kBatchNb * (size_t)std::max<int64_t>(1, blocked_count(bp)));
    d.split_ws = base + off;
    d.split_bytes = split_batched_workspace_bytes(d.a_tiles, d.b_tiles);
    off += d.split_bytes;
    MW_CUDA_CHECK(cudaMemsetAsync(d.split_ws, 0, 256, s));
    d.pa_tiles = inner_a_tiles(bp);
    d.pb_tiles = inner_b_tiles(bp);
    d.panel_ws = base + off;
    d.panel_bytes = split_batched_workspace_bytes(d.pa_tiles, d.pb_tiles);
    MW_CUDA_CHECK(cudaMemsetAsync(d.panel_ws, 0, 256, s));
  }
  return MW_OK;
}

// the split path's panel: columns [k0 + c_off, k0 + c_off + w) factored
// recursively -- left half, the right half's top rows solved, the rows below
// updated by a split product, right half, then the right half's swaps on the
// left half -- down to leaves of MW_TUNE_BATCH_SPLIT_LEAF columns (8, 16 or
// 32; 8 by default) factored on the FP64 pipe
// (on the scratch `ws` laid out for pa x pb slice tiles)
template <int W>
static int split_panel(const BatchPlanHost& p, const BatchView& bv, const BlockedPlanHost& bp, const BlockedDev& bd,
                       int st, int act, int k0, int c_off, int w, double* A, int64_t* piv, int64_t* info,
                       char* ws, size_t ws_bytes, int64_t pa, int64_t pb, cudaStream_t s) {
  if (w <= tune_get(MW_TUNE_BATCH_SPLIT_LEAF, 2)) return launch_bpanel<W>(bv, act, p.nmax, k0, c_off, w, A, piv, info, s);
  const int h = w / 2;
  int q = -1;
  for (int i = 0; i < kNumInner; ++i)
    if (kInner[i].c_off == c_off && kInner[i].h == h) q = i;
  if (q < 0) return MW_EUNSUPPORTED;
  int rc = split_panel<W>(p, bv, bp, bd, st, act, k0, c_off, h, A, piv, info, ws, ws_bytes, pa, pb, s);
  if (rc) return rc;
  rc = launch_btrsm_sub<W>(bv, act, k0, c_off, h, A, piv, s);
  if (rc) return rc;
  const GeomPlanHost& g = bp.pinner[q];
  rc = split_bupdate_dd(bv, kGeomPanelInner, c_off, h, act, g.max_mt[st], g.max_cb[st], bd.pinner[q].tiles + g.toff[st],
                        g.toff[st + 1] - g.toff[st], bd.pinner[q].bases + g.boff[st], pa, pb, k0, A,
                        bd.aux, ws, ws_bytes, bd.status, s);
  if (rc) return rc;
  rc = split_panel<W>(p, bv, bp, bd, st, act, k0, c_off + h, w - h, A, piv, info, ws, ws_bytes, pa, pb, s);
  if (rc) return rc;
  return launch_bswap<W>(bv, act, k0, c_off + h, c_off + w, c_off, c_off + h, h, A, piv, s);
}

// Plain update: panel, swaps left, TRSM (with the swaps right), plain GEMM;
// every element sees the unblocked order.  Split update (DD): the recursive
// panel above, the swaps left and right, M = -(L11^-1) strictly lower, then
// U12 -= M U12 and A22 -= L21 U12 as split tensor-core products.
// Look-ahead (MW_TUNE_LOOKAHEAD, as in the single-system LU): the trailing
// tiles that hold the next panel's columns are updated first, then the next
// panel is factored on the side stream while the caller's stream updates
// the other tiles; the caller's stream joins the panel before the next
// swaps.  The panel touches only its own columns (its inner split products
// use a scratch of their own), the other tiles only columns right of it, and
// each entry gets the same operations in the same order: bitwise the same.
template <int W>
static int lu_blocked_batched_run(const BatchPlanHost& p, const BatchPlanDev& d, const BlockedPlanHost& bp,
                                  const BlockedDev& bd, double* A, int64_t* piv, int64_t* info, cudaStream_t s) {
  const BatchView bv{d.order, d.n, d.moff, d.voff};
  const bool split = bp.update == MW_UPDATE_SPLIT;
  if (split && W != 2) return MW_EUNSUPPORTED;
  if (bp.nsteps <= 0) return MW_OK;
  constexpr int kFar = 1 << 29;
  SideStream la;
  bool ahead = false;
  if (tune_get(MW_TUNE_LOOKAHEAD, W) == 1 && (!split || bd.panel_ws)) {
    int rc = la.open(s, &ahead);
    if (rc) return rc;
  }
  // panel of step st on stream q (the look-ahead panel on its own scratch)
  auto panel = [&](int st, cudaStream_t q, bool own) -> int {
    const int k0 = st * kBatchNb;
    if (split)
      return own ? split_panel<W>(p, bv, bp, bd, st, bp.act[st], k0, 0, kBatchNb, A, piv, info, bd.panel_ws,
                                  bd.panel_bytes, bd.pa_tiles, bd.pb_tiles, q)
                 : split_panel<W>(p, bv, bp, bd, st, bp.act[st], k0, 0, kBatchNb, A, piv, info, bd.split_ws,
                                  bd.split_bytes, bd.a_tiles, bd.b_tiles, q);
    return launch_bpanel<W>(bv, bp.act[st], p.nmax, k0, 0, kBatchNb, A, piv, info, q);
  };
  // trailing tiles [t0, t1) of step st (within the step's list)
  auto trail = [&](int st, int64_t t0, int64_t t1) -> int {
    if (t1 <= t0) return MW_OK;
    const int k0 = st * kBatchNb;
    const TileEntry* tl = bd.trail.tiles + bp.trail.toff[st] + t0;
    if (split)
      return split_bgemm_dd(bv, kGeomTrail, 0, 0, tl, t1 - t0, bd.trail.bases + bp.trail.boff[st], bd.a_tiles,
                            bd.b_tiles, k0, A, bd.aux, bd.split_ws, bd.split_bytes, bd.status, s);
    return launch_bgemm_plain<W>(bv, tl, t1 - t0, k0, A, s);
  };
  int rc = panel(0, s, false);
  if (rc) return rc;
  for (int st = 0; st < bp.nsteps; ++st) {
    const int k0 = st * kBatchNb;
    const int act = bp.act[st];
    const int64_t nt = bp.trail.toff[st + 1] - bp.trail.toff[st];
    if (split) {
      rc = launch_bswap_plan(bv, act, k0, 0, kBatchNb, piv, bd.plans, s);
      if (rc) return rc;
      rc = launch_bswap_apply<W>(bv, act, k0, -k0, 0, k0, A, bd.plans, s);   // left of the panel
      if (rc) return rc;
      if (bp.max_cols[st] <= 0) continue;   // no system has columns right of this panel: the last step
      rc = launch_bswap_apply<W>(bv, act, k0, kBatchNb, kFar, bp.max_cols[st], A, bd.plans, s);   // right
      if (rc) return rc;
      rc = split_binv_l11(bv, act, k0, A, bd.aux, s);
      if (rc) return rc;
      rc = split_bupdate_dd(bv, kGeomTrsmInv, 0, 0, act, bp.tinv.max_mt[st], bp.tinv.max_cb[st],
                            bd.tinv.tiles + bp.tinv.toff[st], bp.tinv.toff[st + 1] - bp.tinv.toff[st],
                            bd.tinv.bases + bp.tinv.boff[st], bd.a_tiles, bd.b_tiles, k0, A, bd.aux, bd.split_ws,
                            bd.split_bytes, bd.status, s);
      if (rc) return rc;
      rc = split_bslice_dd(bv, kGeomTrail, 0, 0, act, bp.trail.max_mt[st], bp.trail.max_cb[st],
                           bd.trail.bases + bp.trail.boff[st], bd.a_tiles, bd.b_tiles, k0, A, bd.aux, bd.split_ws,
                           bd.split_bytes, s);
      if (rc) return rc;
    } else {
      if (k0 > 0) {
        rc = launch_bswap_plan(bv, act, k0, 0, kBatchNb, piv, bd.plans, s);
        if (rc) return rc;
        rc = launch_bswap_apply<W>(bv, act, k0, -k0, 0, k0, A, bd.plans, s);   // left of the panel
        if (rc) return rc;
      }
      if (st + 1 >= bp.nsteps) break;
      rc = launch_btrsm<W>(bv, act, bp.max_cb_trsm[st], k0, A, piv, s);
      if (rc) return rc;
    }
    if (st + 1 >= bp.nsteps) {
      rc = trail(st, 0, nt);
      if (rc) return rc;
      continue;
    }
    const int64_t tn = bp.trail.tnext[st];
    if (ahead && tn < nt) {
      rc = trail(st, 0, tn);
      if (rc) return rc;
      cudaStream_t s2;
      rc = la.fork(&s2);
      if (rc) return rc;
      rc = panel(st + 1, s2, split);
      if (rc) return rc;
      rc = trail(st, tn, nt);
      if (rc) return rc;
      rc = la.join();
    } else {
      rc = trail(st, 0, nt);
      if (rc) return rc;
      rc = panel(st + 1, s, false);
    }
    if (rc) return rc;
  }
  return MW_OK;
}

// refinement work buffer map (after the plan)
struct BatchRefineMap {
  size_t lu, piv, info, r, z, rhat, st, running, total;
};

static BatchRefineMap batch_refine_map(int W, int count, int64_t sum_n, int64_t sum_n2) {
  BatchRefineMap m;
  size_t off = plan_bytes(count);
  m.lu = off;
  off += align256(sizeof(double) * W * (size_t)sum_n2);
  m.piv = off;
  off += align256(sizeof(int64_t) * (size_t)sum_n);
  m.info = off;
  off += align256(sizeof(int64_t) * (size_t)count);
  m.r = off;
  off += align256(sizeof(double) * MW_LONG_WORDS * (size_t)sum_n);
  m.z = off;
  off += align256(sizeof(double) * W * (size_t)sum_n);
  m.rhat = off;
  off += align256(sizeof(double) * W * (size_t)sum_n);
  m.st = off;
  off += align256(sizeof(BatchState) * (size_t)count);
  m.running = off;
  off += 256;
  m.total = off;
  return m;
}

// A stream of the library's own per device, into which the refinement's
// loop body is captured while the caller's stream is being captured.  It is
// created by the first call on the device, which must run outside a capture
// (as the resident plans already require).
static int body_stream(cudaStream_t* out) {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static cudaStream_t streams[kMaxDev] = {};
  int dev = 0;
  MW_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) return MW_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(mu);
  if (!streams[dev]) MW_CUDA_CHECK(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
  *out = streams[dev];
  return MW_OK;
}

// Inside a capture of stream s: appends a while node whose body is one
// refinement step (captured on the library's own stream) followed by
// k_bt_running_cond, which sets the node's condition to "systems still
// running".  The condition starts at 1 on every launch of the graph, so the
// body runs at least once, as the loop outside a capture does.
template <typename F1, typename F2>
static int capture_refine_loop(cudaStream_t s, int count, const BatchState* st, F1& residual_and_check,
                               F2& correct) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  unsigned long long id = 0;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t nd = 0;
  MW_CUDA_CHECK(cudaStreamGetCaptureInfo(s, &cs, &id, &g, &deps, &edata, &nd));
  if (cs != cudaStreamCaptureStatusActive || !g) return MW_EUNSUPPORTED;
  cudaStream_t q = nullptr;
  int rc = body_stream(&q);
  if (rc) return rc;
  cudaGraphConditionalHandle h;
  MW_CUDA_CHECK(cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  MW_CUDA_CHECK(cudaGraphAddNode(&node, g, deps, edata, nd, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  MW_CUDA_CHECK(cudaStreamBeginCaptureToGraph(q, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  rc = residual_and_check(q);
  if (!rc) rc = correct(q);
  if (!rc) {
    prof_count(kPhRefineAux);
    k_bt_running_cond<<<1, 256, 0, q>>>(count, st, h);
  }
  const cudaError_t le = cudaGetLastError();
  cudaGraph_t captured = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(q, &captured);
  if (rc) return rc;
  MW_CUDA_CHECK(le);
  MW_CUDA_CHECK(ee);
  MW_CUDA_CHECK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return MW_OK;
}

// blk: null for the persistent one-CTA-per-system LU, else the blocked LU
template <int W>
static int refine_batched_impl(int count, const BatchPlanHost& p, const BatchPlanDev& d, const double* A, int a_words,
                               const double* b, int b_words, int target_bits, int max_iter, double* x, int x_words,
                               int64_t* stats, char* ws, size_t ws_bytes, cudaStream_t s,
                               const BlockedPlanHost* blk = nullptr, const BlockedDev* blkd = nullptr) {
  const BatchRefineMap mp = batch_refine_map(W, count, p.sum_n, p.sum_n2);
  if (ws_bytes < mp.total) return -15;
  double* LU = reinterpret_cast<double*>(ws + mp.lu);
  int64_t* piv = reinterpret_cast<int64_t*>(ws + mp.piv);
  int64_t* info = reinterpret_cast<int64_t*>(ws + mp.info);
  double* r = reinterpret_cast<double*>(ws + mp.r);
  double* z = reinterpret_cast<double*>(ws + mp.z);
  double* rhat = reinterpret_cast<double*>(ws + mp.rhat);
  BatchState* st = reinterpret_cast<BatchState*>(ws + mp.st);
  int* running_d = reinterpret_cast<int*>(ws + mp.running);
  char* cur = ws;
  bool timed_out = false;
  const int64_t nrb = p.rb[count];
  prof_count(kPhRefineAux);
  k_bt_take_mat<<<(unsigned)((p.sum_n2 + 255) / 256), 256, 0, s>>>(count, d.moff, d.n, p.sum_n2, A, a_words, LU, W);
  MW_LAUNCH_CHECK();
  int rc = blk ? lu_blocked_batched_run<W>(p, d, *blk, *blkd, LU, piv, info, s)
               : lu_batched_launch<W>(count, p.nmax, d.order, d.n, d.moff, d.voff, LU, piv, info, cur, s);
  if (rc) return rc;
  prof_count(kPhRefineAux);
  k_bt_init_state<<<(count + 255) / 256, 256, 0, s>>>(count, info, st);
  prof_count(kPhRefineAux);
  k_bt_take_vec<<<(unsigned)((p.sum_n + 255) / 256), 256, 0, s>>>(count, d.voff, d.n, p.sum_n, b, b_words, rhat, W);
  MW_LAUNCH_CHECK();
  rc = solve_batched_launch<W>(count, p.nmax, d.order, d.n, d.moff, d.voff, LU, piv, rhat, z, st, cur, s);
  if (rc) return rc;
  prof_count(kPhRefineAux);
  k_bt_take_vec<<<(unsigned)((p.sum_n + 255) / 256), 256, 0, s>>>(count, d.voff, d.n, p.sum_n, z, W, x, x_words);
  MW_LAUNCH_CHECK();
  MW_CUDA_CHECK(ensure_smem_limit(k_bt_residual, res_stage_bytes(a_words, x_words),
                                  sizeof(u64) * kRowsPerCta * kNL));   // + the accumulators
  // one refinement step, in two halves: the exact residual and the tests,
  // then the correction solve, the exact update and the correction test
  // (every kernel skips the systems that are no longer running)
  auto residual_and_check = [&](cudaStream_t q) -> int {
    {
      ProfScope ps(kPhResidual, q);
      k_bt_residual<<<(unsigned)nrb, kResThreads, res_stage_bytes(a_words, x_words), q>>>(
          count, d.n, d.moff, d.voff, d.rb, A, a_words, b, b_words, x, x_words, r, x_words, st);
      MW_LAUNCH_CHECK();
    }
    prof_count(kPhRefineAux);
    k_bt_check<<<count, 256, 0, q>>>(count, d.n, d.voff, r, x_words, rhat, W, max_iter, st);
    MW_LAUNCH_CHECK();
    return MW_OK;
  };
  auto correct = [&](cudaStream_t q) -> int {
    int rc2 = solve_batched_launch<W>(count, p.nmax, d.order, d.n, d.moff, d.voff, LU, piv, rhat, z, st, cur, q);
    if (rc2) return rc2;
    prof_count(kPhRefineAux);
    k_bt_update<<<(unsigned)((p.sum_n + kRowsPerCta - 1) / kRowsPerCta), kRowsPerCta, 0, q>>>(
        count, d.n, d.voff, p.sum_n, x, x_words, z, W, st);
    prof_count(kPhRefineAux);
    k_bt_check2<<<count, 256, 0, q>>>(count, d.n, d.voff, z, W, x, x_words, target_bits, st);
    MW_LAUNCH_CHECK();
    return MW_OK;
  };
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  MW_CUDA_CHECK(cudaStreamIsCapturing(s, &cap));
  if (cap == cudaStreamCaptureStatusNone) {
    cudaStream_t q = nullptr;
    rc = body_stream(&q);   // created here, outside any capture
    if (rc) return rc;
  }
  if (cap == cudaStreamCaptureStatusActive) {
    // inside a stream capture: the loop becomes a while node of the graph
    // whose condition the last kernel of each step sets on the device (the
    // number of systems still running), so no value comes back to the host
    rc = capture_refine_loop(s, count, st, residual_and_check, correct);
    if (rc) return rc;
  } else {
    for (int it = 0; it <= max_iter; ++it) {
      rc = residual_and_check(s);
      if (rc) return rc;
      prof_count(kPhRefineAux);
      k_bt_count_running<<<1, 256, 0, s>>>(count, st, running_d);
      MW_LAUNCH_CHECK();
      int running = 0;
      DeviceStatus sv = {};
      MW_CUDA_CHECK(cudaMemcpyAsync(&running, running_d, sizeof(int), cudaMemcpyDeviceToHost, s));
      MW_CUDA_CHECK(cudaMemcpyAsync(&sv, cursor_status(reinterpret_cast<BatchCursor*>(cur)), sizeof(sv),
                                    cudaMemcpyDeviceToHost, s));
      MW_CUDA_CHECK(cudaStreamSynchronize(s));
      if (sv.timeout) timed_out = true;   // a bounded wait of the LU or a substitution gave up
      if (running == 0 || timed_out) break;
      rc = correct(s);
      if (rc) return rc;
    }
  }
  prof_count(kPhRefineAux);
  k_bt_stats<<<(count + 255) / 256, 256, 0, s>>>(count, st, info, cursor_status(reinterpret_cast<BatchCursor*>(cur)),
                                                 stats);
  MW_LAUNCH_CHECK();
  return timed_out ? MW_ETIMEOUT : MW_OK;
}

}  // namespace mw

// ---------------------------------------------------------------------------
// C ABI (declared in include/mwlu.h)
// ---------------------------------------------------------------------------
static bool bprec_ok(int p) { return p == MW_DD || p == MW_TD || p == MW_QD; }

extern "C" int mw_batch_workspace_size(int op, int prec, int count, const int* n_host, size_t* bytes) {
  if (op != MW_OP_LUDECOMP && op != MW_OP_SOLVE && op != MW_OP_REFINE) return -1;
  if (!bprec_ok(prec)) return -2;
  if (count < 0) return -3;
  if (count > 0 && !n_host) return -4;
  if (!bytes) return -5;
  mw::BatchPlanHost p;
  if (!mw::make_plan(count, n_host, p)) return -4;
  if (op == MW_OP_REFINE) *bytes = mw::batch_refine_map(prec, count, p.sum_n, p.sum_n2).total;
  else *bytes = mw::plan_bytes(count);
  return MW_OK;
}

extern "C" int mw_ludecomp_batched(int prec, int count, const int* n_host, double* A, int64_t* piv,
                                   int64_t* info, void* work, size_t work_bytes, void* stream) {
  if (!bprec_ok(prec)) return -1;
  if (count < 0) return -2;
  if (count == 0) return MW_OK;
  if (!n_host) return -3;
  if (!A) return -4;
  if (!piv) return -5;
  if (!info) return -6;
  if (!work) return -7;
  mw::BatchPlanHost p;
  if (!mw::make_plan(count, n_host, p)) return -3;
  if (work_bytes < mw::plan_bytes(count)) return -8;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(work);
  mw::BatchPlanDev d;
  int rc = mw::upload_plan(p, count, ws, d, s);
  if (rc) return rc;
  switch (prec) {
    case 2: return mw::lu_batched_launch<2>(count, p.nmax, d.order, d.n, d.moff, d.voff, A, piv, info, ws, s);
    case 3: return mw::lu_batched_launch<3>(count, p.nmax, d.order, d.n, d.moff, d.voff, A, piv, info, ws, s);
    default: return mw::lu_batched_launch<4>(count, p.nmax, d.order, d.n, d.moff, d.voff, A, piv, info, ws, s);
  }
}

extern "C" int mw_solve_batched(int prec, int count, const int* n_host, const double* LU, const int64_t* piv,
                                const double* b, double* x, void* work, size_t work_bytes, void* stream) {
  if (!bprec_ok(prec)) return -1;
  if (count < 0) return -2;
  if (count == 0) return MW_OK;
  if (!n_host) return -3;
  if (!LU) return -4;
  if (!piv) return -5;
  if (!b) return -6;
  if (!x) return -7;
  if (!work) return -8;
  mw::BatchPlanHost p;
  if (!mw::make_plan(count, n_host, p)) return -3;
  if (work_bytes < mw::plan_bytes(count)) return -9;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(work);
  mw::BatchPlanDev d;
  int rc = mw::upload_plan(p, count, ws, d, s);
  if (rc) return rc;
  switch (prec) {
    case 2: return mw::solve_batched_launch<2>(count, p.nmax, d.order, d.n, d.moff, d.voff, LU, piv, b, x, nullptr, ws, s);
    case 3: return mw::solve_batched_launch<3>(count, p.nmax, d.order, d.n, d.moff, d.voff, LU, piv, b, x, nullptr, ws, s);
    default: return mw::solve_batched_launch<4>(count, p.nmax, d.order, d.n, d.moff, d.voff, LU, piv, b, x, nullptr, ws, s);
  }
}

extern "C" int mw_refine_batched(int count, const int* n_host, const double* A, int a_words, const double* b,
                                 int b_words, int inner, int target_bits, int max_iter, double* x, int x_words,
                                 int64_t* stats, void* work, size_t work_bytes, void* stream) {
  if (count < 0) return -1;
  if (count == 0) return MW_OK;
  if (!n_host) return -2;
  if (!A) return -3;
  if (a_words < 1 || a_words > MW_LONG_WORDS) return -4;
  if (!b) return -5;
  if (b_words < 1 || b_words > MW_LONG_WORDS) return -6;
  if (!bprec_ok(inner)) return -7;
  if (target_bits < 1 || target_bits > 1000) return -8;
  if (max_iter < 0) return -9;
  if (!x) return -10;
  if (x_words < inner || x_words > MW_LONG_WORDS) return -11;
  if (!stats) return -12;
  if (!work) return -13;
  mw::BatchPlanHost p;
  if (!mw::make_plan(count, n_host, p)) return -2;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(work);
  if (work_bytes < mw::batch_refine_map(inner, count, p.sum_n, p.sum_n2).total) return -14;
  mw::BatchPlanDev d;
  int rc = mw::upload_plan(p, count, ws, d, s);
  if (rc) return rc;
  switch (inner) {
    case 2: return mw::refine_batched_impl<2>(count, p, d, A, a_words, b, b_words, target_bits, max_iter, x, x_words, stats, ws, work_bytes, s);
    case 3: return mw::refine_batched_impl<3>(count, p, d, A, a_words, b, b_words, target_bits, max_iter, x, x_words, stats, ws, work_bytes, s);
    default: return mw::refine_batched_impl<4>(count, p, d, A, a_words, b, b_words, target_bits, max_iter, x, x_words, stats, ws, work_bytes, s);
  }
}

// ---- blocked batched LU and refinement ---------------------------------------
extern "C" int mw_batch_blocked_workspace_size(int op, int prec, int update, int count, const int* n_host,
                                               size_t* bytes) {
  if (op != MW_OP_LUDECOMP && op != MW_OP_REFINE) return -1;
  if (!bprec_ok(prec)) return -2;
  if (update != MW_UPDATE_PLAIN && update != MW_UPDATE_SPLIT) return -3;
  if (count < 0) return -4;
  if (count > 0 && !n_host) return -5;
  if (!bytes) return -6;
  if (update == MW_UPDATE_SPLIT && prec != MW_DD) return MW_EUNSUPPORTED;
  mw::BatchPlanHost p;
  if (!mw::make_plan(count, n_host, p)) return -5;
  mw::BlockedPlanHost bp;
  mw::make_blocked_plan(p, prec, update, bp);
  const size_t head = (op == MW_OP_REFINE) ? mw::batch_refine_map(prec, count, p.sum_n, p.sum_n2).total
                                           : mw::plan_bytes(count);
  *bytes = mw::align256(head) + mw::blocked_extra_bytes(bp);
  return MW_OK;
}

extern "C" int mw_ludecomp_batched_blocked(int prec, int update, int count, const int* n_host, double* A,
                                           int64_t* piv, int64_t* info, void* work, size_t work_bytes,
                                           void* stream) {
  if (!bprec_ok(prec)) return -1;
  if (update != MW_UPDATE_PLAIN && update != MW_UPDATE_SPLIT) return -2;
  if (count < 0) return -3;
  if (count == 0) return MW_OK;
  if (!n_host) return -4;
  if (!A) return -5;
  if (!piv) return -6;
  if (!info) return -7;
  if (!work) return -8;
  if (update == MW_UPDATE_SPLIT && prec != MW_DD) return MW_EUNSUPPORTED;
  mw::BatchPlanHost p;
  if (!mw::make_plan(count, n_host, p)) return -4;
  mw::BlockedPlanHost bp;
  mw::make_blocked_plan(p, prec, update, bp);
  const size_t head = mw::align256(mw::plan_bytes(count));
  if (work_bytes < head + mw::blocked_extra_bytes(bp)) return -9;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(work);
  mw::BatchPlanDev d;
  int rc = mw::upload_plan(p, count, ws, d, s);
  if (rc) return rc;
  mw::BlockedDev bd;
  rc = mw::upload_blocked(bp, p.n, prec, ws + head, bd, s);
  if (rc) return rc;
  bd.status = mw::cursor_status(reinterpret_cast<mw::BatchCursor*>(ws));
  switch (prec) {
    case 2: return mw::lu_blocked_batched_run<2>(p, d, bp, bd, A, piv, info, s);
    case 3: return mw::lu_blocked_batched_run<3>(p, d, bp, bd, A, piv, info, s);
    default: return mw::lu_blocked_batched_run<4>(p, d, bp, bd, A, piv, info, s);
  }
}

extern "C" int mw_refine_batched_blocked(int count, const int* n_host, const double* A, int a_words,
                                         const double* b, int b_words, int inner, int update, int target_bits,
                                         int max_iter, double* x, int x_words, int64_t* stats, void* work,
                                         size_t work_bytes, void* stream) {
  if (count < 0) return -1;
  if (count == 0) return MW_OK;
  if (!n_host) return -2;
  if (!A) return -3;
  if (a_words < 1 || a_words > MW_LONG_WORDS) return -4;
  if (!b) return -5;
  if (b_words < 1 || b_words > MW_LONG_WORDS) return -6;
  if (!bprec_ok(inner)) return -7;
  if (update != MW_UPDATE_PLAIN && update != MW_UPDATE_SPLIT) return -8;
  if (target_bits < 1 || target_bits > 1000) return -9;
  if (max_iter < 0) return -10;
  if (!x) return -11;
  if (x_words < inner || x_words > MW_LONG_WORDS) return -12;
  if (!stats) return -13;
  if (!work) return -14;
  if (update == MW_UPDATE_SPLIT && inner != MW_DD) return MW_EUNSUPPORTED;
  mw::BatchPlanHost p;
  if (!mw::make_plan(count, n_host, p)) return -2;
  mw::BlockedPlanHost bp;
  mw::make_blocked_plan(p, inner, update, bp);
  const size_t head = mw::align256(mw::batch_refine_map(inner, count, p.sum_n, p.sum_n2).total);
  if (work_bytes < head + mw::blocked_extra_bytes(bp)) return -15;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(work);
  mw::BatchPlanDev d;
  int rc = mw::upload_plan(p, count, ws, d, s);
  if (rc) return rc;
  mw::BlockedDev bd;
  rc = mw::upload_blocked(bp, p.n, inner, ws + head, bd, s);
  if (rc) return rc;
  bd.status = mw::cursor_status(reinterpret_cast<mw::BatchCursor*>(ws));
  switch (inner) {
    case 2: return mw::refine_batched_impl<2>(count, p, d, A, a_words, b, b_words, target_bits, max_iter, x, x_words, stats, ws, head, s, &bp, &bd);
    case 3: return mw::refine_batched_impl<3>(count, p, d, A, a_words, b, b_words, target_bits, max_iter, x, x_words, stats, ws, head, s, &bp, &bd);
    default: return mw::refine_batched_impl<4>(count, p, d, A, a_words, b, b_words, target_bits, max_iter, x, x_words, stats, ws, head, s, &bp, &bd);
  }
}

extern "C" int mw_batch_work_status(const void* work, void* stream) {
  if (!work) return -1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mw::DeviceStatus sv = {};
  MW_CUDA_CHECK(cudaMemcpyAsync(&sv, mw::cursor_status(reinterpret_cast<mw::BatchCursor*>(const_cast<void*>(work))),
                                sizeof(sv), cudaMemcpyDeviceToHost, s));
  MW_CUDA_CHECK(cudaStreamSynchronize(s));
  return sv.timeout ? MW_ETIMEOUT : MW_OK;
}

extern "C" int mw_batch_plan_reset(void) {
  std::lock_guard<std::mutex> lk(mw::g_plan_mu);
  mw::g_plans.clear();
  return MW_OK;
}

extern "C" int mw_batch_plan_cache(int on) {
  std::lock_guard<std::mutex> lk(mw::g_plan_mu);
  const int prev = mw::g_plan_cache_on ? 1 : 0;
  mw::g_plan_cache_on = on != 0;
  if (!on) mw::g_plans.clear();
  return prev;
}
