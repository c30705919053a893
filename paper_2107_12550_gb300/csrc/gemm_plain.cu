// gemm_plain.cu -- the plain multiword trailing update (Section 2: the
// block product of the blocked LU) on the FP64 and integer pipes: one tile
// routine shared by the single-system launch (k_gemm_plain, tile variant
// chosen per launch) and the batched launch over a tile list
// (k_bgemm_plain).  Every entry receives its updates in ascending t, as in
// unblocked elimination, so every tile variant gives the same bits.
#include <algorithm>
#include <cuda_runtime.h>

#include "mw_arith.cuh"
#include "mw_common.cuh"
#include "lu_internal.cuh"
#include "profile.cuh"

namespace mw {

// ---------------------------------------------------------------------------
// plain trailing update: C -= L21 * U12 with per-element sequential t.
// 16 x 16 threads, micro-tile TM x TN per thread, K chunks of KT staged in
// shared memory with coalesced loads of each word plane.
// ---------------------------------------------------------------------------

// K chunks of KT staged in shared memory, double-buffered: the copies of
// chunk t+1 (cp.async, zero-filled outside the matrix) run while chunk t is
// consumed.  Each entry of C still receives its updates in ascending t:
// c -= l_t u_t, or with ADD c += l_t u_t (a rounded multiword multiply, then
// a rounded addition or subtraction).
template <int W, int TM, int TN, bool ADD = false>
__device__ __forceinline__ void gemm_plain_tile(double* __restrict__ C, int64_t ldc, int64_t planeC,
                                                const double* __restrict__ L, int64_t ldl, int64_t planeL,
                                                const double* __restrict__ U, int64_t ldu, int64_t planeU,
                                                int64_t m, int64_t N, int K, int64_t tile_i, int64_t tile_j) {
  constexpr int KT = 8;
  constexpr int BM = 16 * TM, BN = 16 * TN;
  __shared__ double sL[2][W][KT][BM];
  __shared__ double sU[2][W][KT][BN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t bi = tile_i * BM, bj = tile_j * BN;

  auto stage = [&](int buf, int t0) {
    const int kt_n = (K - t0 < KT) ? K - t0 : KT;
    // L tile: rows bi..bi+BM, columns t0..: consecutive threads -> rows
    for (int e = threadIdx.x; e < BM * KT; e += 256) {
      const int r = e % BM, kt = e / BM;
      const int64_t i = bi + r;
      const bool ok = (i < m) && (kt < kt_n);
#pragma unroll
      for (int c = 0; c < W; ++c) cp_async8(&sL[buf][c][kt][r], ok ? L + c * planeL + (t0 + kt) * ldl + i : L, ok);
    }
    // U tile: rows t0.., columns bj..: consecutive threads -> rows (t)
    for (int e = threadIdx.x; e < BN * KT; e += 256) {
      const int kt = e % KT, cidx = e / KT;
      const int64_t jj = bj + cidx;
      const bool ok = (jj < N) && (kt < kt_n);
#pragma unroll
      for (int c = 0; c < W; ++c) cp_async8(&sU[buf][c][kt][cidx], ok ? U + c * planeU + jj * ldu + t0 + kt : U, ok);
    }
    cp_async_commit();
  };

  stage(0, 0);
  val<W> acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int64_t i = bi + tx + 16 * a, jj = bj + ty + 16 * b;
      if (i < m && jj < N) acc[a][b] = load<W>(C, planeC, jj * ldc + i);
      else {
#pragma unroll
        for (int c = 0; c < W; ++c) acc[a][b].v[c] = 0.0;
      }
    }

  int buf = 0;
  for (int t0 = 0; t0 < K; t0 += KT, buf ^= 1) {
    if (t0 + KT < K) {
      stage(buf ^ 1, t0 + KT);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int kt_n = (K - t0 < KT) ? K - t0 : KT;
    for (int kt = 0; kt < kt_n; ++kt) {
      val<W> l[TM], u[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int c = 0; c < W; ++c) l[a].v[c] = sL[buf][c][kt][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < TN; ++b)
#pragma unroll
        for (int c = 0; c < W; ++c) u[b].v[c] = sU[buf][c][kt][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b)
          acc[a][b] = ADD ? add<W>(acc[a][b], mul<W>(l[a], u[b])) : msub<W>(acc[a][b], l[a], u[b]);
    }
    __syncthreads();   // every thread is done with `buf` before it is refilled
  }
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int64_t i = bi + tx + 16 * a, jj = bj + ty + 16 * b;
      if (i < m && jj < N) store<W>(C, planeC, jj * ldc + i, acc[a][b]);
    }
}

template <int W, int TM, int TN, bool ADD>
__global__ void __launch_bounds__(256)
k_gemm_plain(double* __restrict__ C, int64_t ldc, int64_t planeC, const double* __restrict__ L,
             int64_t ldl, int64_t planeL, const double* __restrict__ U, int64_t ldu, int64_t planeU,
             int64_t m, int64_t N, int K) {
  gemm_plain_tile<W, TM, TN, ADD>(C, ldc, planeC, L, ldl, planeL, U, ldu, planeU, m, N, K, blockIdx.x,
                                  blockIdx.y);
}

// micro-tile of the batched trailing update (tile lists; many systems keep
// the waves full)
template <int W> struct GemmTile;
template <> struct GemmTile<2> { static constexpr int TM = 4, TN = 4; };
template <> struct GemmTile<3> { static constexpr int TM = 2, TN = 4; };
template <> struct GemmTile<4> { static constexpr int TM = 2, TN = 2; };

// Tile variants of the trailing update, largest first.  A launch is a few
// waves of equal tiles over (SMs x resident CTAs) slots; when its last wave
// is partly empty, a smaller tile can finish in fewer slot-units.  Every
// entry of C still receives its updates in ascending k, so all variants give
// bitwise the same result.
template <int W, int V> struct GemmVariant;
template <> struct GemmVariant<2, 0> { static constexpr int TM = 4, TN = 4; };
template <> struct GemmVariant<2, 1> { static constexpr int TM = 2, TN = 4; };
template <> struct GemmVariant<2, 2> { static constexpr int TM = 2, TN = 2; };
template <> struct GemmVariant<3, 0> { static constexpr int TM = 2, TN = 4; };
template <> struct GemmVariant<3, 1> { static constexpr int TM = 1, TN = 2; };
template <> struct GemmVariant<3, 2> { static constexpr int TM = 1, TN = 1; };
template <> struct GemmVariant<4, 0> { static constexpr int TM = 2, TN = 2; };
template <> struct GemmVariant<4, 1> { static constexpr int TM = 1, TN = 2; };
template <> struct GemmVariant<4, 2> { static constexpr int TM = 1, TN = 1; };
constexpr int kGemmVariants = 3;

template <int W, int V>
static int64_t gemm_variant_cost(int64_t m, int64_t N) {
  constexpr int BM = 16 * GemmVariant<W, V>::TM, BN = 16 * GemmVariant<W, V>::TN;
  const int64_t tiles = ((m + BM - 1) / BM) * ((N + BN - 1) / BN);
  const int64_t sms = device_sm_count();
  // the CTAs resident on an SM share its FP64 pipe, so an SM's time is the
  // number of its tiles times the tile size, however many run at once
  return ((tiles + sms - 1) / sms) * BM * BN;
}

// the variant a launch of m x N uses: MW_TUNE_GEMM_TILE 1..3 forces one,
// 0 picks the least per-SM pipe time (the smaller tile on a tie; a full
// wave runs at the same rate with any of the three)
template <int W>
int gemm_plain_variant(int64_t m, int64_t N) {
  const int forced = tune_get(MW_TUNE_GEMM_TILE, W);
  if (forced >= 1 && forced <= kGemmVariants) return forced - 1;
  const int64_t c0 = gemm_variant_cost<W, 0>(m, N);
  const int64_t c1 = gemm_variant_cost<W, 1>(m, N);
  const int64_t c2 = gemm_variant_cost<W, 2>(m, N);
  int v = 2;
  int64_t best = c2;
  if (c1 < best) v = 1, best = c1;
  if (c0 < best) v = 0;
  return v;
}

template <int W, int V>
static void launch_gemm_variant(int64_t m, int64_t N, int K, double* C, int64_t ldc, int64_t planeC,
                                const double* L, int64_t ldl, int64_t planeL, const double* U, int64_t ldu,
                                int64_t planeU, bool add, cudaStream_t s) {
  constexpr int TM = GemmVariant<W, V>::TM, TN = GemmVariant<W, V>::TN;
  dim3 grid((unsigned)((m + 16 * TM - 1) / (16 * TM)), (unsigned)((N + 16 * TN - 1) / (16 * TN)));
  if (add)
    k_gemm_plain<W, TM, TN, true><<<grid, 256, 0, s>>>(C, ldc, planeC, L, ldl, planeL, U, ldu, planeU, m, N, K);
  else
    k_gemm_plain<W, TM, TN, false><<<grid, 256, 0, s>>>(C, ldc, planeC, L, ldl, planeL, U, ldu, planeU, m, N, K);
}

template <int W>
int launch_gemm_plain_ptr(int64_t m, int64_t N, int K, double* C, int64_t ldc, int64_t planeC,
                          const double* L, int64_t ldl, int64_t planeL, const double* U, int64_t ldu,
                          int64_t planeU, cudaStream_t s, bool add) {
  if (m <= 0 || N <= 0 || K <= 0) return MW_OK;
  switch (gemm_plain_variant<W>(m, N)) {
    case 0: launch_gemm_variant<W, 0>(m, N, K, C, ldc, planeC, L, ldl, planeL, U, ldu, planeU, add, s); break;
    case 1: launch_gemm_variant<W, 1>(m, N, K, C, ldc, planeC, L, ldl, planeL, U, ldu, planeU, add, s); break;
    default: launch_gemm_variant<W, 2>(m, N, K, C, ldc, planeC, L, ldl, planeL, U, ldu, planeU, add, s); break;
  }
  MW_LAUNCH_CHECK();
  return MW_OK;
}
template int launch_gemm_plain_ptr<2>(int64_t, int64_t, int, double*, int64_t, int64_t, const double*, int64_t, int64_t, const double*, int64_t, int64_t, cudaStream_t, bool);
template int launch_gemm_plain_ptr<3>(int64_t, int64_t, int, double*, int64_t, int64_t, const double*, int64_t, int64_t, const double*, int64_t, int64_t, cudaStream_t, bool);
template int launch_gemm_plain_ptr<4>(int64_t, int64_t, int, double*, int64_t, int64_t, const double*, int64_t, int64_t, const double*, int64_t, int64_t, cudaStream_t, bool);

template <int W>
int launch_gemm_plain(double* A, int64_t lda, int64_t plane, int64_t row0, int64_t m,
                      int64_t col0, int64_t N, int64_t k0, int nb, cudaStream_t s) {
  return launch_gemm_plain_ptr<W>(m, N, nb, A + col0 * lda + row0, lda, plane, A + k0 * lda + row0, lda,
                                  plane, A + col0 * lda + k0, lda, plane, s);
}


// plain trailing update over a tile list
template <int W, int TM, int TN>
__global__ void __launch_bounds__(256)
k_bgemm_plain(BatchView bv, const TileEntry* __restrict__ tiles, int k0, double* __restrict__ A) {
  const TileEntry t = tiles[blockIdx.x];
  const int sys = bv.order[t.pos];
  const int n = bv.n[sys];
  const int r0 = k0 + kBatchNb;
  const int64_t m = n - r0;
  const int64_t plane = (int64_t)n * n;
  double* a = A + (int64_t)W * bv.moff[sys];
  gemm_plain_tile<W, TM, TN>(a + (int64_t)r0 * n + r0, n, plane, a + (int64_t)k0 * n + r0, n, plane,
                             a + (int64_t)r0 * n + k0, n, plane, m, m, kBatchNb, t.ti, t.tj);
}

void gemm_plain_tile_shape(int W, int* bm, int* bn) {
  switch (W) {
    case 2: *bm = 16 * GemmTile<2>::TM; *bn = 16 * GemmTile<2>::TN; break;
    case 3: *bm = 16 * GemmTile<3>::TM; *bn = 16 * GemmTile<3>::TN; break;
    default: *bm = 16 * GemmTile<4>::TM; *bn = 16 * GemmTile<4>::TN; break;
  }
}

template <int W>
int launch_bgemm_plain(const BatchView& bv, const TileEntry* tiles, int64_t ntiles, int k0, double* A,
                       cudaStream_t s) {
  if (ntiles <= 0) return MW_OK;
  constexpr int TM = GemmTile<W>::TM, TN = GemmTile<W>::TN;
  ProfScope ps(kPhGemmPlain, s);
  k_bgemm_plain<W, TM, TN><<<(unsigned)ntiles, 256, 0, s>>>(bv, tiles, k0, A);
  MW_LAUNCH_CHECK();
  return MW_OK;
}


template int launch_gemm_plain<2>(double*, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int,
                                  cudaStream_t);
template int launch_gemm_plain<3>(double*, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int,
                                  cudaStream_t);
template int launch_gemm_plain<4>(double*, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int,
                                  cudaStream_t);
template int launch_bgemm_plain<2>(const BatchView&, const TileEntry*, int64_t, int, double*, cudaStream_t);
template int launch_bgemm_plain<3>(const BatchView&, const TileEntry*, int64_t, int, double*, cudaStream_t);
template int launch_bgemm_plain<4>(const BatchView&, const TileEntry*, int64_t, int, double*, cudaStream_t);

}  // namespace mw
