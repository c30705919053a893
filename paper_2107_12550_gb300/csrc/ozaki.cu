// ozaki.cu -- split-precision (Ozaki scheme I) trailing update for DD on the
// Blackwell tensor cores: C -= L21 * U12 with C, L21, U12 double-double.
//
// The paper's trailing update is a DD block matrix product (Section 2,
// BNCmatmul).  Here it is reshaped for bf16 tcgen05 MMAs with FP32
// accumulation in tensor memory:
//
//  1. Scaling.  Row i of L21 is scaled by 2^-e_i and column j of U12 by 2^-f_j
//     (powers of two, e = ilogb(row/column max) + 2), so every scaled entry
//     lies in (-1/2, 1/2).
//  2. Slicing.  A scaled entry x is rounded toward minus infinity on the grid
//     2^-120 and written as 15 balanced base-256 digits,
//     x ~ sum_{p=1..15} a_p 2^(-8p), a_p in [-128, 127].  Each digit is a bf16
//     (exact: 8 significant bits).  Slices are stored per 128-row (L21) or
//     32-column (U12) tile in the 128-byte-swizzled K-major layout the MMA
//     reads, K = nb = 64.
//  3. Products.  Every pair (p, q) with p + q <= 16 accumulates A_p B_q^T
//     (128 x 16 x 64) into the FP32 accumulator of diagonal d = p + q (15
//     accumulators x 16 columns = 240 TMEM columns).  The B slices are
//     stored back to back, so for a fixed p the pairs q = 1 .. 16 - p form
//     ONE MMA of N = 16 (16 - p) columns whose output columns are exactly
//     those diagonals: 15 MMA instructions per K step instead of 120 narrow
//     ones, and each A tile is read from shared memory 15 times, not 120.  Diagonal d holds
//     the d - 1 pairs (p, q) with p + q = d, so at most 15 pairs (d = 16)
//     x 64 products of magnitude <= 2^14: every partial sum is an integer
//     of magnitude <= 15 * 64 * 2^14 = 15728640 < 2^24, and the FP32
//     accumulation is exact (kExactSumBound below checks this at compile
//     time; a 16th digit or K = 128 would break it).
//  4. Recombination.  Per output entry the 15 exact diagonal sums D_d are
//     combined in a 160-bit integer R = sum_d D_d 2^(8(16-d)); R 2^(e_i+f_j-128)
//     is the (truncated-digit) product L21 U12 exactly.  When both words of
//     C are integer multiples of that grid below 2^158 of it (the usual
//     case), C - P is formed exactly in the integer and rounded greedily to
//     DD once (recomb.cuh); otherwise, or when the result would be
//     subnormal, R is rounded greedily to DD and subtracted from C with the
//     DD subtraction.  oracle/ozaki.py states the same steps.
//
// Error per entry (stated per result in the tests): the dropped pairs
// p + q > 16 and the digit truncation give
// |dC_ij| <= 2^-111 * 2^(e_i + f_j) <= 2^-107 max_t|l_it| max_t|u_tj|,
// below the rounding of one DD multiply-subtract step.
#include <algorithm>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "mw_arith.cuh"
#include "mw_common.cuh"
#include "lu_internal.cuh"
#include "profile.cuh"
#include "tc.cuh"
#include "recomb.cuh"

namespace mw {

// exact power-of-two scaling, at most one rounding (defined below)
__device__ double scale2_exact(double x, int e);

namespace {

constexpr int kS = 15;                 // digits per operand
constexpr int kDiag = 15;              // diagonals d = 2..16
constexpr int kK = 64;                 // panel width (K of the update)
constexpr int kTileM = 128;            // rows per MMA tile
constexpr int kTileN = 16;             // columns per MMA tile
constexpr int kASliceBytes = kTileM * kK * 2;   // 16 KB
constexpr int kBSliceBytes = kTileN * kK * 2;   // 2 KB
constexpr uint32_t kTmemCols = 256;            // 15 x 16 = 240 used; two CTAs per SM
static_assert(kTileM == kSplitTileM && kTileN == kSplitTileN && kK == kBatchNb, "batched split tile shape");
// FP32 accumulation of a diagonal is exact while every partial sum stays an
// integer below 2^24: (most pairs on one diagonal) x K x (largest digit
// product 128 * 128)
constexpr long long kExactSumBound = (long long)kS * kK * 128 * 128;
static_assert(kExactSumBound < (1ll << 24), "diagonal sums must stay exact in FP32");

// byte offset of element (row r, k) inside a K-major 128B-swizzled tile
__device__ __forceinline__ uint32_t sw128_offset(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + (k & 7) * 2);
}

// magnitude bits of a double for a running maximum: |x| ordered as an
// unsigned integer; a NaN counts as zero (as fmax skips it)
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  return (u > 0x7ff0000000000000ull) ? 0ull : u;
}

__device__ __forceinline__ int exp_of_max(unsigned long long bits) {  // ilogb(mx) + 2 of mx's bits, mx > 0
  const int ex = (int)((bits >> 52) & 0x7ff);
  int lg;
  if (ex) lg = ex - 1023;
  else lg = -1074 + (63 - __clzll((long long)(bits & ((1ull << 52) - 1))));
  return lg + 2;
}

// floor(v * 2^sh) as a signed 128-bit integer (|result| < 2^126)
__device__ __forceinline__ __int128 scaled_floor(double v, int sh) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  if ((bits << 1) == 0ull) return 0;
  const bool neg = (bits >> 63) != 0;
  const int ex = (int)((bits >> 52) & 0x7ff);
  unsigned long long m = bits & ((1ull << 52) - 1);
  int e;
  if (ex) {
    m |= (1ull << 52);
    e = ex - 1075;
  } else {
    e = -1074;
  }
  const int s = e + sh;  // value = m * 2^s
  __int128 r;
  if (s >= 0) {
    r = (__int128)m << s;  // m 2^s < 2^119 by the choice of the scale, so s < 119
  } else if (s <= -64) {
    r = 0;  // |value| < 1 on the grid: floor gives 0 or -1
    if (neg) return -1;
    return 0;
  } else {
    const int rs = -s;
    const unsigned long long q = m >> rs;
    const bool rem = (m & ((1ull << rs) - 1)) != 0;
    r = (__int128)q;
    if (neg) return -(r) - (rem ? 1 : 0);
    return r;
  }
  return neg ? -r : r;
}

// 15 base-256 digits of X (|X| < 2^119), most significant first: the 14
// low digits balanced in [-128, 127], the top digit the exact remainder,
// within [-128, 128].  With Y = X + sum_{p<14} 128 256^p, the low digits are
// the bytes of Y minus 128 and the top digit is Y >> 112 (arithmetic): one
// 128-bit addition and byte extractions instead of a 14-step carry loop
// (balanced digits in [-128, 127] are unique, so both give the same digits)
__device__ __forceinline__ void digits15(__int128 X, int (&a)[kS]) {
  const unsigned __int128 bias = ((unsigned __int128)0x0000808080808080ull << 64) | 0x8080808080808080ull;
  const __int128 Y = X + (__int128)bias;
  const unsigned long long lo = (unsigned long long)Y;
  const unsigned long long hi = (unsigned long long)(Y >> 64);
#pragma unroll
  for (int p = 0; p < 8; ++p) a[kS - 1 - p] = (int)((lo >> (8 * p)) & 0xffull) - 128;
#pragma unroll
  for (int p = 0; p < 6; ++p) a[kS - 9 - p] = (int)((hi >> (8 * p)) & 0xffull) - 128;
  a[0] = (int)((long long)hi >> 48);
}

__device__ __forceinline__ unsigned short bf16_bits_of_int(int d) {
  const __nv_bfloat16 h = __float2bfloat16_rn((float)d);  // exact for |d| <= 256
  return *reinterpret_cast<const unsigned short*>(&h);
}

// ---------------------------------------------------------------------------
// slicing: row operand -> A slices [tile][p][128 x 64] with row exponents
// e_i; column operand -> B slices [tile][q][16 x 64] (column j is a K-major
// row) with column exponents f_j.  One CTA of 128 threads takes 16 rows (or
// columns) x 8 chunks of 8 k: each thread reads its 8 entries, the 8
// threads of a row combine their maxima in shared memory, and each thread
// writes the 16-byte swizzled piece of each of the 15 digit slices that its
// chunk fills.  Rows whose data are contiguous in i are read with
// consecutive threads on consecutive rows, rows contiguous in k with
// consecutive threads on consecutive chunks.  k >= kvalid: zero digits.
// ---------------------------------------------------------------------------
constexpr int kSliceRows = 16;   // rows (or columns) per CTA
constexpr int kSliceThreads = kSliceRows * (kK / 8);

// 8 entries (both words) of row or column r from k = kc*8; returns the
// magnitude bits of max |hi| (integer operations, off the FP64 pipe)
__device__ __forceinline__ unsigned long long slice_load8(const double* __restrict__ X, int64_t rs, int64_t ks, int64_t planeX,
                                              bool ok, int kvalid, int64_t r, int kc, double (&hv)[8],
                                              double (&lv)[8]) {
  unsigned long long mx = 0ull;
  // the entry addresses by pointer increments: a 64 x 64-bit index product
  // per entry would issue on the FP64 pipe
  const double* px = X + (ok ? r * rs + (int64_t)(kc * 8) * ks : 0);
#pragma unroll
  for (int k8 = 0; k8 < 8; ++k8, px += ks) {
    const int k = kc * 8 + k8;
    if (ok && k < kvalid) {
      hv[k8] = px[0];
      lv[k8] = px[planeX];
      const unsigned long long mb = mag_bits(hv[k8]);
      mx = (mb > mx) ? mb : mx;
    } else {
      hv[k8] = 0.0;
      lv[k8] = 0.0;
    }
  }
  return mx;
}

// the 15 digit pieces of 8 scaled entries (exponent e) -> dst + p * pstride
__device__ __forceinline__ void slice_store8(const double (&hv)[8], const double (&lv)[8], int e, bool live,
                                             unsigned char* __restrict__ dst, int pstride) {
  uint32_t packed[kS][4];
#pragma unroll
  for (int p = 0; p < kS; ++p)
#pragma unroll
    for (int h = 0; h < 4; ++h) packed[p][h] = 0u;
#pragma unroll
  for (int k8 = 0; k8 < 8; ++k8) {
    int a[kS];
    if (live) {
      const __int128 X = scaled_floor(hv[k8], 120 - e) + scaled_floor(lv[k8], 120 - e);
      digits15(X, a);
    } else {
#pragma unroll
      for (int p = 0; p < kS; ++p) a[p] = 0;
    }
#pragma unroll
    for (int p = 0; p < kS; ++p) packed[p][k8 >> 1] |= (uint32_t)bf16_bits_of_int(a[p]) << (16 * (k8 & 1));
  }
#pragma unroll
  for (int p = 0; p < kS; ++p) {
    uint4 v = make_uint4(packed[p][0], packed[p][1], packed[p][2], packed[p][3]);
    *reinterpret_cast<uint4*>(dst + (int64_t)p * pstride) = v;
  }
}

// rows [rbase, rbase + 16) of the row operand (element (r, k) at L[r*lrs + k*lks])
__device__ __forceinline__ void slice_rows16(const double* __restrict__ L, int64_t lrs, int64_t lks,
                                             int64_t planeL, int64_t m, int kvalid,
                                             unsigned char* __restrict__ aslices, int* __restrict__ ea,
                                             int64_t rbase) {
  __shared__ unsigned long long smx[kSliceRows][kK / 8];
  const int tid = threadIdx.x;
  const bool rows_fast = lrs == 1;
  const int rl = rows_fast ? (tid & (kSliceRows - 1)) : (tid >> 3);
  const int kc = rows_fast ? (tid / kSliceRows) : (tid & 7);
  const int64_t r = rbase + rl;
  const bool ok = r < m;
  double hv[8], lv[8];
  smx[rl][kc] = slice_load8(L, lrs, lks, planeL, ok, kvalid, r, kc, hv, lv);
  __syncthreads();
  unsigned long long mx = 0ull;
#pragma unroll
  for (int q = 0; q < kK / 8; ++q) mx = (smx[rl][q] > mx) ? smx[rl][q] : mx;
  const int e = mx ? exp_of_max(mx) : 0;
  if (kc == 0) ea[r] = e;
  const int64_t tile = r / kTileM;
  const int rr = (int)(r % kTileM);
  slice_store8(hv, lv, e, ok && mx != 0ull && kc * 8 < kvalid,
               aslices + tile * (int64_t)kS * kASliceBytes + sw128_offset(rr, kc * 8), kASliceBytes);
}

// columns [jbase, jbase + 16) of the column operand (element (k, j) at U[k*uks + j*ujs])
__device__ __forceinline__ void slice_cols16(const double* __restrict__ U, int64_t uks, int64_t ujs,
                                             int64_t planeU, int64_t N, int kvalid,
                                             unsigned char* __restrict__ bslices, int* __restrict__ fb,
                                             int64_t jbase) {
  __shared__ unsigned long long smx[kSliceRows][kK / 8];
  const int tid = threadIdx.x;
  const bool cols_fast = ujs == 1;
  const int jl = cols_fast ? (tid & (kSliceRows - 1)) : (tid >> 3);
  const int kc = cols_fast ? (tid / kSliceRows) : (tid & 7);
  const int64_t j = jbase + jl;
  const bool ok = j < N;
  double hv[8], lv[8];
  smx[jl][kc] = slice_load8(U, ujs, uks, planeU, ok, kvalid, j, kc, hv, lv);
  __syncthreads();
  unsigned long long mx = 0ull;
#pragma unroll
  for (int q = 0; q < kK / 8; ++q) mx = (smx[jl][q] > mx) ? smx[jl][q] : mx;
  const int f = mx ? exp_of_max(mx) : 0;
  if (kc == 0) fb[j] = f;
  const int64_t tile = j / kTileN;
  const int jj = (int)(j % kTileN);
  slice_store8(hv, lv, f, ok && mx != 0ull && kc * 8 < kvalid,
               bslices + tile * (int64_t)kS * kBSliceBytes + sw128_offset(jj, kc * 8), kBSliceBytes);
}

// grid: (rows padded to 128) / 16
__global__ void __launch_bounds__(kSliceThreads)
k_slice_rows(SplitOperands o, unsigned char* __restrict__ aslices, int* __restrict__ ea) {
  slice_rows16(o.L, o.lrs, o.lks, o.planeL, o.m, o.K, aslices, ea, (int64_t)blockIdx.x * kSliceRows);
}

// grid: (columns padded to 32) / 16
__global__ void __launch_bounds__(kSliceThreads)
k_slice_cols(SplitOperands o, unsigned char* __restrict__ bslices, int* __restrict__ fb) {
  slice_cols16(o.U, o.uks, o.ujs, o.planeU, o.N, o.K, bslices, fb, (int64_t)blockIdx.x * kSliceRows);
}

// ---------------------------------------------------------------------------
// 192-bit two's-complement accumulator and greedy rounding to DD
// ---------------------------------------------------------------------------
struct I192 {
  unsigned long long w0, w1, w2;
};

__device__ __forceinline__ int i192_top(const I192& R) {  // index of highest set bit, -1 if 0
  if (R.w2) return 128 + 63 - __clzll((long long)R.w2);
  if (R.w1) return 64 + 63 - __clzll((long long)R.w1);
  if (R.w0) return 63 - __clzll((long long)R.w0);
  return -1;
}

__device__ __forceinline__ void i192_neg(I192& R) {
  R.w0 = ~R.w0;
  R.w1 = ~R.w1;
  R.w2 = ~R.w2;
  R.w0 += 1;
  const unsigned long long c0 = (R.w0 == 0);
  R.w1 += c0;
  R.w2 += (c0 && R.w1 == 0);
}

// subtract q * 2^lo from a non-negative R (q <= 2^53, result may go negative)
__device__ __forceinline__ void i192_sub_shifted(I192& R, unsigned long long q, int lo) {
  unsigned __int128 v = (unsigned __int128)q << (lo & 63);
  const unsigned long long vlo = (unsigned long long)v, vhi = (unsigned long long)(v >> 64);
  if (lo < 64) {
    const unsigned long long b0 = R.w0 < vlo;
    R.w0 -= vlo;
    const unsigned long long t = R.w1 - vhi;
    const unsigned long long b1a = R.w1 < vhi;
    const unsigned long long b1b = t < b0;
    R.w1 = t - b0;
    R.w2 -= (b1a + b1b);
  } else if (lo < 128) {
    const unsigned long long b1 = R.w1 < vlo;
    R.w1 -= vlo;
    R.w2 -= vhi + b1;
  } else {
    R.w2 -= vlo;
  }
}

// the 160-bit product integer widened to 192 bits (sign-extended)
__device__ __forceinline__ I192 to_i192(const rc::I160& r) {
  I192 R;
  R.w0 = (unsigned long long)r.l0 | ((unsigned long long)r.l1 << 32);
  R.w1 = (unsigned long long)r.l2 | ((unsigned long long)r.l3 << 32);
  R.w2 = (unsigned long long)(long long)(int)r.l4;
  return R;
}

// x * 2^k for an integer-valued double x: the exponent field moved when the
// result stays normal, the FP64 route otherwise
__device__ __forceinline__ double scale_pow2(double x, int k) {
  const long long bits = __double_as_longlong(x);
  if (((unsigned long long)bits << 1) == 0ull) return x;   // +-0, tested off the FP64 pipe
  const int ex = (int)((bits >> 52) & 0x7ff);
  if (ex + k >= 1 && ex + k <= 2046) return __longlong_as_double(bits + ((long long)k << 52));
  return scale2_exact(x, k);
}

// RN of a non-negative M (top = index of its highest set bit) as double d
// with M ~ d * 2^shift: the 64 bits below and including the top bit, with
// the OR of every lower bit folded into bit 0, round to the same 53 bits as
// M itself (the rounding position is bit 10 of the window), so the
// hardware's RN conversion of that window is RN(M)
__device__ __forceinline__ double i192_window_rn(const I192& M, int top, int& shift) {
  if (top < 64) {
    shift = 0;
    return __ull2double_rn(M.w0);
  }
  const int sh = top - 63;   // 1 .. 128
  unsigned long long w, sticky;
  if (sh < 64) {
    w = (M.w1 << (64 - sh)) | (M.w0 >> sh);
    sticky = M.w0 & ((1ull << sh) - 1);
  } else if (sh == 64) {
    w = M.w1;
    sticky = M.w0;
  } else {
    const int s2 = sh - 64;   // 1 .. 64
    w = (s2 < 64) ? ((M.w2 << (64 - s2)) | (M.w1 >> s2)) : M.w2;
    sticky = M.w0 | ((s2 < 64) ? (M.w1 & ((1ull << s2) - 1)) : M.w1);
  }
  shift = sh;
  return __ull2double_rn(w | (sticky ? 1ull : 0ull));
}

// greedy rounding of the signed R * 2^scale to two doubles: hi = RN(v),
// lo = RN(v - hi)
__device__ __forceinline__ void i192_to_dd(I192 R, int scale, double& hi, double& lo) {
  const bool neg = (long long)R.w2 < 0;
  if (neg) i192_neg(R);
  const int top = i192_top(R);
  hi = lo = 0.0;
  if (top < 0) return;
  int sh;
  const double hd = i192_window_rn(R, top, sh);
  // subtract RN(M) = mant * 2^(ex - 52 + sh) exactly
  const unsigned long long hb = (unsigned long long)__double_as_longlong(hd);
  const int ex = (int)((hb >> 52) & 0x7ff) - 1023;
  const unsigned long long mant = (hb & ((1ull << 52) - 1)) | (1ull << 52);
  const int pos = ex - 52 + sh;
  double ld = 0.0;
  int sh2 = 0;
  bool lneg = false;
  if (pos >= 0) {   // otherwise M < 2^53 and the conversion was exact
    i192_sub_shifted(R, mant, pos);
    lneg = (long long)R.w2 < 0;
    if (lneg) i192_neg(R);
    const int top2 = i192_top(R);
    if (top2 >= 0) ld = i192_window_rn(R, top2, sh2);
  }
  hi = scale_pow2(neg ? -hd : hd, sh + scale);
  lo = scale_pow2((neg != lneg) ? -ld : ld, sh2 + scale);
}

// ---------------------------------------------------------------------------
// the tensor-core kernel: one CTA per 128 x 16 output tile, two CTAs per SM
// warp 0: bulk-copy producer; warp 1: TMEM owner + MMA issuer;
// warps 2..9: epilogue (TMEM lane quarter = warp % 4; warps 2..5 take
// columns 0..7 of the tile, warps 6..9 columns 8..15)
// ---------------------------------------------------------------------------
struct SplitSmem {
  unsigned char b[kS][kBSliceBytes];       // all B slices of the tile (60 KB)
  unsigned char a[2][kASliceBytes];        // double-buffered A slice (32 KB)
  uint64_t full_b;
  uint64_t full_a[2];
  uint64_t empty_a[2];
  uint64_t mma_done;
  uint32_t tmem_base;
  int abort;
};

constexpr int kEpiWarps = 8;                       // two warpgroups over the 4 TMEM lane quarters
constexpr int kSplitThreads = 64 + 32 * kEpiWarps;  // producer + MMA warps + epilogue

// entry (i, j) of C at C[i * crs + j * cjs]
__device__ __forceinline__ void split_tile(double* __restrict__ C, int64_t crs, int64_t cjs, int64_t planeC, int64_t m,
                                           int64_t N, const unsigned char* __restrict__ aslices,
                                           const unsigned char* __restrict__ bslices,
                                           const int* __restrict__ ea, const int* __restrict__ fb,
                                           DeviceStatus* status, int64_t tm, int64_t tn, bool plus = false) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzle atoms
  SplitSmem& sm = *reinterpret_cast<SplitSmem*>(
      (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    tc::mbar_init(&sm.full_b, 1);
    tc::mbar_init(&sm.full_a[0], 1);
    tc::mbar_init(&sm.full_a[1], 1);
    tc::mbar_init(&sm.empty_a[0], 1);
    tc::mbar_init(&sm.empty_a[1], 1);
    tc::mbar_init(&sm.mma_done, 1);
    sm.abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) tc::tmem_alloc(&sm.tmem_base, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = sm.tmem_base;

  int issued = 0;   // A slices whose copies the producer started
  if (warp == 0) {
    if (lane == 0) {
      const unsigned char* bsrc = bslices + tn * (int64_t)kS * kBSliceBytes;
      tc::mbar_arrive_expect_tx(&sm.full_b, kS * kBSliceBytes);
      tc::bulk_g2s(&sm.b[0][0], bsrc, kS * kBSliceBytes, &sm.full_b);
      const unsigned char* asrc = aslices + tm * (int64_t)kS * kASliceBytes;
      for (int p = 0; p < kS; ++p) {
        const int buf = p & 1;
        if (p >= 2) {
          if (!tc::mbar_wait(&sm.empty_a[buf], ((p >> 1) - 1) & 1)) {
            atomicExch(&sm.abort, 1);
            break;
          }
        }
        tc::mbar_arrive_expect_tx(&sm.full_a[buf], kASliceBytes);
        tc::bulk_g2s(&sm.a[buf][0], asrc + (int64_t)p * kASliceBytes, kASliceBytes, &sm.full_a[buf]);
        issued = p + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = tc::mbar_wait(&sm.full_b, 0);
      const uint32_t b_addr = tc::smem_u32(&sm.b[0][0]);
      for (int p = 0; p < kS && ok; ++p) {
        const int buf = p & 1;
        if (!tc::mbar_wait(&sm.full_a[buf], (p >> 1) & 1)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t a_addr = tc::smem_u32(&sm.a[buf][0]);
        // digit p of A against digits q = 0 .. 14 - p of B in ONE product:
        // the B slices lie back to back (16 rows each, 1024-byte atoms), so
        // they form one operand of 16 (15 - p) rows, and pair (p, q) lands
        // in the accumulator of diagonal p + q, whose columns start at
        // (p + q) 16: the product's columns are exactly diagonals p .. 14
        const uint32_t dcol = tmem + (uint32_t)(p * kTileN);
        const uint32_t idesc = tc::idesc_bf16_f32(kTileM, kTileN * (kS - p));
#pragma unroll
        for (int kk = 0; kk < kK / 16; ++kk) {
          const uint64_t adesc = tc::sdesc_sw128_kmajor(a_addr + kk * 32);
          const uint64_t bdesc = tc::sdesc_sw128_kmajor(b_addr + kk * 32);
          tc::mma_bf16(dcol, adesc, bdesc, idesc, (p > 0 || kk > 0) ? 1u : 0u);
        }
        tc::mma_commit(&sm.empty_a[buf]);   // frees the A buffer when these MMAs finish
      }
      if (!ok) atomicExch(&sm.abort, 1);
      tc::mma_commit(&sm.mma_done);
    }
  } else {
    // epilogue: thread <-> row (TMEM lane) of the tile, half of the columns
    const int quarter = warp & 3;
    constexpr int kCols = kTileN / (kEpiWarps / 4);   // columns per epilogue warp
    constexpr int CW = 2;                             // columns per TMEM read
    const int cpart = (warp - 2) / 4;
    const int rr = quarter * 32 + lane;
    const int64_t i = tm * kTileM + rr;
    const int64_t jw = tn * kTileN + cpart * kCols;   // first column of this warp
    // C entries of a chunk, loaded one chunk ahead so that their latency
    // overlaps the MMAs (first chunk) or the previous chunk's work
    auto load_chunk = [&](int ch, val<2> (&cv)[CW]) {
#pragma unroll
      for (int cc = 0; cc < CW; ++cc) {
        const int64_t j = jw + ch * CW + cc;
        if (i < m && j < N) cv[cc] = load<2>(C, planeC, i * crs + j * cjs);
      }
    };
    val<2> cnext[CW];
    load_chunk(0, cnext);
    // the row and column scale exponents, also before the wait
    const int ei = (i < m) ? ea[i] : 0;
    int fbv[kCols];
#pragma unroll
    for (int k = 0; k < kCols; ++k) fbv[k] = (jw + k < N) ? fb[jw + k] : 0;
    bool ok = tc::mbar_wait(&sm.mma_done, 0);
    tc::tc_fence_after();
    // one decision per warp: the TMEM loads below are warp-collective
    ok = __all_sync(0xffffffffu, ok && (*(volatile int*)&sm.abort == 0));
    if (!ok) {
      if (threadIdx.x == 64) atomicExch(&status->timeout, 1u);
    } else {
      const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
      for (int ch = 0; ch < kCols / CW; ++ch) {
        const int c0 = cpart * kCols + ch * CW;
        val<2> cvs[CW];
#pragma unroll
        for (int cc = 0; cc < CW; ++cc) cvs[cc] = cnext[cc];
        if (ch + 1 < kCols / CW) load_chunk(ch + 1, cnext);
        uint32_t v[kDiag][CW];
#pragma unroll
        for (int d = 0; d < kDiag; ++d) tc::tmem_ld_x2(lane_base + (uint32_t)(d * kTileN + c0), v[d]);
        tc::tmem_ld_wait();
#pragma unroll
        for (int cc = 0; cc < CW; ++cc) {
          const int64_t j = jw + ch * CW + cc;
          if (i >= m || j >= N) continue;
          int D[kDiag];
#pragma unroll
          for (int d = 0; d < kDiag; ++d) D[d] = __float2int_rn(__uint_as_float(v[d][cc]));
          const int scale = ei + fbv[ch * CW + cc] - 128;
          const int64_t idx = i * crs + j * cjs;
          val<2> cv = cvs[cc];
          // exact form: T = P + C (plus) or P - C, both C words added on the
          // product's grid 2^scale, then the greedy DD rounding of T (plus)
          // or -T; the other form (C off the grid or out of the 160-bit
          // range, or a subnormal result) rounds P to DD and uses the DD
          // addition (subtraction)
          rc::I160 T = rc::diag_sum(D);
          const unsigned long long flipc = plus ? 0ull : 0x8000000000000000ull;
          const double w0 = __longlong_as_double((long long)((unsigned long long)__double_as_longlong(cv.v[0]) ^ flipc));
          const double w1 = __longlong_as_double((long long)((unsigned long long)__double_as_longlong(cv.v[1]) ^ flipc));
          double rh, rl;
          if (rc::add_word(T, w0, scale) && rc::add_word(T, w1, scale) && rc::round_dd(T, scale, !plus, rh, rl)) {
            cv.v[0] = rh;
            cv.v[1] = rl;
          } else {
            val<2> pr;
            i192_to_dd(to_i192(rc::diag_sum(D)), scale, pr.v[0], pr.v[1]);
            cv = plus ? add<2>(cv, pr) : sub<2>(cv, pr);
          }
          store<2>(C, planeC, idx, cv);
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0 && lane == 0 && sm.abort) {
    // after an aborted tile, let the copies this thread started land before
    // the CTA's shared memory is released (bounded waits)
    tc::mbar_wait(&sm.full_b, 0);
    for (int p = (issued > 2 ? issued - 2 : 0); p < issued; ++p) tc::mbar_wait(&sm.full_a[p & 1], (p >> 1) & 1);
  }
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

__global__ void __launch_bounds__(kSplitThreads, 2)
k_split_gemm(SplitOperands o, const unsigned char* __restrict__ aslices, const unsigned char* __restrict__ bslices,
             const int* __restrict__ ea, const int* __restrict__ fb, DeviceStatus* status) {
  split_tile(o.C, o.crs, o.cjs, o.planeC, o.m, o.N, aslices, bslices, ea, fb, status, blockIdx.x, blockIdx.y,
             o.plus != 0);
}

// ---- batched forms: per active system of a batch at panel step k0 ----------
// Operand geometry of one split product C -= L U inside system `a` (lda = n):
//  kGeomTrail: the trailing update, L = L21 (rows [r0, n) of columns
//    [k0, r0)), U = U12, C = A22, r0 = k0 + 64;
//  kGeomTrsmInv: U12 := U12 - M U12 with M the strictly lower part of
//    -(L11^-1) (64 x 64, column-major in `aux`), which is U12 := L11^-1 U12,
//    in transposed form C^T -= U12^T M^T: the rows of the product are the
//    columns of U12;
//  kGeomPanelInner: inside the panel, for a block of 2h columns starting at
//    column k0 + c_off whose left h columns are factored and whose right
//    half's top h rows are solved: the right half's rows below them
//    -= L (left half, same rows) U (the solved rows), K = h (zero digits
//    beyond).
__device__ __forceinline__ SplitOperands batch_operands(int geom, double* a, int n, int k0, const double* aux,
                                                        int c_off, int h) {
  SplitOperands o;
  const int64_t plane = (int64_t)n * n;
  const int r0 = k0 + kK;
  o.K = kK;
  if (geom == kGeomPanelInner) {
    const int c0 = k0 + c_off;
    const int q0 = c0 + h;
    o.L = a + (int64_t)c0 * n + q0;
    o.lrs = 1;
    o.lks = n;
    o.planeL = plane;
    o.U = a + (int64_t)q0 * n + c0;
    o.uks = 1;
    o.ujs = n;
    o.planeU = plane;
    o.C = a + (int64_t)q0 * n + q0;
    o.crs = 1;
    o.cjs = n;
    o.planeC = plane;
    o.m = n - q0;
    o.N = min(h, n - q0);
    o.K = h;
  } else if (geom == kGeomTrsmInv) {
    o.L = a + (int64_t)r0 * n + k0;   // (j, t) -> U12(t, j)
    o.lrs = n;
    o.lks = 1;
    o.planeL = plane;
    o.U = aux;                        // (t, i) -> M(i, t)
    o.uks = kK;
    o.ujs = 1;
    o.planeU = (int64_t)kK * kK;
    o.C = a + (int64_t)r0 * n + k0;   // (j, i) -> U12(i, j)
    o.crs = n;
    o.cjs = 1;
    o.planeC = plane;
    o.m = n - r0;
    o.N = kK;
  } else {
    o.L = a + (int64_t)k0 * n + r0;
    o.lrs = 1;
    o.lks = n;
    o.planeL = plane;
    o.U = a + (int64_t)r0 * n + k0;
    o.uks = 1;
    o.ujs = n;
    o.planeU = plane;
    o.C = a + (int64_t)r0 * n + r0;
    o.crs = 1;
    o.cjs = n;
    o.planeC = plane;
    o.m = n - r0;
    o.N = n - r0;
  }
  return o;
}

// grid (act, 8 * max_mt): 16 rows blockIdx.y of system order[blockIdx.x]
__global__ void __launch_bounds__(kSliceThreads)
k_bslice_rows(BatchView bv, int geom, int c_off, int h, const int2* __restrict__ bases, int k0,
              double* __restrict__ A, const double* __restrict__ aux, unsigned char* __restrict__ aslices,
              int* __restrict__ ea) {
  const int pos = blockIdx.x;
  const int sys = bv.order[pos];
  const int n = bv.n[sys];
  const SplitOperands o =
      batch_operands(geom, A + 2 * bv.moff[sys], n, k0, aux + (int64_t)pos * 2 * kK * kK, c_off, h);
  const int64_t rbase = (int64_t)blockIdx.y * kSliceRows;
  if (o.m <= 0 || o.N <= 0 || rbase >= (o.m + kTileM - 1) / kTileM * kTileM) return;   // uniform per CTA
  const int abase = bases[pos].x;
  slice_rows16(o.L, o.lrs, o.lks, o.planeL, o.m, o.K, aslices + (int64_t)abase * kS * kASliceBytes,
               ea + (int64_t)abase * kTileM, rbase);
}

// grid (act, 8 * max_cb): 16 columns blockIdx.y of system order[blockIdx.x]
__global__ void __launch_bounds__(kSliceThreads)
k_bslice_cols(BatchView bv, int geom, int c_off, int h, const int2* __restrict__ bases, int k0,
              double* __restrict__ A, const double* __restrict__ aux, unsigned char* __restrict__ bslices,
              int* __restrict__ fb) {
  const int pos = blockIdx.x;
  const int sys = bv.order[pos];
  const int n = bv.n[sys];
  const SplitOperands o =
      batch_operands(geom, A + 2 * bv.moff[sys], n, k0, aux + (int64_t)pos * 2 * kK * kK, c_off, h);
  const int64_t jbase = (int64_t)blockIdx.y * kSliceRows;
  if (o.m <= 0 || o.N <= 0 || jbase >= (o.N + kTileN - 1) / kTileN * kTileN) return;   // uniform per CTA
  const int bbase = bases[pos].y;
  slice_cols16(o.U, o.uks, o.ujs, o.planeU, o.N, o.K, bslices + (int64_t)bbase * kS * kBSliceBytes,
               fb + (int64_t)bbase * kTileN, jbase);
}

__global__ void __launch_bounds__(kSplitThreads, 2)
k_bsplit_gemm(BatchView bv, int geom, int c_off, int h, const TileEntry* __restrict__ tiles,
              const int2* __restrict__ bases, int k0, double* __restrict__ A, const double* __restrict__ aux,
              const unsigned char* __restrict__ aslices, const unsigned char* __restrict__ bslices,
              const int* __restrict__ ea, const int* __restrict__ fb, DeviceStatus* status) {
  const TileEntry t = tiles[blockIdx.x];
  const int sys = bv.order[t.pos];
  const int n = bv.n[sys];
  const SplitOperands o =
      batch_operands(geom, A + 2 * bv.moff[sys], n, k0, aux + (int64_t)t.pos * 2 * kK * kK, c_off, h);
  const int2 b = bases[t.pos];
  split_tile(o.C, o.crs, o.cjs, o.planeC, o.m, o.N, aslices + (int64_t)b.x * kS * kASliceBytes,
             bslices + (int64_t)b.y * kS * kBSliceBytes, ea + (int64_t)b.x * kTileM, fb + (int64_t)b.y * kTileN,
             status, t.ti, t.tj);
}

// M = strictly lower part of -(L11^-1) for every active system with columns
// right of the panel; L11 = the unit lower 64 x 64 block at (k0, k0).
// X = L11^-1 by column-oriented substitution on all 64 columns of the
// identity at once: for t ascending, x_it -= l_it x_tc for i > t, c <= t.
// dynamic shared memory: X, 2 words x 64 x 64 doubles
__device__ __forceinline__ void inv_l11_body(const double* __restrict__ a, int64_t lda, int64_t plane, int k0,
                                             double* __restrict__ m) {
  extern __shared__ double xs[];     // [2][64 cols][64 rows]
  constexpr int P = kK * kK;
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    const int c = e / kK, i = e % kK;
    xs[e] = (i == c) ? 1.0 : 0.0;
    xs[P + e] = 0.0;
  }
  for (int t = 0; t < kK - 1; ++t) {
    __syncthreads();
    const int rows = kK - 1 - t;          // i in (t, 64)
    const int items = rows * (t + 1);     // c in [0, t]
    const int64_t lcol = (int64_t)(k0 + t) * lda + k0;
    for (int q = threadIdx.x; q < items; q += blockDim.x) {
      const int i = t + 1 + q % rows, c = q / rows;
      val<2> x, l, u;
      x.v[0] = xs[c * kK + i];
      x.v[1] = xs[P + c * kK + i];
      l.v[0] = __ldg(a + lcol + i);
      l.v[1] = __ldg(a + plane + lcol + i);
      u.v[0] = xs[c * kK + t];
      u.v[1] = xs[P + c * kK + t];
      x = msub<2>(x, l, u);
      xs[c * kK + i] = x.v[0];
      xs[P + c * kK + i] = x.v[1];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    const int c = e / kK, i = e % kK;
    const bool below = i > c;
    m[e] = below ? -xs[e] : 0.0;
    m[P + e] = below ? -xs[P + e] : 0.0;
  }
}

__global__ void __launch_bounds__(256)
k_binv_l11(BatchView bv, int k0, const double* __restrict__ A, double* __restrict__ aux) {
  const int pos = blockIdx.x;
  const int sys = bv.order[pos];
  const int n = bv.n[sys];
  if (n - k0 - kK <= 0) return;
  inv_l11_body(A + 2 * bv.moff[sys], n, (int64_t)n * n, k0, aux + (int64_t)pos * 2 * kK * kK);
}

// one system with leading dimension lda: one CTA per column c of X = L11^-1
// (thread i holds X(i, c)), the same operations per entry as inv_l11_body:
// for t ascending from c, X(i, c) -= l_it X(t, c) for i > t.
// dynamic shared memory: L11, 2 words x 64 x 64 doubles
__global__ void __launch_bounds__(kK)
k_inv_l11_cols(const double* __restrict__ A, int64_t lda, int64_t plane, int k0, double* __restrict__ aux) {
  extern __shared__ double ls[];     // [2][64 cols t][64 rows i]
  __shared__ double xt[2];
  constexpr int P = kK * kK;
  const int c = blockIdx.x, i = threadIdx.x;
  for (int e = i; e < P; e += kK) {
    const int t = e / kK, r = e % kK;
    const int64_t idx = (int64_t)(k0 + t) * lda + k0 + r;
    ls[e] = __ldg(A + idx);
    ls[P + e] = __ldg(A + plane + idx);
  }
  val<2> x;
  x.v[0] = (i == c) ? 1.0 : 0.0;
  x.v[1] = 0.0;
  for (int t = c; t < kK - 1; ++t) {
    __syncthreads();
    if (i == t) {
      xt[0] = x.v[0];
      xt[1] = x.v[1];
    }
    __syncthreads();
    if (i > t) {
      val<2> l, u;
      l.v[0] = ls[t * kK + i];
      l.v[1] = ls[P + t * kK + i];
      u.v[0] = xt[0];
      u.v[1] = xt[1];
      x = msub<2, false>(x, l, u);
    }
  }
  const bool below = i > c;
  aux[c * kK + i] = below ? -x.v[0] : 0.0;
  aux[P + c * kK + i] = below ? -x.v[1] : 0.0;
}

size_t split_smem_bytes() {
  // at least 100 KB: never more than two CTAs (2 x 256 TMEM columns) on one SM
  return (sizeof(SplitSmem) + 1024 > 100 * 1024) ? sizeof(SplitSmem) + 1024 : 100 * 1024;
}

}  // namespace

__device__ double scale2_exact(double x, int e) {
  while (e > 1000) {
    x = __dmul_rn(x, 0x1p+1000);
    e -= 1000;
  }
  while (e < -1000) {
    x = __dmul_rn(x, 0x1p-1000);
    e += 1000;
  }
  return __dmul_rn(x, __longlong_as_double((long long)(e + 1023) << 52));
}

// workspace: [status 256 | A slices | B slices | ea | fb | L11 inverse (2 x 64 x 64)]
static size_t split_slices_bytes(int64_t n) {
  const int64_t mt = (n + kTileM - 1) / kTileM, nt = (n + kTileN - 1) / kTileN;
  return 256 + align256((size_t)mt * kS * kASliceBytes) + align256((size_t)nt * kS * kBSliceBytes) +
         align256(sizeof(int) * (size_t)mt * kTileM) + align256(sizeof(int) * (size_t)nt * kTileN);
}

size_t split_workspace_bytes(int64_t n, int nb) {
  (void)nb;
  return split_slices_bytes(n) + align256(sizeof(double) * 2 * kK * kK);
}

double* split_aux(char* ws, int64_t n) { return reinterpret_cast<double*>(ws + split_slices_bytes(n)); }

size_t split_product_bytes(int64_t m, int64_t N) {
  const int64_t mt = (m + kTileM - 1) / kTileM, nt = (N + kTileN - 1) / kTileN;
  return 256 + align256((size_t)mt * kS * kASliceBytes) + align256((size_t)nt * kS * kBSliceBytes) +
         align256(sizeof(int) * (size_t)mt * kTileM) + align256(sizeof(int) * (size_t)nt * kTileN);
}

// C (m x N) -= L (m x K) * U (K x N) with the strides of `o` (K <= 64)
int split_product_dd(const SplitOperands& o, char* ws, size_t ws_bytes, int phase, cudaStream_t s) {
  if (o.m <= 0 || o.N <= 0 || o.K <= 0) return MW_OK;
  if (o.K > kK) return MW_EUNSUPPORTED;
  const int64_t mt = (o.m + kTileM - 1) / kTileM, nt = (o.N + kTileN - 1) / kTileN;
  size_t off = 256;
  unsigned char* aslices = reinterpret_cast<unsigned char*>(ws + off);
  off += align256((size_t)mt * kS * kASliceBytes);
  unsigned char* bslices = reinterpret_cast<unsigned char*>(ws + off);
  off += align256((size_t)nt * kS * kBSliceBytes);
  int* ea = reinterpret_cast<int*>(ws + off);
  off += align256(sizeof(int) * (size_t)mt * kTileM);
  int* fb = reinterpret_cast<int*>(ws + off);
  off += align256(sizeof(int) * (size_t)nt * kTileN);
  if (off > ws_bytes) return MW_EUNSUPPORTED;
  DeviceStatus* status = reinterpret_cast<DeviceStatus*>(ws + kWsStatus);
  {
    ProfScope ps(kPhSplitAux, s);
    k_slice_rows<<<(unsigned)(mt * kTileM / kSliceRows), kSliceThreads, 0, s>>>(o, aslices, ea);
    MW_LAUNCH_CHECK();
    k_slice_cols<<<(unsigned)(nt * kTileN / kSliceRows), kSliceThreads, 0, s>>>(o, bslices, fb);
    MW_LAUNCH_CHECK();
  }
  {
    ProfScope ps(phase, s);
    const size_t shmem = split_smem_bytes();
    MW_CUDA_CHECK(ensure_smem_limit(k_split_gemm, shmem));
    dim3 grid((unsigned)mt, (unsigned)nt);
    k_split_gemm<<<grid, kSplitThreads, shmem, s>>>(o, aslices, bslices, ea, fb, status);
    MW_LAUNCH_CHECK();
  }
  return MW_OK;
}

// C (m x N) -= L (m x 64) * U (64 x N), all DD component-planar column-major
int split_gemm_sub_dd(int64_t m, int64_t N, double* C, int64_t ldc, int64_t planeC, const double* L,
                      int64_t ldl, int64_t planeL, const double* U, int64_t ldu, int64_t planeU,
                      char* ws, size_t ws_bytes, cudaStream_t s, bool plus) {
  SplitOperands o;
  o.plus = plus ? 1 : 0;
  o.L = L;
  o.lrs = 1;
  o.lks = ldl;
  o.planeL = planeL;
  o.U = U;
  o.uks = 1;
  o.ujs = ldu;
  o.planeU = planeU;
  o.C = C;
  o.crs = 1;
  o.cjs = ldc;
  o.planeC = planeC;
  o.m = m;
  o.N = N;
  o.K = kK;
  return split_product_dd(o, ws, ws_bytes, kPhGemmSplit, s);
}

int split_inv_l11(const double* A, int64_t lda, int64_t plane, int64_t k0, double* aux, cudaStream_t s) {
  const size_t shmem = sizeof(double) * 2 * kK * kK;
  MW_CUDA_CHECK(ensure_smem_limit(k_inv_l11_cols, shmem));
  ProfScope ps(kPhTrsm, s);
  k_inv_l11_cols<<<kK, kK, shmem, s>>>(A, lda, plane, (int)k0, aux);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

// batched: [status 256 | A slices | B slices | ea | fb]
size_t split_batched_workspace_bytes(int64_t a_tiles, int64_t b_tiles) {
  return 256 + align256((size_t)a_tiles * kS * kASliceBytes) + align256((size_t)b_tiles * kS * kBSliceBytes) +
         align256(sizeof(int) * (size_t)a_tiles * kTileM) + align256(sizeof(int) * (size_t)b_tiles * kTileN);
}

namespace {
struct BSliceArea {
  unsigned char* aslices;
  unsigned char* bslices;
  int* ea;
  int* fb;
};
BSliceArea bslice_area(char* ws, int64_t a_tiles, int64_t b_tiles) {
  BSliceArea r;
  size_t off = 256;
  r.aslices = reinterpret_cast<unsigned char*>(ws + off);
  off += align256((size_t)a_tiles * kS * kASliceBytes);
  r.bslices = reinterpret_cast<unsigned char*>(ws + off);
  off += align256((size_t)b_tiles * kS * kBSliceBytes);
  r.ea = reinterpret_cast<int*>(ws + off);
  off += align256(sizeof(int) * (size_t)a_tiles * kTileM);
  r.fb = reinterpret_cast<int*>(ws + off);
  return r;
}
}  // namespace

int split_bslice_dd(const BatchView& bv, int geom, int c_off, int h, int act, int max_mt, int max_cb,
                    const int2* bases, int64_t a_tiles, int64_t b_tiles, int k0, double* A, const double* aux,
                    char* ws, size_t ws_bytes, cudaStream_t s) {
  if (act <= 0) return MW_OK;
  if (split_batched_workspace_bytes(a_tiles, b_tiles) > ws_bytes) return MW_EUNSUPPORTED;
  const BSliceArea z = bslice_area(ws, a_tiles, b_tiles);
  ProfScope ps(kPhSplitAux, s);
  k_bslice_rows<<<dim3((unsigned)act, (unsigned)(max_mt * kTileM / kSliceRows)), kSliceThreads, 0, s>>>(
      bv, geom, c_off, h, bases, k0, A, aux, z.aslices, z.ea);
  MW_LAUNCH_CHECK();
  k_bslice_cols<<<dim3((unsigned)act, (unsigned)(max_cb * 128 / kSliceRows)), kSliceThreads, 0, s>>>(
      bv, geom, c_off, h, bases, k0, A, aux, z.bslices, z.fb);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

int split_bgemm_dd(const BatchView& bv, int geom, int c_off, int h, const TileEntry* tiles, int64_t ntiles,
                   const int2* bases, int64_t a_tiles, int64_t b_tiles, int k0, double* A, const double* aux,
                   char* ws, size_t ws_bytes, DeviceStatus* status, cudaStream_t s) {
  if (ntiles <= 0) return MW_OK;
  if (split_batched_workspace_bytes(a_tiles, b_tiles) > ws_bytes) return MW_EUNSUPPORTED;
  const BSliceArea z = bslice_area(ws, a_tiles, b_tiles);
  ProfScope ps(geom == kGeomTrsmInv ? kPhTrsm : (geom == kGeomPanelInner ? kPhPanelInner : kPhGemmSplit), s);
  const size_t shmem = split_smem_bytes();
  MW_CUDA_CHECK(ensure_smem_limit(k_bsplit_gemm, shmem));
  k_bsplit_gemm<<<(unsigned)ntiles, kSplitThreads, shmem, s>>>(bv, geom, c_off, h, tiles, bases, k0, A, aux,
                                                              z.aslices, z.bslices, z.ea, z.fb, status);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

int split_bupdate_dd(const BatchView& bv, int geom, int c_off, int h, int act, int max_mt, int max_cb,
                     const TileEntry* tiles, int64_t ntiles, const int2* bases, int64_t a_tiles, int64_t b_tiles,
                     int k0, double* A, const double* aux, char* ws, size_t ws_bytes, DeviceStatus* status,
                     cudaStream_t s) {
  if (act <= 0 || ntiles <= 0) return MW_OK;
  int rc = split_bslice_dd(bv, geom, c_off, h, act, max_mt, max_cb, bases, a_tiles, b_tiles, k0, A, aux, ws,
                           ws_bytes, s);
  if (rc) return rc;
  return split_bgemm_dd(bv, geom, c_off, h, tiles, ntiles, bases, a_tiles, b_tiles, k0, A, aux, ws, ws_bytes,
                        status, s);
}

int split_binv_l11(const BatchView& bv, int act, int k0, const double* A, double* aux, cudaStream_t s) {
  if (act <= 0) return MW_OK;
  const size_t shmem = sizeof(double) * 2 * kK * kK;
  MW_CUDA_CHECK(ensure_smem_limit(k_binv_l11, shmem));
  ProfScope ps(kPhTrsm, s);
  k_binv_l11<<<(unsigned)act, 256, shmem, s>>>(bv, k0, A, aux);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

int split_update_dd(double* A, int64_t lda, int64_t plane, int64_t row0, int64_t m, int64_t col0,
                    int64_t N, int64_t k0, int nb, char* ws, size_t ws_bytes, cudaStream_t s) {
  if (nb != kK) return MW_EUNSUPPORTED;
  return split_gemm_sub_dd(m, N, A + col0 * lda + row0, lda, plane, A + k0 * lda + row0, lda, plane,
                           A + col0 * lda + k0, lda, plane, ws, ws_bytes, s);
}

}  // namespace mw
