// mw_arith.cuh -- multiword (DD/TD/QD) arithmetic as device inlines.
//
// A value of precision W (2 = double-double, 3 = triple-double, 4 =
// quad-double; Section 1 of Kouya's paper) is W binary64 words.  Every
// floating-point step below is an explicit round-to-nearest intrinsic, so the
// compiler can neither contract a*b+c nor reassociate: the bits of each result
// are fixed by the algorithm alone.
//
// Algorithms (the paper names Bailey et al.'s QD library but prints none):
//   * error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum, and
//     TwoProd via a fused multiply-add;
//   * W = 2: Joldes, Muller and Popescu, ACM TOMS 44(2) 2017 --
//     AccurateDWPlusDW (Alg. 6), DWTimesDW3 (Alg. 12) and a DWDivDW2-shaped
//     division (Alg. 17) whose DW-times-FP step uses the FMA;
//   * W = 3, 4: gather the exact partial results (TwoSum of matching words;
//     TwoProd of the products up to order W-2, plain products at order W-1)
//     and renormalise: a bottom-up TwoSum cascade (Ogita-Rump-Oishi VecSum),
//     a top-down extraction of W words that skips zero errors and folds the
//     tail into the last word, then a top-down FastTwoSum sweep
//     (renormalisation in the manner of Hida, Li and Bailey, ARITH 2001);
//     division is long division with W+1 quotient digits.
//
// Additions are issued as fma(a, 1, b): one rounding of a + b, hence the same
// bits as an add, and the fused pipe issues faster than the add pipe on this
// GPU's FP64 units.  TwoSum's two results are fixed by its operands, so by
// default they are computed on the integer pipes (exact integer sum of the
// aligned significands, then round to nearest-even); every operation gives
// the same bits with either form (template argument I).
#pragma once
#include <cstdint>

namespace mw {

template <int W>
struct val {
  double v[W];
};

__device__ __forceinline__ double fadd(double a, double b) { return __fma_rn(a, 1.0, b); }
__device__ __forceinline__ double fsub(double a, double b) { return __fma_rn(b, -1.0, a); }
__device__ __forceinline__ double fmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ffma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double fdiv(double a, double b) { return __ddiv_rn(a, b); }

// Knuth's TwoSum as six FP64 operations: s = RN(a + b), e = a + b - s
// exactly (for finite a, b without overflow)
__device__ __forceinline__ void two_sum_fp64(double a, double b, double& s, double& e) {
  s = fadd(a, b);
  const double a_virt = fsub(s, b);
  const double b_virt = fsub(s, a_virt);
  const double a_err = fsub(a, a_virt);
  const double b_err = fsub(b, b_virt);
  e = fadd(a_err, b_err);
}

namespace eft_int {
typedef unsigned long long u64;
constexpr u64 kMan = (1ull << 52) - 1;
constexpr u64 kHid = 1ull << 52;
constexpr u64 kSign = 1ull << 63;
__device__ __forceinline__ u64 bits(double x) { return (u64)__double_as_longlong(x); }
__device__ __forceinline__ double dbl(u64 b) { return __longlong_as_double((long long)b); }

// the double |r| 2^(E - 1075) with sign bit sg (r < 2^64, exactly
// representable); false when it would be subnormal or overflow
__device__ __forceinline__ bool pack(u64 r, int E, u64 sg, double& out) {
  const int L = 64 - __clzll((long long)r);
  const int Ee = E + (L - 53);
  if (Ee < 1 || Ee > 2046) return false;
  const u64 m = (L >= 53) ? (r >> (L - 53)) : (r << (53 - L));
  out = dbl(sg | ((u64)Ee << 52) | (m & kMan));
  return true;
}

// s = RN(a + b), e = a + b - s for the bit patterns A, B of two doubles with
// |a| >= |b|; false (and the caller falls back) outside the normal range
__device__ __forceinline__ bool sum_ordered(u64 A, u64 B, double& s, double& e) {
  const u64 ua = A & ~kSign, ub = B & ~kSign;
  const int ea = (int)(ua >> 52), eb = (int)(ub >> 52);
  if (ea == 2047) return false;              // a infinite or NaN
  if (ub == 0ull) {                          // b = +-0: s = a + b, e = +0 (both zero: -0 only if both are)
    s = dbl(ua ? A : (A & B & kSign));
    e = 0.0;
    return true;
  }
  if (eb == 0) return false;                 // b subnormal
  const int d = ea - eb;
  if (d > 54) {                              // |b| < ulp(a) / 4: RN(a + b) = a, exactly b left over
    s = dbl(A);
    e = dbl(B);
    return true;
  }
  const u64 sa = A & kSign;
  const u64 ma = (ua & kMan) | kHid, mb = (ub & kMan) | kHid;
  // M = ma 2^d +- mb (< 2^108) in (hi, lo); a + b = M 2^(eb - 1075) with a's sign
  u64 lo = ma << d;
  u64 hi = d ? (ma >> (64 - d)) : 0ull;
  if ((A ^ B) & kSign) {
    const u64 l2 = lo - mb;
    hi -= (l2 > lo) ? 1ull : 0ull;
    lo = l2;
  } else {
    const u64 l2 = lo + mb;
    hi += (l2 < lo) ? 1ull : 0ull;
    lo = l2;
  }
  if ((hi | lo) == 0ull) {                   // a = -b: +0, +0
    s = 0.0;
    e = 0.0;
    return true;
  }
  const int L = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
  if (L <= 53) {                             // the sum is exact: e = +0
    e = 0.0;
    return pack(lo, eb, sa, s);
  }
  const int sh = L - 53;                     // 1 .. 55 bits below s's last place
  u64 q = (lo >> sh) | (hi << (64 - sh));
  const u64 r = lo & ((1ull << sh) - 1ull);
  const u64 half = 1ull << (sh - 1);
  const bool up = (r > half) || (r == half && (q & 1ull));   // to nearest, ties to even
  int Es = eb + sh;
  const long long rem = (long long)r - (up ? (long long)(1ull << sh) : 0ll);
  if (up && ++q == (1ull << 53)) {
    q >>= 1;
    Es += 1;
  }
  if (Es > 2046) return false;
  s = dbl(sa | ((u64)Es << 52) | (q & kMan));
  if (rem == 0) {
    e = 0.0;
    return true;
  }
  return pack((u64)(rem < 0 ? -rem : rem), eb, rem < 0 ? (sa ^ kSign) : sa, e);
}
}  // namespace eft_int

// TwoSum: s = RN(a + b) and e = a + b - s exactly (Knuth).  Both values are
// fixed by a and b alone, so they are computed here on the integer pipes,
// which run at 32 times the FP64 pipe's lane rate on this GPU: the two
// significands are aligned into a 128-bit integer and added exactly, the sum
// is rounded to nearest-even, and the remainder is e.  Operands or results
// outside the normal range (zeros, subnormals, infinities, NaNs, overflow)
// take the six-operation FP64 sequence, which gives the same values wherever
// both apply; either way the bits are those of the FP64 sequence.
// I = false: Knuth's FP64 sequence itself.  The integer form costs more
// issue slots and a longer dependency chain but 6 fewer FP64 instructions:
// it wins where many warps share the FP64 pipe (throughput loops) and loses
// on a lone serial chain, so the multiword operations below take I as a
// template argument (default: the integer form).
template <bool I = true>
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  if constexpr (!I) {
    two_sum_fp64(a, b, s, e);
    return;
  }
  eft_int::u64 A = eft_int::bits(a), B = eft_int::bits(b);
  if ((A << 1) < (B << 1)) {
    const eft_int::u64 t = A;
    A = B;
    B = t;
  }
  if (!eft_int::sum_ordered(A, B, s, e)) two_sum_fp64(a, b, s, e);
}

// x != 0 (either sign) tested on the bit pattern, off the FP64 pipe
__device__ __forceinline__ bool nonzero(double x) {
  return (((unsigned long long)__double_as_longlong(x)) << 1) != 0ull;
}

// exact when exponent(a) >= exponent(b)
__device__ __forceinline__ void quick_two_sum(double a, double b, double& s, double& e) {
  s = fadd(a, b);
  const double t = fsub(s, a);
  e = fsub(b, t);
}

__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  p = fmul(a, b);
  e = ffma(a, b, -p);
}

// ---------------------------------------------------------------------------
// W = 2
// ---------------------------------------------------------------------------
template <bool I = true>
__device__ __forceinline__ val<2> dd_add(const val<2>& x, const val<2>& y) {
  double sh, sl, th, tl, vh, vl;
  two_sum<I>(x.v[0], y.v[0], sh, sl);
  two_sum<I>(x.v[1], y.v[1], th, tl);
  const double c = fadd(sl, th);
  quick_two_sum(sh, c, vh, vl);
  const double w = fadd(tl, vl);
  val<2> z;
  quick_two_sum(vh, w, z.v[0], z.v[1]);
  return z;
}

__device__ __forceinline__ val<2> dd_mul(const val<2>& x, const val<2>& y) {
  double ch, cl1;
  two_prod(x.v[0], y.v[0], ch, cl1);
  const double tl0 = fmul(x.v[1], y.v[1]);
  const double tl1 = ffma(x.v[0], y.v[1], tl0);
  const double cl2 = ffma(x.v[1], y.v[0], tl1);
  const double cl3 = fadd(cl1, cl2);
  val<2> z;
  quick_two_sum(ch, cl3, z.v[0], z.v[1]);
  return z;
}

__device__ __forceinline__ val<2> dd_div(const val<2>& x, const val<2>& y) {
  const double q0 = fdiv(x.v[0], y.v[0]);
  double ph, pl, rh, rl;
  two_prod(y.v[0], q0, ph, pl);
  pl = ffma(y.v[1], q0, pl);
  quick_two_sum(ph, pl, rh, rl);
  const double dh = fsub(x.v[0], rh);
  const double dl = fsub(x.v[1], rl);
  const double d = fadd(dh, dl);
  const double q1 = fdiv(d, y.v[0]);
  val<2> z;
  quick_two_sum(q0, q1, z.v[0], z.v[1]);
  return z;
}

// ---------------------------------------------------------------------------
// Renormalisation of M terms into W words (W = 3, 4)
// ---------------------------------------------------------------------------
template <int W, int M, bool I = true>
__device__ __forceinline__ val<W> renormalise(double (&t)[M]) {
  // bottom-up exact cascade
  double s = t[M - 1];
#pragma unroll
  for (int i = M - 2; i >= 0; --i) {
    double hi, lo;
    two_sum<I>(t[i], s, hi, lo);
    s = hi;
    t[i + 1] = lo;
  }
  t[0] = s;
  // top-down extraction; k = number of words emitted so far
  val<W> z;
#pragma unroll
  for (int j = 0; j < W; ++j) z.v[j] = 0.0;
  int k = 0;
  s = t[0];
#pragma unroll
  for (int i = 1; i < M; ++i) {
    if (k < W - 1) {
      double hi, lo;
      two_sum<I>(s, t[i], hi, lo);
      if (nonzero(lo)) {
#pragma unroll
        for (int j = 0; j < W - 1; ++j) z.v[j] = (k == j) ? hi : z.v[j];
        k += 1;
        s = lo;
      } else {
        s = hi;
      }
    } else {
      s = fadd(s, t[i]);
    }
  }
#pragma unroll
  for (int j = 0; j < W; ++j) z.v[j] = (k == j) ? s : z.v[j];
  // top-down sweep
#pragma unroll
  for (int j = 0; j < W - 1; ++j) {
    double hi, lo;
    quick_two_sum(z.v[j], z.v[j + 1], hi, lo);
    z.v[j] = hi;
    z.v[j + 1] = lo;
  }
  return z;
}

template <int W, bool I = true>
__device__ __forceinline__ val<W> gen_add(const val<W>& x, const val<W>& y) {
  double s[W], e[W];
#pragma unroll
  for (int i = 0; i < W; ++i) two_sum<I>(x.v[i], y.v[i], s[i], e[i]);
  double t[2 * W - 1];
  t[0] = s[0];
#pragma unroll
  for (int i = 1; i < W; ++i) {
    t[2 * i - 1] = s[i];
    t[2 * i] = e[i - 1];
  }
  return renormalise<W, 2 * W - 1, I>(t);
}

template <bool I = true>
__device__ __forceinline__ val<3> td_mul(const val<3>& x, const val<3>& y) {
  double p00, q00, p01, q01, p10, q10;
  two_prod(x.v[0], y.v[0], p00, q00);
  two_prod(x.v[0], y.v[1], p01, q01);
  two_prod(x.v[1], y.v[0], p10, q10);
  double c = fmul(x.v[1], y.v[1]);
  c = ffma(x.v[0], y.v[2], c);
  c = ffma(x.v[2], y.v[0], c);
  c = fadd(c, q01);
  c = fadd(c, q10);
  double t[5] = {p00, q00, p01, p10, c};
  return renormalise<3, 5, I>(t);
}

template <bool I = true>
__device__ __forceinline__ val<4> qd_mul(const val<4>& x, const val<4>& y) {
  double p00, q00, p01, q01, p10, q10, p02, q02, p11, q11, p20, q20;
  two_prod(x.v[0], y.v[0], p00, q00);
  two_prod(x.v[0], y.v[1], p01, q01);
  two_prod(x.v[1], y.v[0], p10, q10);
  two_prod(x.v[0], y.v[2], p02, q02);
  two_prod(x.v[1], y.v[1], p11, q11);
  two_prod(x.v[2], y.v[0], p20, q20);
  double c = fmul(x.v[1], y.v[2]);
  c = ffma(x.v[2], y.v[1], c);
  c = ffma(x.v[0], y.v[3], c);
  c = ffma(x.v[3], y.v[0], c);
  c = fadd(c, q02);
  c = fadd(c, q11);
  c = fadd(c, q20);
  double t[10] = {p00, q00, p01, p10, q01, q10, p02, p11, p20, c};
  return renormalise<4, 10, I>(t);
}

template <int W, bool I = true>
__device__ __forceinline__ val<W> gen_mul_d(const val<W>& x, double d) {
  double p[W], q[W];
#pragma unroll
  for (int i = 0; i < W - 1; ++i) two_prod(x.v[i], d, p[i], q[i]);
  p[W - 1] = fmul(x.v[W - 1], d);
  double t[2 * W - 1];
  t[0] = p[0];
#pragma unroll
  for (int i = 1; i < W; ++i) {
    t[2 * i - 1] = p[i];
    t[2 * i] = q[i - 1];
  }
  return renormalise<W, 2 * W - 1, I>(t);
}

template <int W>
__device__ __forceinline__ val<W> neg(const val<W>& x) {
  val<W> z;
#pragma unroll
  for (int i = 0; i < W; ++i) z.v[i] = -x.v[i];
  return z;
}

template <int W, bool I = true>
__device__ __forceinline__ val<W> gen_div(const val<W>& x, const val<W>& y) {
  double q[W + 1];
  q[0] = fdiv(x.v[0], y.v[0]);
  val<W> r = x;
#pragma unroll
  for (int i = 1; i <= W; ++i) {
    r = gen_add<W, I>(r, neg<W>(gen_mul_d<W, I>(y, q[i - 1])));
    q[i] = fdiv(r.v[0], y.v[0]);
  }
  return renormalise<W, W + 1, I>(q);
}

// ---------------------------------------------------------------------------
// Precision-generic entry points
// ---------------------------------------------------------------------------
template <int W, bool I = true>
__device__ __forceinline__ val<W> add(const val<W>& x, const val<W>& y) {
  if constexpr (W == 2) return dd_add<I>(x, y);
  else return gen_add<W, I>(x, y);
}

template <int W, bool I = true>
__device__ __forceinline__ val<W> sub(const val<W>& x, const val<W>& y) { return add<W, I>(x, neg<W>(y)); }

template <int W, bool I = true>
__device__ __forceinline__ val<W> mul(const val<W>& x, const val<W>& y) {
  if constexpr (W == 2) return dd_mul(x, y);
  else if constexpr (W == 3) return td_mul<I>(x, y);
  else return qd_mul<I>(x, y);
}

template <int W, bool I = true>
__device__ __forceinline__ val<W> div(const val<W>& x, const val<W>& y) {
  if constexpr (W == 2) return dd_div(x, y);
  else return gen_div<W, I>(x, y);
}

// c - a*b as a rounded multiply followed by a rounded subtraction (the
// per-element step of the elimination and of the substitutions)
template <int W, bool I = true>
__device__ __forceinline__ val<W> msub(const val<W>& c, const val<W>& a, const val<W>& b) {
  return sub<W, I>(c, mul<W, I>(a, b));
}

// |x| vs |y| on the sign-adjusted words (|x0|, s x1, s x2, ...): -1, 0, +1,
// with s = -1 where x0 < 0.  Decided on the bit patterns with integer
// operations (the FP64 pipe is slow here and this sits on the pivot search's
// critical path), with the floating-point comparison's outcome in every case:
// a key that orders non-NaN doubles by value (+0 and -0 equal), negated for
// the sign adjustment; a word pair with a NaN is unordered and skipped.
__device__ __forceinline__ bool bits_nan(unsigned long long u) {
  return (u & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
}
__device__ __forceinline__ long long order_key(unsigned long long u) {
  const long long mag = (long long)(u & 0x7fffffffffffffffull);
  return (u >> 63) ? -mag : mag;
}
template <int W>
__device__ __forceinline__ int cmp_abs(const val<W>& x, const val<W>& y) {
  const unsigned long long x0 = (unsigned long long)__double_as_longlong(x.v[0]);
  const unsigned long long y0 = (unsigned long long)__double_as_longlong(y.v[0]);
  // x0 < 0: sign set, not a zero, not a NaN
  const bool nx = (x0 >> 63) && (x0 << 1) != 0ull && !bits_nan(x0);
  const bool ny = (y0 >> 63) && (y0 << 1) != 0ull && !bits_nan(y0);
#pragma unroll
  for (int c = 0; c < W; ++c) {
    const unsigned long long ux = (unsigned long long)__double_as_longlong(x.v[c]);
    const unsigned long long uy = (unsigned long long)__double_as_longlong(y.v[c]);
    if (bits_nan(ux) || bits_nan(uy)) continue;
    const long long a = nx ? -order_key(ux) : order_key(ux);
    const long long b = ny ? -order_key(uy) : order_key(uy);
    if (a > b) return 1;
    if (a < b) return -1;
  }
  return 0;
}

template <int W>
__device__ __forceinline__ bool is_zero(const val<W>& x) {
  bool z = true;
#pragma unroll
  for (int c = 0; c < W; ++c) z = z && !nonzero(x.v[c]);
  return z;
}

// planar loads/stores: word c at p[c * plane + idx]
template <int W>
__device__ __forceinline__ val<W> load(const double* p, int64_t plane, int64_t idx) {
  val<W> z;
#pragma unroll
  for (int c = 0; c < W; ++c) z.v[c] = p[c * plane + idx];
  return z;
}
template <int W>
__device__ __forceinline__ val<W> load_cg(const double* p, int64_t plane, int64_t idx) {
  val<W> z;
#pragma unroll
  for (int c = 0; c < W; ++c) z.v[c] = __ldcg(p + c * plane + idx);
  return z;
}
template <int W>
__device__ __forceinline__ val<W> load_ro(const double* __restrict__ p, int64_t plane, int64_t idx) {
  val<W> z;
#pragma unroll
  for (int c = 0; c < W; ++c) z.v[c] = __ldg(p + c * plane + idx);
  return z;
}
template <int W>
__device__ __forceinline__ void store(double* p, int64_t plane, int64_t idx, const val<W>& x) {
#pragma unroll
  for (int c = 0; c < W; ++c) p[c * plane + idx] = x.v[c];
}
template <int W>
__device__ __forceinline__ void store_cg(double* p, int64_t plane, int64_t idx, const val<W>& x) {
#pragma unroll
  for (int c = 0; c < W; ++c) __stcg(p + c * plane + idx, x.v[c]);
}

}  // namespace mw
