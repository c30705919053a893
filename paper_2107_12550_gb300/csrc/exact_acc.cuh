// exact_acc.cuh -- exact fixed-point accumulation of binary64 words and
// products of words in shared memory, with greedy round-to-nearest read-back
// (see residual.cu for the description).
#pragma once
#include <cstdint>

namespace mw {

constexpr int kNL = 141;             // digits
constexpr int kLow = -2208;          // weight exponent of digit 0
constexpr int kRowsPerCta = 32;      // residual rows per CTA (lane = row)
constexpr int kResThreads = 256;
constexpr int kRelMinExp = -1074 - kLow;   // lowest result bit (subnormal grid), relative

typedef unsigned long long u64;

struct Dec {
  u64 m;      // integer significand (<= 53 bits)
  int e;      // exponent: value = m * 2^e
  bool neg;
};

__device__ __forceinline__ Dec decompose(double v) {
  const u64 bits = (u64)__double_as_longlong(v);
  Dec d;
  d.neg = (bits >> 63) != 0;
  const int ex = (int)((bits >> 52) & 0x7ff);
  const u64 man = bits & ((1ull << 52) - 1);
  if (ex == 0) {
    d.m = man;
    d.e = -1074;
  } else {
    d.m = man | (1ull << 52);
    d.e = ex - 1075;
  }
  return d;
}

// add (neg ? -1 : 1) * (hi:lo) * 2^e, (hi:lo) < 2^106
__device__ __forceinline__ void deposit128(u64* acc, u64 hi, u64 lo, int e, bool neg) {
  const int off = e - kLow;
  const int slot = off >> 5, sh = off & 31;
  const u64 w0 = lo << sh;
  const u64 w1 = sh ? ((hi << sh) | (lo >> (64 - sh))) : hi;
  const u64 w2 = sh ? (hi >> (64 - sh)) : 0ull;
  const u64 d[5] = {w0 & 0xffffffffull, w0 >> 32, w1 & 0xffffffffull, w1 >> 32, w2};
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    if (d[q]) atomicAdd(acc + slot + q, neg ? (0ull - d[q]) : d[q]);
  }
}

// +-0 tested on the bit pattern: a floating-point comparison would issue on
// the FP64 pipe, which runs at 2 lanes per clock per SM on this part
__device__ __forceinline__ bool zero_bits(double v) { return ((u64)__double_as_longlong(v) << 1) == 0ull; }

__device__ __forceinline__ void deposit_double(u64* acc, double v, int extra_exp, bool negate) {
  if (zero_bits(v)) return;
  const Dec d = decompose(v);
  deposit128(acc, 0ull, d.m, d.e + extra_exp, d.neg != negate);
}

__device__ __forceinline__ void deposit_product(u64* acc, double a, double b, int extra_exp, bool negate) {
  if (zero_bits(a) || zero_bits(b)) return;
  const Dec da = decompose(a), db = decompose(b);
  // the 106-bit product of the two 53-bit significands from 32 x 32-bit
  // products (integer multiply-adds only)
  const uint32_t al = (uint32_t)da.m, ah = (uint32_t)(da.m >> 32);
  const uint32_t bl = (uint32_t)db.m, bh = (uint32_t)(db.m >> 32);
  const u64 ll = (u64)al * bl;
  const u64 mid = (u64)al * bh + (u64)ah * bl;      // < 2^54
  const u64 hh = (u64)ah * bh;                       // < 2^42
  const u64 lo = ll + (mid << 32);
  const u64 hi = hh + (mid >> 32) + (lo < ll ? 1ull : 0ull);
  deposit128(acc, hi, lo, da.e + db.e + extra_exp, (da.neg != db.neg) != negate);
}

// ---- single-thread read-back on one accumulator -------------------------
__device__ __forceinline__ void acc_normalise(u64* s) {
  for (int k = 0; k < kNL - 1; ++k) {
    const long long v = (long long)s[k];
    const long long carry = v >> 32;  // floor
    s[k] = (u64)(v - carry * 4294967296ll);
    s[k + 1] = (u64)((long long)s[k + 1] + carry);
  }
}

__device__ __forceinline__ void acc_negate(u64* s) {
  for (int k = 0; k < kNL; ++k) s[k] = 0ull - s[k];
  acc_normalise(s);
}

__device__ __forceinline__ int acc_bit(const u64* s, int rel) {
  if (rel < 0) return 0;
  return (int)((s[rel >> 5] >> (rel & 31)) & 1ull);
}

__device__ __forceinline__ bool acc_any_below(const u64* s, int rel) {
  if (rel <= 0) return false;
  const int full = rel >> 5;
  for (int k = 0; k < full; ++k)
    if (s[k]) return true;
  const int part = rel & 31;
  if (part && (s[full] & ((1ull << part) - 1))) return true;
  return false;
}

// s holds a normalised non-negative value: return RN(value) and subtract it.
__device__ __forceinline__ double acc_take_magnitude(u64* s) {
  int top = -1;
  for (int k = kNL - 1; k >= 0; --k)
    if (s[k]) {
      top = k;
      break;
    }
  if (top < 0) return 0.0;
  const int hb = 63 - __clzll((long long)s[top]);
  const int B = 32 * top + hb;                     // relative index of the leading bit
  int lsb = B - 52;
  if (lsb < kRelMinExp) lsb = kRelMinExp;
  u64 q = 0;
  for (int r = B; r >= lsb; --r) q = (q << 1) | (u64)acc_bit(s, r);
  if (acc_bit(s, lsb - 1) && (acc_any_below(s, lsb - 1) || (q & 1ull))) q += 1;
  // subtract q * 2^lsb (q <= 2^53)
  {
    const int slot = lsb >> 5, sh = lsb & 31;
    const u64 w0 = q << sh;
    const u64 w1 = sh ? (q >> (64 - sh)) : 0ull;
    const u64 d[3] = {w0 & 0xffffffffull, w0 >> 32, w1};
    for (int t = 0; t < 3; ++t)
      if (d[t] && slot + t < kNL) s[slot + t] -= d[t];
  }
  acc_normalise(s);
  // build the double q * 2^(lsb + kLow)
  int e = lsb + kLow;
  if (q == (1ull << 53)) {
    q >>= 1;
    e += 1;
  }
  if (q == 0) return 0.0;
  if (q >= (1ull << 52)) {
    const int biased = e + 52 + 1023;
    if (biased >= 2047) return __longlong_as_double(0x7ff0000000000000ll);
    return __longlong_as_double((long long)(((u64)biased << 52) | (q - (1ull << 52))));
  }
  return __longlong_as_double((long long)q);       // subnormal: e == -1074
}

// signed greedy round-to-nearest: returns RN(S) and leaves S - RN(S)
__device__ __forceinline__ double acc_take(u64* s) {
  acc_normalise(s);
  const bool neg = ((long long)s[kNL - 1]) < 0;
  if (neg) acc_negate(s);
  double c = acc_take_magnitude(s);
  if (neg) {
    acc_negate(s);
    c = -c;
  }
  return c;
}


// exact power-of-two scaling for |e| <= 2100: x * 2^e with one rounding at most
__device__ __forceinline__ double scale2(double x, int e) {
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

__device__ __forceinline__ int ilogb_pos(double v) {  // v > 0, finite
  const u64 bits = (u64)__double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7ff);
  if (ex) return ex - 1023;
  const u64 man = bits & ((1ull << 52) - 1);
  return -1074 + (63 - __clzll((long long)man));
}


}  // namespace mw
