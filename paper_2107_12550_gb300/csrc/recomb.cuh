// recomb.cuh -- the exact form of the split update's epilogue: the slab
// product recombined from its 15 diagonal sums, C added or subtracted
// exactly, and the result rounded greedily to a DD pair, all in 32-bit
// integer limbs (the FP64 pipe issues 2 lanes per clock per SM on this part,
// the integer pipes 64).
//
// Numbers are 160-bit two's complement integers in five 32-bit limbs; a
// value v stands for v 2^s with s = e_i + f_j - 128 the slab product's grid.
//   diag_sum:  R = sum_k D_k 2^(8 (14 - k)) from the 15 diagonal sums D_k
//              (|D_k| < 2^24, so |R| < 2^137);
//   add_word:  T += w 2^-s for a double w that is an integer multiple of
//              2^s with |w| < 2^(s + 158); false (T unchanged) otherwise;
//   round_dd:  hi = RN(T 2^s), lo = RN(T 2^s - hi), each with the sign
//              flipped on request; false when hi or lo would not be a
//              normal double or zero.
// The carry chains are inline PTX (add.cc / addc) inside one asm statement
// each, so the carry flag never has to survive between statements.
#pragma once
#include <cstdint>

namespace mw {
namespace rc {

struct I160 {
  uint32_t l0, l1, l2, l3, l4;   // l0 least significant
};

__device__ __forceinline__ uint32_t lo32(long long v) { return (uint32_t)(unsigned long long)v; }
__device__ __forceinline__ uint32_t hi32(long long v) { return (uint32_t)((unsigned long long)v >> 32); }
__device__ __forceinline__ uint32_t sx32(long long v) { return (uint32_t)(v >> 63); }   // 0 or all ones

// R from the diagonal sums in four int64 groups of (up to) four diagonals,
// each |G| < 2^49, at limb offsets 0..3
__device__ __forceinline__ I160 diag_sum(const int (&D)[15]) {
  const long long G0 = (long long)D[14] + (long long)D[13] * 256 + (long long)D[12] * 65536 +
                       (long long)D[11] * 16777216;
  const long long G1 = (long long)D[10] + (long long)D[9] * 256 + (long long)D[8] * 65536 +
                       (long long)D[7] * 16777216;
  const long long G2 = (long long)D[6] + (long long)D[5] * 256 + (long long)D[4] * 65536 +
                       (long long)D[3] * 16777216;
  const long long G3 = (long long)D[2] + (long long)D[1] * 256 + (long long)D[0] * 65536;
  I160 r;
  r.l0 = lo32(G0);
  r.l1 = hi32(G0);
  r.l2 = r.l3 = r.l4 = sx32(G0);
  asm("add.cc.u32 %0, %0, %4;\n\t"
      "addc.cc.u32 %1, %1, %5;\n\t"
      "addc.cc.u32 %2, %2, %6;\n\t"
      "addc.u32 %3, %3, %6;"
      : "+r"(r.l1), "+r"(r.l2), "+r"(r.l3), "+r"(r.l4)
      : "r"(lo32(G1)), "r"(hi32(G1)), "r"(sx32(G1)));
  asm("add.cc.u32 %0, %0, %3;\n\t"
      "addc.cc.u32 %1, %1, %4;\n\t"
      "addc.u32 %2, %2, %5;"
      : "+r"(r.l2), "+r"(r.l3), "+r"(r.l4)
      : "r"(lo32(G2)), "r"(hi32(G2)), "r"(sx32(G2)));
  asm("add.cc.u32 %0, %0, %2;\n\t"
      "addc.u32 %1, %1, %3;"
      : "+r"(r.l3), "+r"(r.l4)
      : "r"(lo32(G3)), "r"(hi32(G3)));
  return r;
}

// T += w 2^-s when w is exactly representable on the grid 2^s within the
// 160-bit range (see the file comment); false (T unchanged) otherwise
__device__ __forceinline__ bool add_word(I160& T, double w, int s) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(w);
  const uint32_t hw = (uint32_t)(bits >> 32);
  const int ex = (int)((hw >> 20) & 0x7ff);
  uint32_t mhi = (hw & 0xfffffu) | (ex ? 0x100000u : 0u);
  uint32_t mlo = (uint32_t)bits;
  if ((mhi | mlo) == 0u) return true;           // +-0 adds nothing
  if (ex == 0x7ff) return false;                // Inf or NaN
  int k = (ex ? ex : 1) - 1075 - s;             // w = m 2^(k + s)
  if (k < 0) {                                  // the low -k bits of m must be zero
    if (k < -63) return false;
    const unsigned long long m = ((unsigned long long)mhi << 32) | mlo;
    if (m & ((1ull << -k) - 1ull)) return false;
    const unsigned long long q = m >> -k;
    mhi = (uint32_t)(q >> 32);
    mlo = (uint32_t)q;
    k = 0;
  }
  if (k > 105) return false;                    // |w| >= 2^(s + 158)
  const int j = k >> 5, b = k & 31;
  const uint32_t t0 = mlo << b;
  const uint32_t t1 = __funnelshift_l(mlo, mhi, b);
  const uint32_t t2 = __funnelshift_l(mhi, 0u, b);   // zero when j == 3 (b <= 9, mhi < 2^21)
  const uint32_t p0 = (j == 0) ? t0 : 0u;
  const uint32_t p1 = (j == 1) ? t0 : ((j == 0) ? t1 : 0u);
  const uint32_t p2 = (j == 2) ? t0 : ((j == 1) ? t1 : ((j == 0) ? t2 : 0u));
  const uint32_t p3 = (j == 3) ? t0 : ((j == 2) ? t1 : ((j == 1) ? t2 : 0u));
  const uint32_t p4 = (j == 3) ? t1 : ((j == 2) ? t2 : 0u);
  // w < 0: T + ~p + 1 = T - p; the first instruction sets the carry to the
  // sign (msk + msk carries out exactly when msk is all ones)
  const uint32_t msk = (uint32_t)((int)hw >> 31);
  asm("{\n\t.reg .u32 t;\n\t"
      "add.cc.u32 t, %5, %5;\n\t"
      "addc.cc.u32 %0, %0, %6;\n\t"
      "addc.cc.u32 %1, %1, %7;\n\t"
      "addc.cc.u32 %2, %2, %8;\n\t"
      "addc.cc.u32 %3, %3, %9;\n\t"
      "addc.u32 %4, %4, %10;\n\t}"
      : "+r"(T.l0), "+r"(T.l1), "+r"(T.l2), "+r"(T.l3), "+r"(T.l4)
      : "r"(msk), "r"(p0 ^ msk), "r"(p1 ^ msk), "r"(p2 ^ msk), "r"(p3 ^ msk), "r"(p4 ^ msk));
  return true;
}

// a double from a 53-bit significand (implicit bit included, possibly
// 2^53 after rounding: the carry then moves into the exponent field), the
// biased exponent of its leading bit and a sign bit (bit 31)
__device__ __forceinline__ double assemble(uint32_t mhi, uint32_t mlo, int ebias, uint32_t sign) {
  return __hiloint2double((int)((((uint32_t)(ebias - 1)) << 20) + mhi) | (int)sign, (int)mlo);
}

// RN of a normalised 64-bit window (top bit set at bit 63 of h:l) to 53
// bits with the bits below it folded into `sticky`; returns the rounded
// significand in (mhi, mlo) and whether the rounding went up
__device__ __forceinline__ uint32_t rn53(uint32_t h, uint32_t l, uint32_t sticky, uint32_t& mhi, uint32_t& mlo) {
  mlo = __funnelshift_r(l, h, 11);
  mhi = h >> 11;
  const uint32_t guard = (l >> 10) & 1u;
  const uint32_t rest = (l & 0x3ffu) | sticky;
  const uint32_t inc = guard & ((rest != 0u) | (mlo & 1u));
  asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+r"(mlo), "+r"(mhi) : "r"(inc));
  return inc;
}

// greedy rounding of (flip ? -T : T) 2^s to (hi, lo): hi = RN of the value,
// lo = RN of the remainder, +0 for a zero value or remainder; false when hi
// or lo is not a normal double or zero (the caller then takes the other form)
__device__ __forceinline__ bool round_dd(const I160& T, int s, bool flip, double& hi, double& lo) {
  // |T|: ones' complement, then + 1 when negative
  const uint32_t sg = (uint32_t)((int)T.l4 >> 31);
  uint32_t a0 = T.l0 ^ sg, a1 = T.l1 ^ sg, a2 = T.l2 ^ sg, a3 = T.l3 ^ sg, a4 = T.l4 ^ sg;
  asm("{\n\t.reg .u32 t;\n\t"
      "add.cc.u32 t, %5, %5;\n\t"
      "addc.cc.u32 %0, %0, 0;\n\t"
      "addc.cc.u32 %1, %1, 0;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.cc.u32 %3, %3, 0;\n\t"
      "addc.u32 %4, %4, 0;\n\t}"
      : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3), "+r"(a4)
      : "r"(sg));
  const uint32_t sign = (sg ^ (flip ? 0xffffffffu : 0u)) & 0x80000000u;
  const int lz = a4 ? __clz(a4)
                    : (a3 ? 32 + __clz(a3) : (a2 ? 64 + __clz(a2) : (a1 ? 96 + __clz(a1) : 128 + __clz(a0))));
  if (lz == 160) {
    hi = lo = 0.0;
    return true;
  }
  // normalise: N = |T| 2^lz has its top bit at bit 159
  uint32_t n0 = a0, n1 = a1, n2 = a2, n3 = a3, n4 = a4;
  if (lz & 128) {
    n4 = n0;
    n3 = n2 = n1 = n0 = 0u;
  }
  if (lz & 64) {
    n4 = n2;
    n3 = n1;
    n2 = n0;
    n1 = n0 = 0u;
  }
  if (lz & 32) {
    n4 = n3;
    n3 = n2;
    n2 = n1;
    n1 = n0;
    n0 = 0u;
  }
  const int b = lz & 31;
  n4 = __funnelshift_l(n3, n4, b);
  n3 = __funnelshift_l(n2, n3, b);
  n2 = __funnelshift_l(n1, n2, b);
  n1 = __funnelshift_l(n0, n1, b);
  n0 <<= b;
  // hi: the top 53 bits of N, rounded; N's bit 159 weighs 2^(159 - lz + s)
  uint32_t mhi, mlo;
  const uint32_t inc = rn53(n4, n3, n2 | n1 | n0, mhi, mlo);
  const int ehi = 159 - lz + s + 1023;
  if (ehi < 1 || ehi + (int)(mhi >> 21) > 2046) return false;
  hi = assemble(mhi, mlo, ehi, sign);
  // remainder r = (low 107 bits of N) - inc 2^107, |r| <= 2^106, in N's frame
  const int r3 = (int)(n3 & 0x7ffu) - (int)(inc << 11);
  const uint32_t rsg = (uint32_t)(r3 >> 31);
  uint32_t q0 = n0 ^ rsg, q1 = n1 ^ rsg, q2 = n2 ^ rsg, q3 = (uint32_t)r3 ^ rsg;
  asm("{\n\t.reg .u32 t;\n\t"
      "add.cc.u32 t, %4, %4;\n\t"
      "addc.cc.u32 %0, %0, 0;\n\t"
      "addc.cc.u32 %1, %1, 0;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.u32 %3, %3, 0;\n\t}"
      : "+r"(q0), "+r"(q1), "+r"(q2), "+r"(q3)
      : "r"(rsg));
  const int lz2 = q3 ? __clz(q3) : (q2 ? 32 + __clz(q2) : (q1 ? 64 + __clz(q1) : 96 + __clz(q0)));
  if (lz2 == 128) {
    lo = 0.0;
    return true;
  }
  if (lz2 & 64) {
    q3 = q1;
    q2 = q0;
    q1 = q0 = 0u;
  }
  if (lz2 & 32) {
    q3 = q2;
    q2 = q1;
    q1 = q0;
    q0 = 0u;
  }
  const int b2 = lz2 & 31;
  q3 = __funnelshift_l(q2, q3, b2);
  q2 = __funnelshift_l(q1, q2, b2);
  q1 = __funnelshift_l(q0, q1, b2);
  q0 <<= b2;
  uint32_t lhi, llo;
  rn53(q3, q2, q1 | q0, lhi, llo);
  const int elo = 127 - lz2 - lz + s + 1023;
  if (elo < 1 || elo + (int)(lhi >> 21) > 2046) return false;
  lo = assemble(lhi, llo, elo, sign ^ (rsg & 0x80000000u));
  return true;
}

}  // namespace rc
}  // namespace mw
