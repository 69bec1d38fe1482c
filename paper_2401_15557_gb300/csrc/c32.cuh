// Compensated FP32 ("double-float") arithmetic for the element blocks.
//
// A value is held as an unevaluated sum h + l of two floats.  The error-free
// transformations are the classical ones: Knuth's TwoSum (a + b = s + e
// exactly, six additions), Dekker's product with a fused multiply-add
// (a b = p + e exactly, one FMA), and Newton's iteration for the reciprocal.
// GB300 issues FP32 arithmetic at 64x its FP64 rate, so an element block in
// compensated FP32 costs a fraction of the FP64 one while keeping about 47
// bits: the trace-form entries come out within a few 1e-14 of the FP64 ones
// relative to the row scale.
//
// Everything here is __host__ __device__, spelled with explicitly rounded
// FP32 operations (no contraction) and integer operations only (the one
// reciprocal is seeded from the bits, not by a special-function unit), so a
// host build computes bitwise the same values; the CPU tests check the
// arithmetic against exact rational results.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define PH_HD __host__ __device__ __forceinline__
#else
#include <cmath>
#define PH_HD inline
#endif

namespace phfem {
namespace c32 {

#if defined(__CUDA_ARCH__)
PH_HD float fadd(float a, float b) { return __fadd_rn(a, b); }
PH_HD float fsub(float a, float b) { return __fsub_rn(a, b); }
PH_HD float fmul(float a, float b) { return __fmul_rn(a, b); }
PH_HD float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
PH_HD uint32_t fbits(float x) { return __float_as_uint(x); }
PH_HD float bfloat(uint32_t u) { return __uint_as_float(u); }
PH_HD uint32_t dhi(double x) { return (uint32_t)__double2hiint(x); }
PH_HD uint32_t dlo(double x) { return (uint32_t)__double2loint(x); }
PH_HD double bdouble(uint32_t hi, uint32_t lo) { return __hiloint2double((int)hi, (int)lo); }
#else
// host build (tests): IEEE single arithmetic, compiled without contraction
PH_HD float fadd(float a, float b) { return a + b; }
PH_HD float fsub(float a, float b) { return a - b; }
PH_HD float fmul(float a, float b) { return a * b; }
PH_HD float ffma(float a, float b, float c) { return std::fmaf(a, b, c); }
PH_HD uint32_t fbits(float x) { uint32_t u; std::memcpy(&u, &x, 4); return u; }
PH_HD float bfloat(uint32_t u) { float x; std::memcpy(&x, &u, 4); return x; }
PH_HD uint32_t dhi(double x) { uint64_t u; std::memcpy(&u, &x, 8); return (uint32_t)(u >> 32); }
PH_HD uint32_t dlo(double x) { uint64_t u; std::memcpy(&u, &x, 8); return (uint32_t)u; }
PH_HD double bdouble(uint32_t hi, uint32_t lo) {
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double x;
  std::memcpy(&x, &u, 8);
  return x;
}
#endif

struct f2 {
  float h, l;
};

// 1/x for a positive normal float x to within 2^-22, in FP32 arithmetic
// only, the same on host and device: an integer estimate from the exponent
// field (bits(1/x) ~ const - bits(x), within 1/8) and three Newton steps
// r <- r + r (1 - x r), each squaring the relative error.
PH_HD float frcp(float x) {
  float r = bfloat(0x7EF311C3u - fbits(x));
  for (int i = 0; i < 3; ++i) r = ffma(r, ffma(-x, r, 1.0f), r);
  return r;
}

PH_HD f2 neg(f2 a) { return {-a.h, -a.l}; }

// Knuth's TwoSum: s + e == a + b exactly.
PH_HD f2 two_sum(float a, float b) {
  const float s = fadd(a, b);
  const float bb = fsub(s, a);
  const float e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
  return {s, e};
}

// Dekker's product with one FMA: p + e == a b exactly.
PH_HD f2 two_prod(float a, float b) {
  const float p = fmul(a, b);
  return {p, ffma(a, b, -p)};
}

// (hi << 3) | (lo >> 29).
PH_HD uint32_t funnel_l3(uint32_t lo, uint32_t hi) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_l(lo, hi, 3);
#else
  return (hi << 3) | (lo >> 29);
#endif
}

// Splits x = 0 or 2^-40 <= |x| < 2^40 into h + l: h is x with its significand
// cut to 24 bits, l the remaining 29 bits rounded to a float, so
// |x - h - l| <= 2^-48 |x| and |l| < 2^-23 |h|.  Integer operations, and the
// float conversion of the 29 low bits m as 64 (m >> 6) + (m & 63), each part
// exact through 2^23 + k (k in the low bits of a float).
// Returns false (and nothing usable) outside that range.
PH_HD bool split(double x, f2& out) {
  const uint32_t hi = dhi(x), lo = dlo(x);
  const uint32_t E = (hi >> 20) & 0x7FFu;  // biased exponent
  if (((hi << 1) | lo) == 0) {             // +-0
    out = {0.0f, 0.0f};
    return true;
  }
  if (E - (1023u - 40u) >= 80u) return false;
  const uint32_t sign = hi & 0x80000000u;
  // t: the high word with the exponent rebiased for a float (E - 896 >= 87
  // stays within the 11-bit field, so the sign bit is untouched); shifted left
  // by 3 with the top 3 bits of lo it is h without its sign
  const uint32_t t = hi - (896u << 20);
  out.h = bfloat(sign | funnel_l3(lo, t));
  // x - h = +-m 2^(E - 1075), m the low 29 significand bits = 64 ma + mb
  const float s64 = bfloat(sign | (((t - (46u << 20)) << 3) & 0x7F800000u));  // +-2^(E - 1069)
  const float s1 = fmul(s64, 0.015625f);                                       // +-2^(E - 1075)
  const float ma = fsub(bfloat(0x4B000000u | ((lo >> 6) & 0x7FFFFFu)), 8388608.0f);
  const float mb = fsub(bfloat(0x4B000000u | (lo & 63u)), 8388608.0f);
  out.l = ffma(ma, s64, fmul(mb, s1));
  return true;
}

// Index of the highest set bit of k > 0.
PH_HD int top_bit(uint32_t k) {
#if defined(__CUDA_ARCH__)
  return 31 - __clz((int)k);
#else
  return 31 - __builtin_clz(k);
#endif
}

// The float x as a double, exactly (infinities and NaNs included), with
// 32-bit integer operations only (GB300 runs conversions involving FP64 on
// its narrow FP64 pipe).
PH_HD double widen(float x) {
  const uint32_t u = fbits(x);
  const uint32_t sign = u & 0x80000000u, E = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  if (E == 255u) return bdouble(sign | 0x7FF00000u | (m >> 3), (m & 7u) << 29);  // the payload keeps a NaN a NaN
  if (E == 0) {  // zero or subnormal: x = m 2^-149
    if (m == 0) return bdouble(sign, 0u);
    const int p = top_bit(m);       // x = 1.f 2^(p - 149), f = the p bits below the top one
    const uint32_t f = m << (23 - p) & 0x7FFFFFu;  // f left-aligned in 23 bits
    return bdouble(sign | ((uint32_t)(p + 874) << 20) | (f >> 3), (f & 7u) << 29);
  }
  return bdouble(sign | ((E + 896u) << 20) | (m >> 3), (m & 7u) << 29);
}

// The double x rounded to the nearest float (ties to even), with integer
// operations only; results below the normal floats are flushed to zero.
PH_HD float narrow(double x) {
  const uint32_t hi = dhi(x), lo = dlo(x);
  const uint32_t sign = hi & 0x80000000u, E = (hi >> 20) & 0x7FFu;
  if (E >= 1151u) {  // |x| >= 2^128: infinity, or NaN
    const bool nan = E == 2047u && ((hi & 0xFFFFFu) | lo) != 0;
    return bfloat(sign | (nan ? 0x7FC00000u : 0x7F800000u));
  }
  if (E < 897u) return bfloat(sign);  // |x| < 2^-126 (and zero)
  uint32_t f = ((E - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const uint32_t r = lo & 0x1FFFFFFFu;  // the 29 dropped bits
  f += (r > 0x10000000u || (r == 0x10000000u && (f & 1u))) ? 1u : 0u;  // a carry moves into the exponent
  return bfloat(sign | f);
}

// h + l as a double for a pair as TwoSum leaves it (|l| <= ulp(h)/2), with
// integer operations only: h's 24-bit significand at the top of a 53-bit
// one, l's significand added or subtracted in place (bits below the double's
// last place dropped), and one renormalising step when h is a power of two
// and l has the other sign.  Within 2^-52 of h + l.
PH_HD double to_double(f2 a) {
  const uint32_t uh = fbits(a.h), ul = fbits(a.l);
  const uint32_t Eh = (uh >> 23) & 0xFFu;
  if (Eh == 0) return widen(a.h);  // h zero or subnormal: l is then zero (sums there are exact)
  // the 53-bit significand as (mh, ml): the top 21 bits and the low 32 bits
  const uint32_t sh24 = (uh & 0x7FFFFFu) | 0x800000u;
  uint32_t mh = sh24 >> 3, ml = (sh24 & 7u) << 29;
  uint32_t Ed = Eh + 896u;  // the double's biased exponent
  if ((ul << 1) != 0) {
    const uint32_t El = (ul >> 23) & 0xFFu;
    const uint32_t Sl = El ? ((ul & 0x7FFFFFu) | 0x800000u) : (ul & 0x7FFFFFu);
    const int sh = (int)(El ? El : 1u) - (int)Eh + 29;  // <= 5: |l| <= 2^-24 |h|, so L < 2^29
    const uint32_t L = sh >= 0 ? (Sl << sh) : (sh > -32 ? (Sl >> -sh) : 0u);
    if ((ul ^ uh) & 0x80000000u) {
      mh -= (ml < L) ? 1u : 0u;
      ml -= L;
      if (mh < (1u << 20)) {  // below 2^52: h = 2^k and l < 0
        mh = (mh << 1) | (ml >> 31);
        ml <<= 1;
        Ed -= 1u;
      }
    } else {
      ml += L;
      mh += (ml < L) ? 1u : 0u;  // stays below 2^53
    }
  }
  return bdouble((uh & 0x80000000u) | (Ed << 20) | (mh & 0xFFFFFu), ml);
}

// a b + c d for compensated a, b, c, d with |l| < 2^-23 |h|: the two leading
// products and their sum are exact; the cross terms, the products' errors
// and the sum's error are gathered in one float.  The result is within
// about 2^-45 (|a b| + |c d|) of the exact value.
PH_HD f2 dot2(f2 a, f2 b, f2 c, f2 d) {
  const f2 p = two_prod(a.h, b.h);
  const f2 q = two_prod(c.h, d.h);
  const f2 s = two_sum(p.h, q.h);
  float t = fadd(p.l, q.l);
  t = ffma(a.h, b.l, t);
  t = ffma(a.l, b.h, t);
  t = ffma(a.l, b.l, t);
  t = ffma(c.h, d.l, t);
  t = ffma(c.l, d.h, t);
  t = ffma(c.l, d.l, t);
  return two_sum(s.h, fadd(s.l, t));
}

// a b for compensated a, b (within about 2^-46 |a b|).
PH_HD f2 mul(f2 a, f2 b) {
  const f2 p = two_prod(a.h, b.h);
  float t = ffma(a.h, b.l, p.l);
  t = ffma(a.l, b.h, t);
  t = ffma(a.l, b.l, t);
  return two_sum(p.h, t);
}

// 1 / a for compensated a > 0 given r0, a float reciprocal of a.h to 2^-22:
// with e = 1 - a r0 (|e| < 2^-22; 1 - a.h r0 is formed exactly), 1/a =
// r0 / (1 - e) = r0 (1 + e + e^2 + ...), kept to e^2; the roundings of e
// and of r0 e leave at most about 2.5 2^-46 relative.
PH_HD f2 rcp(f2 a, float r0) {
  const f2 p = two_prod(a.h, r0);  // p.h within 2^-23 of 1, so 1 - p.h is exact
  const float e = fsub(fsub(fsub(1.0f, p.h), p.l), fmul(a.l, r0));
  return two_sum(r0, fmul(r0, ffma(e, e, e)));
}

// Trace-form record of the triangle (x0, y0), (x1, y1), (x2, y2) with the
// isotropic coefficient a:  L_ij = -(a / |T|) e_i . e_j  for (ij) = (01),
// (12), (20), and |T| / 3, where e_k = P_{k+2} - P_{k+1} (so |T| grad
// lambda_k is e_k turned by a right angle, over 2, and K^CR_T = (a/|T|)
// e_i . e_j + delta |T|/3 I, L = -K^CR off the diagonal).  The edge vectors
// are FP64 differences; the rest is compensated FP32, rounded to doubles at
// the end.
//
// Returns false (outputs unspecified) when a or a nonzero edge component is
// outside [2^-40, 2^40), the triangle is not counterclockwise, the angle at
// P0 has a sine below 1/4 (2|T| = e1 x e2 is then computed with a relative
// error above 2^-42), or a result is not finite: such triangles take FP64.
PH_HD bool tri_record(double x0, double y0, double x1, double y1, double x2, double y2, double a,
                      double out64[4]) {
  f2 E0x, E0y, E1x, E1y, E2x, E2y, A;
  bool ok = split(x2 - x1, E0x);
  ok &= split(y2 - y1, E0y);
  ok &= split(x0 - x2, E1x);
  ok &= split(y0 - y2, E1y);
  ok &= split(x1 - x0, E2x);
  ok &= split(y1 - y0, E2y);
  ok &= split(a, A);
  if (!ok) return false;
  const f2 ar = dot2(E1x, E2y, neg(E1y), E2x);  // 2|T| = e1 x e2
  if (!(ar.h > 0.0f)) return false;
  const float ir = frcp(ar.h);
  // 1 / sin^2 of the angle at P0 = (|e1|^2 / 2|T|) (|e2|^2 / 2|T|)
  const float q1 = fmul(ffma(E1x.h, E1x.h, fmul(E1y.h, E1y.h)), ir);
  const float q2 = fmul(ffma(E2x.h, E2x.h, fmul(E2y.h, E2y.h)), ir);
  if (!(fmul(q1, q2) <= 16.0f)) return false;
  const f2 nc = mul(f2{-2.0f * A.h, -2.0f * A.l}, rcp(ar, ir));  // -a / |T|
  const f2 L01 = mul(nc, dot2(E0x, E1x, E0y, E1y));
  const f2 L12 = mul(nc, dot2(E1x, E2x, E1y, E2y));
  const f2 L20 = mul(nc, dot2(E2x, E0x, E2y, E0y));
  const float big = 1e37f;
  if (!(L01.h <= big && L01.h >= -big && L12.h <= big && L12.h >= -big && L20.h <= big && L20.h >= -big))
    return false;
  out64[0] = to_double(L01);
  out64[1] = to_double(L12);
  out64[2] = to_double(L20);
  out64[3] = to_double(mul(ar, f2{0.166666672f, -4.96705388e-09f}));  // 1/6 to 2^-50
  return true;
}

}  // namespace c32
}  // namespace phfem
