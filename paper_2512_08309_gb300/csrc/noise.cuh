// Seed function G of InfiniteDiffusion (App. B, "Seeds and initial noise"):
// N(seed, level, step, x, y), a standard normal in binary32 that is a pure
// function of its arguments, so that any region of any step can be drawn in
// any order (Sec. 3.5, seed consistency).
//
// Definition (bit for bit):
//   Philox4x32-10 (Salmon et al., SC'11) with key (seed lo, seed hi) and
//   counter (x mod 2^32, y mod 2^32, step, level); words o0, o1 give
//   u1 = ((o0 >> 8) + 1) 2^-24 in (0, 1] and k = o1 >> 8 (u2 = k 2^-24);
//   N = sqrt(-2 ln u1) cos(2 pi u2).
// ln and cos are evaluated by this library's own series polynomials with
// every operation an explicitly rounded binary32 intrinsic (no contraction
// into fused multiply-adds), so the value does not depend on the compiler:
//   ln u:  u = m 2^e, m in [1,2) moved to [sqrt2/2, sqrt2] when its mantissa
//          bits exceed 0x3504F3; z = (m-1)/(m+1), w = z^2,
//          p = ((((w/11 + 1/9) w + 1/7) w + 1/5) w + 1/3) w, t = 2z,
//          ln m = t + t p  (atanh series); ln u = e LN2_HI + (e LN2_LO + ln m)
//          with LN2_HI = 22713/32768 and LN2_LO = fl(ln2 - LN2_HI).
//   cos:   q = (k + 2^21) >> 22, r = (k - q 2^22) 2^-24, th = r fl(2 pi),
//          x = th^2, Taylor polynomials of cos and sin in x (coefficients
//          fl(1/n!), innermost term 1/12! and 1/11!), quadrant q mod 4 picks
//          C, -S, -C, S.
// Each coefficient fl(1/n) is a correctly rounded binary32 division.
#pragma once
#include <stdint.h>

namespace idf {

__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                              uint32_t& c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
}

__device__ __forceinline__ float inv_n(float n) { return __fdiv_rn(1.0f, n); }

// ln of a normal binary32 u in (0, 1].
__device__ __forceinline__ float series_ln(float u) {
  const uint32_t bits = __float_as_uint(u);
  int e = (int)(bits >> 23) - 127;
  const uint32_t mb = bits & 0x7FFFFFu;
  float m;
  if (mb > 0x3504F3u) {
    m = __uint_as_float(mb | 0x3F000000u);
    e += 1;
  } else {
    m = __uint_as_float(mb | 0x3F800000u);
  }
  const float f = __fsub_rn(m, 1.0f);
  const float z = __fdiv_rn(f, __fadd_rn(m, 1.0f));
  const float w = __fmul_rn(z, z);
  float p = __fmul_rn(inv_n(11.0f), w);
  p = __fmul_rn(__fadd_rn(p, inv_n(9.0f)), w);
  p = __fmul_rn(__fadd_rn(p, inv_n(7.0f)), w);
  p = __fmul_rn(__fadd_rn(p, inv_n(5.0f)), w);
  p = __fmul_rn(__fadd_rn(p, inv_n(3.0f)), w);
  const float t = __fmul_rn(2.0f, z);
  const float lnm = __fadd_rn(t, __fmul_rn(t, p));
  const float ef = (float)e;
  const float ln2_hi = 0.693145751953125f;   // 22713 / 32768, exact
  const float ln2_lo = 0x1.7f7d1cp-20f;      // fl(ln 2 - 22713/32768)
  const float r = __fadd_rn(__fmul_rn(ef, ln2_lo), lnm);
  return __fadd_rn(__fmul_rn(ef, ln2_hi), r);
}

// cos(2 pi k 2^-24) for 0 <= k < 2^24.
__device__ __forceinline__ float series_cos2pi(int32_t k) {
  const int32_t q = (k + (1 << 21)) >> 22;
  const int32_t rk = k - (q << 22);
  const float r = __fmul_rn((float)rk, 0x1p-24f);
  const float th = __fmul_rn(r, 0x1.921fb6p+2f);  // fl(2 pi)
  const float x = __fmul_rn(th, th);
  float c = __fadd_rn(__fmul_rn(inv_n(479001600.0f), x), -inv_n(3628800.0f));
  c = __fadd_rn(__fmul_rn(c, x), inv_n(40320.0f));
  c = __fadd_rn(__fmul_rn(c, x), -inv_n(720.0f));
  c = __fadd_rn(__fmul_rn(c, x), inv_n(24.0f));
  c = __fadd_rn(__fmul_rn(c, x), -0.5f);
  const float C = __fadd_rn(1.0f, __fmul_rn(x, c));
  float s = __fadd_rn(__fmul_rn(-inv_n(39916800.0f), x), inv_n(362880.0f));
  s = __fadd_rn(__fmul_rn(s, x), -inv_n(5040.0f));
  s = __fadd_rn(__fmul_rn(s, x), inv_n(120.0f));
  s = __fadd_rn(__fmul_rn(s, x), -inv_n(6.0f));
  const float S = __fadd_rn(th, __fmul_rn(__fmul_rn(th, x), s));
  switch (q & 3) {
    case 0: return C;
    case 1: return -S;
    case 2: return -C;
    default: return S;
  }
}

__device__ __forceinline__ float normal_at(uint64_t seed, uint32_t level, uint32_t step,
                                           int64_t x, int64_t y) {
  uint32_t c0 = (uint32_t)(uint64_t)x, c1 = (uint32_t)(uint64_t)y, c2 = step, c3 = level;
  philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float u1 = __fmul_rn((float)((c0 >> 8) + 1u), 0x1p-24f);
  const float l = series_ln(u1);
  const float s = __fsqrt_rn(__fmul_rn(-2.0f, l));
  return __fmul_rn(s, series_cos2pi((int32_t)(c1 >> 8)));
}

}  // namespace idf
