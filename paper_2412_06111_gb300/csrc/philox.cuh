// Device DRM generator: Philox4x32-10 (Salmon et al., SC'11) and the
// Box-Muller transform with ln / sin / cos evaluated from their series using
// only correctly rounded binary64 +, -, *, / and sqrt (the __d*_rn
// intrinsics, which are never contracted into FMAs).  The same operation
// sequence on any IEEE-754 machine gives the same bits, which is how the
// device factors are made identical to an independent host generator.
#pragma once

#include <stdint.h>

namespace ttnn {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// nearest binary64 values of ln 2, sqrt 2, pi / 4
constexpr double kLn2 = 0.6931471805599453;
constexpr double kSqrt2 = 1.4142135623730951;
constexpr double kPi4 = 0.7853981633974483;
constexpr int kLnTerms = 11;   // atanh series z^(2k)/(2k+1), k = 0..11
constexpr int kSinTerms = 8;   // to psi^17 / 17!
constexpr int kCosTerms = 9;   // to psi^18 / 18!

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c[0]), lo0 = kPhiloxM0 * c[0];
    const uint32_t hi1 = __umulhi(kPhiloxM1, c[2]), lo1 = kPhiloxM1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
}

// ln u for u in (0, 1]: u = m 2^e with m in [sqrt2/2, sqrt2] (exact bit
// split), ln m = 2 atanh((m - 1)/(m + 1)) by its odd power series.
__device__ __forceinline__ double ln_series(double u) {
  const long long bits = __double_as_longlong(u);
  const int ex = (int)((bits >> 52) & 0x7ff) - 1023;          // u is normal here
  double m = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFLL) | (1023LL << 52));
  double e = (double)ex;
  if (m > kSqrt2) {
    m = __dmul_rn(m, 0.5);
    e = __dadd_rn(e, 1.0);
  }
  const double z = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double z2 = __dmul_rn(z, z);
  double p = __ddiv_rn(1.0, (double)(2 * kLnTerms + 1));
  for (int k = kLnTerms - 1; k >= 0; --k) {
    p = __dmul_rn(p, z2);
    p = __dadd_rn(p, __ddiv_rn(1.0, (double)(2 * k + 1)));
  }
  const double t = __dmul_rn(z, p);
  const double lnm = __dadd_rn(t, t);
  return __dadd_rn(__dmul_rn(e, kLn2), lnm);
}

// (sin 2 pi u, cos 2 pi u), u in [0, 1): exact octant reduction t = 8u.
__device__ __forceinline__ void sincos_2pi(double u, double* s_out, double* c_out) {
  const double t = __dmul_rn(u, 8.0);
  const int k = (int)t;                       // floor, t >= 0
  const double f = __dsub_rn(t, (double)k);   // exact
  const double g = (k & 1) ? __dsub_rn(1.0, f) : f;   // exact
  const double psi = __dmul_rn(g, kPi4);
  const double x2 = __dmul_rn(psi, psi);
  double s = 1.0;
  for (int j = kSinTerms; j >= 1; --j) {
    double q = __dmul_rn(x2, s);
    q = __ddiv_rn(q, (double)((2 * j) * (2 * j + 1)));
    s = __dsub_rn(1.0, q);
  }
  s = __dmul_rn(psi, s);
  double c = 1.0;
  for (int j = kCosTerms; j >= 1; --j) {
    double q = __dmul_rn(x2, c);
    q = __ddiv_rn(q, (double)((2 * j - 1) * (2 * j)));
    c = __dsub_rn(1.0, q);
  }
  double sn, cs;
  switch (k) {
    case 0: sn = s; cs = c; break;
    case 1: sn = c; cs = s; break;
    case 2: sn = c; cs = -s; break;
    case 3: sn = s; cs = -c; break;
    case 4: sn = -s; cs = -c; break;
    case 5: sn = -c; cs = -s; break;
    case 6: sn = -c; cs = s; break;
    default: sn = -s; cs = c; break;
  }
  *s_out = sn;
  *c_out = cs;
}

// N(0,1) value of element (i, j) of factor (kind, ident) for `seed`.
__device__ __forceinline__ double philox_gaussian(uint64_t seed, uint32_t kind, uint32_t ident,
                                                  uint64_t i, uint64_t j) {
  uint32_t c[4] = {(uint32_t)i, (uint32_t)(j >> 1), (kind << 24) | (ident & 0xFFFFFFu), 0u};
  philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  const unsigned long long hi = ((unsigned long long)c[0] << 32) | c[1];
  const unsigned long long lo = ((unsigned long long)c[2] << 32) | c[3];
  const double s53 = 1.1102230246251565e-16;  // 2^-53
  const double u1 = __dmul_rn(__dadd_rn(__ull2double_rn(hi >> 11), 1.0), s53);
  const double u2 = __dmul_rn(__ull2double_rn(lo >> 11), s53);
  const double r = __dsqrt_rn(__dmul_rn(ln_series(u1), -2.0));
  double sn, cs;
  sincos_2pi(u2, &sn, &cs);
  return (j & 1) ? __dmul_rn(r, sn) : __dmul_rn(r, cs);
}

// Round-to-nearest-even of x into a format with p significand bits,
// exponent floor emin and largest finite value vmax (saturate or inf).
__device__ __forceinline__ double round_fmt(double x, int fmt) {
  if (fmt == 0) return x;
  int p, emin;
  double vmax;
  bool sat;
  if (fmt == 1) { p = 24; emin = -126; vmax = 3.4028234663852886e38; sat = false; }
  else if (fmt == 2) { p = 8; emin = -126; vmax = 3.3895313892515355e38; sat = false; }
  else { p = 4; emin = -6; vmax = 448.0; sat = true; }
  const double a = fabs(x);
  if (a == 0.0 || !(a == a)) return x;
  const long long bits = __double_as_longlong(a);
  int ex = (int)((bits >> 52) & 0x7ff);
  if (ex == 0x7ff) return x;                       // inf stays inf
  ex = (ex == 0) ? -1023 : ex - 1023;              // binary64 subnormals: far below emin
  int e = ex < emin ? emin : ex;
  const int se = e - (p - 1);
  // exact scalings by powers of two (se in [-133, 127] for these formats)
  const double q = rint(ldexp(a, -se));
  double r = ldexp(q, se);
  if (r > vmax) r = sat ? vmax : __longlong_as_double(0x7FF0000000000000LL);
  return copysign(r, x);
}

}  // namespace ttnn
