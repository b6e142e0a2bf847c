// Key path of the preprocess kernel (included by preprocess.cu only; it owns the constant).
#pragma once

#include "common.cuh"

namespace ges {

// Coefficients of the key-path exp2 series (ln2^k / k!, rounded to float), set by the host.
__constant__ float c_exp2_coef[8];

// 2^x: x = n + f with n = rint(x); 2^f by its degree-7 Taylor series in f (coefficients
// ln2^k/k!), Horner order, then an exact scaling by 2^n.  x is clamped to [-100, 126].
__device__ __forceinline__ float key_exp2(float x) {
  if (!(x <= 126.0f)) x = 126.0f;
  if (!(x >= -100.0f)) x = -100.0f;
  float n = rintf(x);
  float f = ksub(x, n);
  float p = c_exp2_coef[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) {
    p = kmul(p, f);
    p = kadd(p, c_exp2_coef[k]);
  }
  return ldexpf(p, (int)n);
}

// log2(x) for finite normal x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)];
// ln m = 2 atanh(s), s = (m-1)/(m+1), series to s^11.
__device__ __forceinline__ float key_log2(float x) {
  uint32_t b = __float_as_uint(x);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
  const float sqrt2 = (float)1.4142135623730951;
  if (m > sqrt2) {
    m = kmul(m, 0.5f);
    e = e + 1;
  }
  float s = kdiv(ksub(m, 1.0f), kadd(m, 1.0f));
  float s2 = kmul(s, s);
  float p = (float)(1.0 / 11.0);
  p = kmul(p, s2); p = kadd(p, (float)(1.0 / 9.0));
  p = kmul(p, s2); p = kadd(p, (float)(1.0 / 7.0));
  p = kmul(p, s2); p = kadd(p, (float)(1.0 / 5.0));
  p = kmul(p, s2); p = kadd(p, (float)(1.0 / 3.0));
  p = kmul(p, s2); p = kadd(p, 1.0f);
  float ln_m = kmul(kmul(2.0f, s), p);
  const float log2e = (float)1.4426950408889634;
  return kadd((float)e, kmul(ln_m, log2e));
}

// ln Gamma(x) for x > 0: Gamma(x) = Gamma(z) / (x (x+1) ... (z-1)) with z = x + k the first shift at
// or above 4 (k <= 4), then Stirling's series for ln Gamma(z),
//   (z - 1/2) ln z - z + ln(2 pi)/2 + 1/(12 z) - 1/(360 z^3) + 1/(1260 z^5) - 1/(1680 z^7),
// whose first omitted term, 1/(1188 z^9), is below 4e-9 at z >= 4.  ln via key_log2 * ln 2.
__device__ __forceinline__ float key_lgamma(float x) {
  const float ln2 = (float)0.6931471805599453;
  float z = x, acc = 1.0f;
  for (int k = 0; k < 4 && z < 4.0f; ++k) {
    acc = kmul(acc, z);
    z = kadd(z, 1.0f);
  }
  const float r = kdiv(1.0f, z);
  const float r2 = kmul(r, r);
  float ser = -(float)(1.0 / 1680.0);
  ser = kmul(ser, r2); ser = kadd(ser, (float)(1.0 / 1260.0));
  ser = kmul(ser, r2); ser = ksub(ser, (float)(1.0 / 360.0));
  ser = kmul(ser, r2); ser = kadd(ser, (float)(1.0 / 12.0));
  ser = kmul(ser, r);
  const float lz = kmul(key_log2(z), ln2);
  float lg = kmul(ksub(z, 0.5f), lz);
  lg = ksub(lg, z);
  lg = kadd(lg, (float)0.91893853320467274);  // ln(2 pi) / 2
  lg = kadd(lg, ser);
  return ksub(lg, kmul(key_log2(acc), ln2));
}

// The scale modification phi(beta) (Sec. 4.2) applied to the scale vector:
//   phi_mode 0: phi_bar_rho(beta) = 2 / (1 + 2^(-rho (beta - 2) log2 e))                   Eq. approx
//   phi_mode 1: phi_n(beta) = 2 Gamma(3/beta) / Gamma(1/beta)                            Eq. probablity
//               = 2^((ln Gamma(3/beta) - ln Gamma(1/beta) + ln 2) log2 e), 1 at beta = 2
//   phi_mode 2: sqrt(phi_n(beta)), phi_n read as a ratio of variances (Eq. effective)
__device__ __forceinline__ float key_phi(float beta, const Params& P) {
  const float log2e = (float)1.4426950408889634;
  if (P.phi_mode == 0) {
    const float rdb = kmul(P.rho, ksub(beta, 2.0f));
    const float ex = key_exp2(kmul(-rdb, log2e));
    return kdiv(2.0f, kadd(1.0f, ex));
  }
  const float g3 = key_lgamma(kdiv(3.0f, beta));
  const float g1 = key_lgamma(kdiv(1.0f, beta));
  float e = kmul(kadd(ksub(g3, g1), (float)0.6931471805599453), log2e);
  if (P.phi_mode == 2) e = kmul(e, 0.5f);
  return key_exp2(e);
}

}  // namespace ges
