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

}  // namespace ges
