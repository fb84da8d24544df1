// fastrcp.cuh - double reciprocal and reciprocal square root from a float seed, and the
// float approximations they start from; shared by the update kernel and the small dense
// kernels (FP64 division and square root are long sequences on this GPU).
#pragma once
#include "common.cuh"

namespace tdb {

// ---------------------------------------------------------------------------
// Double reciprocal and reciprocal square root by Newton-Raphson iteration from a
// float seed (the textbook method; e.g. P. Markstein, IA-64 and Elementary
// Functions, 2000, ch. 8).  The seed is the hardware float approximation
// (rcp.approx / rsqrt.approx) of x truncated to float, built from the bit pattern with
// integer operations (no double-pipe conversion).  Reciprocal: with e0 = 1 - x y0,
// Newton's step on f(y) = 1/y - x gives y1 = y0 (1 + e0), whose residual is e0^2; a
// second step y1 (1 + e0^2) leaves e0^4 (the square formed alongside the first step,
// three dependent operations).  Reciprocal square root: two Newton steps on
// f(y) = 1/y^2 - x, y <- y + (y/2)(1 - x y^2), each squaring the relative error.  The
// float seed is good to about 2^-22, so two steps leave far less than one double ulp
// before the final rounding; tests check both against 1/x and 1/sqrt(x) within 2 ulp.
// |x| outside [2^-120, 2^120] takes the plain division (and square root).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool seedable(double x) {
  const unsigned e = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
  return e >= 903u && e <= 1143u;
}
__device__ __forceinline__ float f32_trunc(double x) {        // mantissa truncated to 23 bits
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  return __uint_as_float((hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
__device__ __forceinline__ double f64_exact(float f) {        // normal float to double, exact
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  return __hiloint2double((int)((b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)),
                          (int)((b & 7u) << 29));
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double drcp(double x) {
  if (!seedable(x)) return 1.0 / x;
  const double y0 = f64_exact(rcp_approx(f32_trunc(x)));
  const double e0 = fma(-x, y0, 1.0);           // x y0 = 1 - e0
  const double y1 = fma(y0, e0, y0);            // y0 (1 + e0)
  const double e1 = e0 * e0;                    // alongside y1
  return fma(y1, e1, y1);                       // y0 (1 + e0)(1 + e0^2): residual e0^4
}
__device__ __forceinline__ double drsqrt(double x) {           // x > 0
  if (!seedable(x)) return 1.0 / sqrt(x);
  double y = f64_exact(rsqrt_approx(f32_trunc(x)));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double h = x * y;
    const double t = fma(-h, y, 1.0);                          // 1 - x y^2
    y = fma(0.5 * y, t, y);
  }
  return y;
}


}  // namespace tdb
