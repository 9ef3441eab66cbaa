// FP64 sine and cosine of the HMF stages (Eq. 7 needs cos and sin of every new
// angle), table-driven, with most of the work off the FP64 pipe.
//
// Method (Tang's table-driven reduction, ACM TOMS 15, 1989, applied to sine and
// cosine by Gal and Bachelis, ACM TOMS 17, 1991): theta = k h + r with
// h = pi/2048, k a nearest integer to theta / h and |r| <= h/2 (1 + 1e-4), then
//   sin(theta) = S_k (1 + cm) + C_k sr,   cos(theta) = C_k (1 + cm) - S_k sr
// with (S_k, C_k) = (sin, cos)(k h) from a 4096-entry FP64 table (k mod 4096),
// sr = sin r and cm = cos r - 1.
//
// On GB300 the FP64 pipe issues 2 operations per SM per clock against 128 for FP32,
// so only what needs 53 bits runs in FP64:
// * k comes from FP32 arithmetic on a two-float split of theta (th_hi = theta
//   truncated to 24 bits, th_lo the next 24) and of 2048/pi (hi + lo): the product's
//   rounding error (2MultFMA) and the small cross terms are kept, so the estimate of
//   theta / h is off by less than 4e-5 for |theta| < 2^20 and k is a nearest integer
//   up to that margin.  k as a double is assembled from its bits on the integer pipe.
// * r1 = theta - k h1 (h1 = fl(h)) is one FMA and exact: theta and k h1 are
//   multiples of 2^-63 and |r1| < 2^-10, so the difference has at most 53 bits.
//   The true r is r1 + c2 with c2 = -k h2 (h2 = fl(h - h1); h - h1 - h2 < 2e-36),
//   |c2| < 5e-11.
// * The terms below 2^-33 run in FP32 on rt = fl32(r1) + c2:
//     dlt = sin r - r1 = c2 - r^3/6           (|.| < 1.3e-10; first omitted term
//                                               r^5/5! < 2.3e-18)
//     eps = cos r - 1 + r1^2/2 = r^4/24 - r1 c2  (|.| < 5e-14; omitted c2^2/2 < 2e-21,
//                                               r^6/6! < 3e-22)
//   Their FP32 rounding errors are below 5e-17 (dlt) and 1e-20 (eps), under half a
//   unit in the last place of the FP64 results (|S_k|, |C_k| ~ 1).
// * FP64 (8 operations): r1, r1^2, cm = -r1^2/2 + eps, sr = r1 + dlt, and two FMAs
//   for each of sin and cos.  Float <-> double moves are bit manipulations.
// |theta| >= 2^20, infinities and NaN (found from the exponent bits) use sincos.
//
// The arithmetic is written with explicitly rounded operations only (no
// contraction) and compiles for the host as well, so the CPU can check it against a
// long-double libm bit for bit with what the GPU computes.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cuda_runtime.h>

namespace sc64 {

constexpr int kTabN = 4096;                        // table entries over one turn
constexpr double kH1 = 0x1.921fb54442d18p-10;      // pi / 2048 rounded to double
constexpr double kH2 = 0x1.1a62633145c07p-64;      // pi / 2048 - kH1
constexpr float kH2f = 0x1.1a6264p-64f;            // kH2 rounded to float
constexpr float kInvHHi = 0x1.45f306p+9f;          // 2048 / pi rounded to float
constexpr float kInvHLo = 0x1.b93910p-16f;         // 2048 / pi - kInvHHi rounded to float
constexpr unsigned kExpLimit = 1023u + 20u;        // table path for |theta| < 2^20

// ----------------------------------------------------------- bit moves ------
__host__ __device__ __forceinline__ uint64_t dbits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  memcpy(&u, &d, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ double bitsd(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  memcpy(&d, &u, sizeof d);
  return d;
#endif
}
__host__ __device__ __forceinline__ unsigned fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ float bitsf(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, sizeof f);
  return f;
#endif
}

// ------------------------------------------------- rounded arithmetic ------
__host__ __device__ __forceinline__ float fmul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  volatile float r = a * b;
  return r;
#endif
}
__host__ __device__ __forceinline__ float fadd(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  volatile float r = a + b;
  return r;
#endif
}
__host__ __device__ __forceinline__ double dmul(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  volatile double r = a * b;
  return r;
#endif
}
__host__ __device__ __forceinline__ double dadd(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(a, b);
#else
  volatile double r = a + b;
  return r;
#endif
}
// Nearest integer (ties to even) of a float, as a float.
__host__ __device__ __forceinline__ float frint(float x) { return rintf(x); }
// An integer-valued float of magnitude below 2^31 as an int (exact).
__host__ __device__ __forceinline__ int f2i_exact(float x) {
#ifdef __CUDA_ARCH__
  return __float2int_rz(x);
#else
  return (int)x;
#endif
}
// An unsigned integer below 2^29 as a float, rounded to nearest.
__host__ __device__ __forceinline__ float u2f(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(u);
#else
  return (float)u;
#endif
}
__host__ __device__ __forceinline__ int clz32(unsigned u) {
#ifdef __CUDA_ARCH__
  return __clz((int)u);
#else
  return u ? __builtin_clz(u) : 32;
#endif
}

// Exact float -> double (bits); zero and subnormal floats give a signed zero.
// Infinities and NaN never reach it.
__host__ __device__ __forceinline__ double f2d(float f) {
  const unsigned u = fbits(f);
  const unsigned a = u & 0x7fffffffu;
  if (a < 0x00800000u) return bitsd((uint64_t)(u & 0x80000000u) << 32);
  const uint64_t hi = (uint64_t)((u & 0x80000000u) | ((a >> 3) + 0x38000000u));
  return bitsd((hi << 32) | (uint64_t)(a << 29));
}

// double -> float rounded to nearest (halves away from zero) for |d| < 2^127 by adding
// half a float unit to the 64-bit pattern and truncating; below the float normal
// range it gives a signed zero.
__host__ __device__ __forceinline__ float d2f_rn(double d) {
  const uint64_t b = dbits(d) + (1ull << 28);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned a = hi & 0x7fffffffu;
  unsigned fb = ((a - 0x38000000u) << 3) | (lo >> 29);
  if (a < 0x38100000u) fb = 0u;
  return bitsf((hi & 0x80000000u) | fb);
}

// An int of magnitude below 2^31 as a double (exact): sign, exponent 1023 + 31 - clz,
// and the bits below the leading one as the top of the 52-bit fraction.
__host__ __device__ __forceinline__ double i2d(int k) {
  const unsigned a = k < 0 ? 0u - (unsigned)k : (unsigned)k;
  if (a == 0u) return 0.0;
  const int lz = clz32(a);
  const unsigned m = (a << lz) << 1;  // fraction bits, left-aligned
  const unsigned hi = (k < 0 ? 0x80000000u : 0u) | ((unsigned)(1054 - lz) << 20) | (m >> 12);
  return bitsd(((uint64_t)hi << 32) | (uint64_t)(m << 20));
}

// ------------------------------------------------------ sine and cosine ------
// tab[k] = (sin, cos)(k pi / 2048), k = 0 .. kTabN - 1, each rounded to double.
__host__ __device__ __forceinline__ void sincos_tab(double th, const double2 *tab, double *sp, double *cp) {
  const uint64_t b = dbits(th);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned E = (hi >> 20) & 0x7ffu;
  if (E >= kExpLimit) {  // |theta| >= 2^20, infinities, NaN
#ifdef __CUDA_ARCH__
    sincos(th, sp, cp);
#else
    *sp = sin(th);
    *cp = cos(th);
#endif
    return;
  }
  // k: theta = th_hi + th_lo (+ < 2^-47 |theta|), th_hi the top 24 bits of theta, th_lo
  // the next 29 bits rounded to a float (units of 2^(E - 1075))
  const unsigned sign = hi & 0x80000000u, a = hi & 0x7fffffffu;
  float th_hi = bitsf(sign | (((a - 0x38000000u) << 3) | (lo >> 29)));
  if (a < 0x38100000u) th_hi = 0.0f;  // |theta| < 2^-126: k = 0
  float th_lo = 0.0f;
  if (E >= 949u) th_lo = bitsf(fbits(fmul(u2f(lo & 0x1fffffffu), bitsf((E - 948u) << 23))) | sign);
  const float pr = fmul(th_hi, kInvHHi);
  const float pe = fmaf(th_hi, kInvHHi, -pr);                    // exact: th_hi kInvHHi = pr + pe
  const float ps = fmaf(th_hi, kInvHLo, fmul(th_lo, kInvHHi));   // the cross terms
  const float kp = frint(pr);
  const float ka = frint(fadd(fadd(pr, -kp), fadd(pe, ps)));     // pr - kp is exact
  const int k = f2i_exact(kp) + f2i_exact(ka);
  // r = r1 + c2: r1 exact in FP64, c2 and the small terms in FP32
  const double r1 = fma(-i2d(k), kH1, th);
  const float c2 = fmul(fadd(kp, ka), -kH2f);
  const float rf = d2f_rn(r1);
  const float rt = fadd(rf, c2);
  const float r2f = fmul(rt, rt);
  const float dlt = fmaf(fmul(r2f, rt), -1.0f / 6.0f, c2);
  const float eps = fmaf(r2f, fmul(r2f, 1.0f / 24.0f), -fmul(rf, c2));
  const double r2 = dmul(r1, r1);
  const double cm = fma(r2, -0.5, f2d(eps));
  const double sr = dadd(r1, f2d(dlt));
  const double2 t = tab[k & (kTabN - 1)];
  *sp = fma(t.x, cm, fma(t.y, sr, t.x));
  *cp = fma(t.y, cm, fma(-t.x, sr, t.y));
}

}  // namespace sc64
