// Activation functions of the calculation stage (f_n of Sec. 3.3 applies one
// per node), written for short dependent chains without divergent branches:
// a node evaluation sits on the critical path of every layer, and the
// library's general-purpose expf / tanhf / sinf carry slow paths and
// branches that a warp evaluating nodes of mixed activations pays for in
// full.  Methods (all in fp32):
//   exp   the argument clamped to [-87, 88] (NaN passes through), then Cody
//         and Waite's reduction x = k ln2 + r, |r| <= ln2 / 2 (ln2 split in a
//         15-bit high part, so k ln2_hi is exact, and a low part);
//         e^r - 1 = r Q(r) with Q the Taylor series of (e^r - 1) / r to
//         degree 6 (truncation below 2e-8 relative); e^x = (r Q(r) + 1) 2^k,
//         k in [-126, 127], scaled exactly; e^x - 1 = r Q(r) itself when
//         k = 0 (no cancellation near x = 0), else e^x - 1 (|e^x - 1| >= 0.29:
//         no cancellation either).  The clamp keeps every result finite and
//         normal: below e^-87 the result is e^-87 (1.6e-38) and above e^88 it
//         is e^88, which moves sigmoid, tanh and gaussian by less than 2e-38
//         where it applies.
//   1/d   (1 <= d < 2^128) the hardware reciprocal approximation refined by
//         one Newton-Raphson step, y = y0 + y0 (1 - d y0); a result below
//         2^-126 flushes to 0.
//   tanh  tanh |z| = -m / (2 + m) with m = e^{-2|z|} - 1 from the above (the
//         reciprocal shared with sigmoid's 1 / (2 + (e^{-z} - 1))), sign of z.
//   sin   Cody-Waite reduction by pi/2 with a three-part constant, each step a
//         fused multiply-add (the product k c_i exact inside it, one rounding
//         of a result below 1 in magnitude), then the Taylor polynomials of
//         sin (to r^9) and cos (to r^10) on |r| <= pi/4 and the quadrant
//         k mod 4.  Valid for |k| < 2^22; beyond |z| = 2^22 pi/2 (6.5e6)
//         sinf takes the argument.
// Each of sigmoid, tanh and sin stays within a few units of the last place of
// the exact value (the error bound the parity tests assume is 8 * 2^-24
// relative for them); gaussian e^{-z^2} adds the rounding of z^2.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace neat {
namespace am {

constexpr float LOG2E = 1.44269504088896340736f;
constexpr float LN2_HI = 0.693145751953125f;  // 0x3f317200: 15 significant bits
constexpr float LN2_LO = 1.42860676533018725e-06f;
constexpr float MAGIC = 12582912.0f;  // 1.5 * 2^23: x + MAGIC rounds x to an integer
constexpr int MAGIC_BITS = 0x4B400000;
constexpr float TWO_OVER_PI = 0.636619772367581343076f;
constexpr float PIO2_1 = 1.5707963705062866f;      // fp32(pi/2)
constexpr float PIO2_2 = -4.371138828673793e-08f;  // fp32(pi/2 - PIO2_1)
constexpr float PIO2_3 = -1.7151245100058819e-15f; // fp32(pi/2 - PIO2_1 - PIO2_2)
constexpr float SIN_ARG_MAX = 6.5e6f;

// e^x and e^x - 1 (see the header comment)
__device__ __forceinline__ void exp_expm1_cw(float x, float &e, float &m) {
  float xc;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(xc) : "f"(x), "f"(-87.0f));
  asm("min.NaN.f32 %0, %1, %2;" : "=f"(xc) : "f"(xc), "f"(88.0f));
  const float t = fmaf(xc, LOG2E, MAGIC);
  const float k = t - MAGIC;
  const int ki = __float_as_int(t) - MAGIC_BITS;
  float r = fmaf(k, -LN2_HI, xc);
  r = fmaf(k, -LN2_LO, r);
  float p = 1.98412698412698413e-4f;        // 1/7!
  p = fmaf(p, r, 1.38888888888888889e-3f);  // 1/6!
  p = fmaf(p, r, 8.33333333333333333e-3f);  // 1/5!
  p = fmaf(p, r, 4.16666666666666667e-2f);  // 1/4!
  p = fmaf(p, r, 1.66666666666666667e-1f);  // 1/3!
  p = fmaf(p, r, 0.5f);
  p = fmaf(p, r, 1.0f);
  const float rq = r * p;  // e^r - 1
  // (a NaN argument leaves rq NaN, whatever the scale's bits)
  e = (rq + 1.0f) * __int_as_float((ki + 127) << 23);
  m = ki == 0 ? rq : e - 1.0f;
}

// 1 / d for finite d >= 1, or NaN
__device__ __forceinline__ float rcp_nr(float d) {
  float y0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(d));
  return fmaf(fmaf(-d, y0, 1.0f), y0, y0);
}

// sin z and cos z for |z| <= SIN_ARG_MAX (quadrant k mod 4 of the reduction)
__device__ __forceinline__ void sincos_cw(float z, float &s_out, float &c_out) {
  const float t = fmaf(z, TWO_OVER_PI, MAGIC);
  const float k = t - MAGIC;
  const int q = __float_as_int(t) - MAGIC_BITS;
  float r = fmaf(k, -PIO2_1, z);
  r = fmaf(k, -PIO2_2, r);
  r = fmaf(k, -PIO2_3, r);
  const float w = r * r;
  float ps = 2.75573192239858907e-6f;        // 1/9!
  ps = fmaf(ps, w, -1.98412698412698413e-4f);  // -1/7!
  ps = fmaf(ps, w, 8.33333333333333333e-3f);   // 1/5!
  ps = fmaf(ps, w, -1.66666666666666667e-1f);  // -1/3!
  const float s = fmaf(r * w, ps, r);
  float pc = -2.75573192239858907e-7f;        // -1/10!
  pc = fmaf(pc, w, 2.48015873015873016e-5f);   // 1/8!
  pc = fmaf(pc, w, -1.38888888888888889e-3f);  // -1/6!
  pc = fmaf(pc, w, 4.16666666666666667e-2f);   // 1/4!
  pc = fmaf(pc, w, -0.5f);
  const float c = fmaf(w, pc, 1.0f);
  // sin z = (s, c, -s, -c)[q mod 4]; cos z = (c, -s, -c, s)[q mod 4]
  const float a = (q & 1) ? c : s, b = (q & 1) ? s : c;
  s_out = (q & 2) ? -a : a;
  c_out = ((q + 1) & 2) ? -b : b;
}

__device__ __forceinline__ float sin_cw(float z) {
  float s, c;
  sincos_cw(z, s, c);
  return s;
}

__device__ __forceinline__ float cos_cw(float z) {
  float s, c;
  sincos_cw(z, s, c);
  return c;
}

}  // namespace am
}  // namespace neat
