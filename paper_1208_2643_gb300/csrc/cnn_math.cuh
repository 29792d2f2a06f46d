// GELU of the learned guess's network and its derivative, shared by the convolution
// kernels (mma.sync and tcgen05) so that both paths evaluate the same function.
//
// GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, GELU'(z) = Phi(z) + z phi(z).
// erf is Hastings' rational approximation as tabulated by Abramowitz & Stegun (1964),
// formula 7.1.26: for x >= 0, erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5))))
// exp(-x^2) with t = 1 / (1 + p x), absolute error <= 1.5e-7, extended to x < 0 by
// oddness.
//
// GELU itself is evaluated in the equivalent form
//   GELU(z) = max(z, 0) - (|z| / 2) t P(t) exp(-x^2),   x = |z| / sqrt 2,
// (for z >= 0, 1 + erf = 2 - t P e; for z < 0, 1 + erf = t P e), which needs no sign
// transfer and no separate product with z / 2.  With y = x sqrt(log2 e), exp(-x^2) =
// 2^(-y^2) is one hardware base-2 exponential, p x = (p / sqrt(log2 e)) y, and the
// factor |z| / 2 = y / (2 kGy) is folded into the polynomial's coefficients.  Each value
// takes its own hardware reciprocal: about 13 instructions a value, two of them on the
// special-function pipe.  A NaN input gives NaN (through |z| kGy); so does +-Inf.
#pragma once

namespace mpfc_cnn_math {

struct ErfExp {
  float erf;   // erf(z / sqrt 2)
  float e;     // exp(-z^2 / 2)
};

__device__ __forceinline__ ErfExp erf_exp_of(float z) {
  const float x = fabsf(z) * 0.70710678118654752f;
  const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
  const float poly =
      t * fmaf(fmaf(fmaf(fmaf(1.061405429f, t, -1.453152027f), t, 1.421413741f), t, -0.284496736f), t, 0.254829592f);
  const float e = __expf(-x * x);
  ErfExp r;
  r.erf = copysignf(fmaf(-poly, e, 1.0f), z);
  r.e = e;
  return r;
}

// 2^a (ex2.approx.ftz: subnormal results flush to 0) and 1/a (rcp.approx.ftz).
__device__ __forceinline__ float ex2_approx(float a) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ float rcp_approx(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

constexpr float kGy = 0.84932180028801907f;   // y = |z| kGy = (|z| / sqrt 2) sqrt(log2 e)
constexpr float kGp = 0.27273748087922250f;   // p / sqrt(log2 e), p = 0.3275911
constexpr float kGh = 0.58870501125773730f;   // 1 / (2 kGy): (|z| / 2) = y kGh

__device__ __forceinline__ float gelu(float z) {
  const float yr = fabsf(z) * kGy;
  const float t = rcp_approx(fmaf(kGp, yr, 1.0f));
  const float tp =
      t * fmaf(fmaf(fmaf(fmaf(1.061405429f * kGh, t, -1.453152027f * kGh), t, 1.421413741f * kGh), t,
                    -0.284496736f * kGh),
               t, 0.254829592f * kGh);
  const float e = ex2_approx(-yr * yr);
  return fmaf(-(yr * e), tp, fmaxf(z, 0.0f));
}

__device__ __forceinline__ float gelu_grad(float z) {
  const ErfExp r = erf_exp_of(z);
  return fmaf(z * 0.39894228040143268f, r.e, 0.5f * (1.0f + r.erf));
}

// GELU of 8 values (the epilogues' channel groups): gelu() on each, as independent
// instruction streams.
__device__ __forceinline__ void gelu8(const float (&z)[8], float (&g)[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) g[i] = gelu(z[i]);
}

}  // namespace mpfc_cnn_math
