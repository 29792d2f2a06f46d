// GELU of the learned guess's network and its derivative, shared by the convolution
// kernels (mma.sync and tcgen05) so that both paths evaluate the same function.
//
// GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, GELU'(z) = Phi(z) + z phi(z).
// erf is Hastings' rational approximation as tabulated by Abramowitz & Stegun (1964),
// formula 7.1.26: for x >= 0, erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5))))
// exp(-x^2) with t = 1 / (1 + p x), absolute error <= 1.5e-7, extended to x < 0 by
// oddness.  It has no branches, so the 8-32 channel values a thread handles are
// evaluated as independent instruction streams; exp(-x^2) = exp(-z^2 / 2) also gives
// the normal density phi(z) of GELU' without a second exponential.
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

__device__ __forceinline__ float gelu(float z) {
  const ErfExp r = erf_exp_of(z);
  return 0.5f * z * (1.0f + r.erf);
}

__device__ __forceinline__ float gelu_grad(float z) {
  const ErfExp r = erf_exp_of(z);
  return fmaf(z * 0.39894228040143268f, r.e, 0.5f * (1.0f + r.erf));
}

}  // namespace mpfc_cnn_math

namespace mpfc_cnn_math {

// GELU of 8 values with one shared reciprocal: t_i = 1 / d_i is formed as
// (prod_{j != i} d_j) / (prod_j d_j), which trades 7 reciprocals for multiplies.
// x = |z| / sqrt 2 is clamped to 6 first (erf(6) rounds to 1 in binary32 and
// exp(-36) is below its resolution there), so d_i <= 3 and the product of eight
// stays below 3^8.  Same approximation and error bound as gelu() above, up to a few
// roundings of t.
__device__ __forceinline__ void gelu8(const float (&z)[8], float (&g)[8]) {
  float x[8], d[8], pre[8];
  float prod = 1.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    x[i] = fminf(fabsf(z[i]) * 0.70710678118654752f, 6.0f);
    d[i] = fmaf(0.3275911f, x[i], 1.0f);
    pre[i] = prod;          // d_0 ... d_{i-1}
    prod *= d[i];
  }
  float inv = __fdividef(1.0f, prod);   // 1 / (d_0 ... d_7)
#pragma unroll
  for (int i = 7; i >= 0; --i) {
    const float t = inv * pre[i];        // = 1 / d_i
    inv *= d[i];                         // 1 / (d_0 ... d_{i-1})
    const float poly =
        t * fmaf(fmaf(fmaf(fmaf(1.061405429f, t, -1.453152027f), t, 1.421413741f), t, -0.284496736f), t, 0.254829592f);
    const float e = __expf(-x[i] * x[i]);
    const float erf = copysignf(fmaf(-poly, e, 1.0f), z[i]);
    g[i] = 0.5f * z[i] * (1.0f + erf);
  }
}

}  // namespace mpfc_cnn_math
