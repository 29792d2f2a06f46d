/*
 * mpfc_probe.h -- measurement helpers of libmpfc (no counterpart in the paper).
 *
 * The FP64 kernels of the solver are bound by FP64 instruction issue on GB300, so
 * their roofline needs the FP64 FMA rate of the GPU they run on.
 */
#ifndef MPFC_PROBE_H
#define MPFC_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Measures the sustained FP64 FMA rate of the current device with a kernel of
 * independent FMA chains on every SM (about 10 ms of work, timed with CUDA events on
 * `cuda_stream`, best of three).  *tflops receives 2 x FMAs per second / 1e12.
 * `d_scratch` is device memory of at least SMs * 8 * 256 doubles, SMs the device's
 * multiprocessor count (written).  Returns 0 or MPFC_ERR_CUDA. */
int mpfc_probe_fp64_fma(void* d_scratch, void* cuda_stream, double* tflops);

/* Applies the smoother's double-precision reciprocal (one Newton-Raphson step from
 * the correctly rounded single-precision reciprocal) to n device doubles, for tests
 * of its error bound.  Asynchronous on `cuda_stream`. */
int mpfc_probe_rcp(const double* d_x, double* d_out, int n, void* cuda_stream);

/* Applies the library's integer-pipe binary64 <-> binary32 conversions to n device
 * doubles: d_rn = rounded to nearest even, d_trunc = rounded toward zero, d_back = d_rn
 * widened back to binary64.  Any input: zero, the normal binary32 range, underflow to
 * subnormals, overflow, infinities and NaN (the last four through the hardware
 * conversion).  For tests against the hardware conversions.  Asynchronous on
 * `cuda_stream`. */
int mpfc_probe_convert(const double* d_x, float* d_rn, float* d_trunc, double* d_back, int n, void* cuda_stream);

/* Evaluates the convolution kernels' GELU and its derivative (erf by the rational
 * approximation of Abramowitz & Stegun 7.1.26, absolute error <= 1.5e-7) on n device
 * floats: d_g = GELU(z), d_dg = GELU'(z).  For tests against the exact functions.
 * Asynchronous on `cuda_stream`. */
int mpfc_probe_gelu(const float* d_z, float* d_g, float* d_dg, int n, void* cuda_stream);

/* The same GELU in the 8-wide form the tcgen05 convolution uses (one reciprocal shared
 * by eight values): d_g[i] = GELU(d_z[i]) for n device floats, evaluated in groups of
 * eight consecutive values.  Asynchronous on `cuda_stream`. */
int mpfc_probe_gelu8(const float* d_z, float* d_g, int n, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif
