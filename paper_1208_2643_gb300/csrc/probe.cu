// Measurement and test helpers (see include/mpfc_probe.h): the FP64 FMA-rate probe used
// for the roofline of the FP64 kernels, and device evaluations of the library's own
// reciprocal, precision conversions and GELU for tests against their error bounds.
#include <cuda_runtime.h>

#include "../../include/mpfc.h"
#include "../../include/mpfc_probe.h"
#include "cnn_math.cuh"
#include "mpfc_common.cuh"

namespace {
constexpr int kBlocksPerSM = 8, kThreads = 256, kIters = 2000;

__global__ void k_fma_chains(double* out, double seed) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  double a0 = seed + t * 1e-9, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
         a7 = a0 + 7;
  const double m = 0.999999, c = 1e-7;
  for (int i = 0; i < kIters; ++i) {
    a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
  }
  out[t] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}
}  // namespace

extern "C" int mpfc_probe_fp64_fma(void* d_scratch, void* cuda_stream, double* tflops) {
  if (!d_scratch || !tflops) return MPFC_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MPFC_ERR_CUDA;
  const int kBlocks = kBlocksPerSM * mpfc::sm_count();
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_chains<<<kBlocks, kThreads, 0, s>>>((double*)d_scratch, 1.0);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return MPFC_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return MPFC_ERR_CUDA;
  double fmas = (double)kBlocks * kThreads * kIters * 8.0;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return MPFC_OK;
}

namespace {
__global__ void k_rcp(const double* __restrict__ x, double* __restrict__ y, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = mpfc::rcp_nr(x[i]);
}
}  // namespace

extern "C" int mpfc_probe_rcp(const double* d_x, double* d_out, int n, void* cuda_stream) {
  if (!d_x || !d_out || n < 0) return MPFC_ERR_INVALID;
  if (n == 0) return MPFC_OK;
  k_rcp<<<(n + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(d_x, d_out, n);
  return cudaGetLastError() == cudaSuccess ? MPFC_OK : MPFC_ERR_CUDA;
}

namespace {
__global__ void k_convert(const double* __restrict__ x, float* __restrict__ rn, float* __restrict__ tr,
                          double* __restrict__ back, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    rn[i] = mpfc::f64_to_f32_rn(x[i]);
    tr[i] = mpfc::f64_to_f32_trunc(x[i]);
    back[i] = mpfc::f32_to_f64(rn[i]);
  }
}
}  // namespace

extern "C" int mpfc_probe_convert(const double* d_x, float* d_rn, float* d_trunc, double* d_back, int n,
                                  void* cuda_stream) {
  if (!d_x || !d_rn || !d_trunc || !d_back || n < 0) return MPFC_ERR_INVALID;
  if (n == 0) return MPFC_OK;
  k_convert<<<(n + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(d_x, d_rn, d_trunc, d_back, n);
  return cudaGetLastError() == cudaSuccess ? MPFC_OK : MPFC_ERR_CUDA;
}

namespace {
__global__ void k_gelu(const float* __restrict__ z, float* __restrict__ g, float* __restrict__ dg, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    g[i] = mpfc_cnn_math::gelu(z[i]);
    dg[i] = mpfc_cnn_math::gelu_grad(z[i]);
  }
}

// the 8-wide form: thread i evaluates z[8i .. 8i+7] (zero-padded past n)
__global__ void k_gelu8(const float* __restrict__ z, float* __restrict__ g, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (8 * i < n) {
    float zz[8], gg[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) zz[j] = 8 * i + j < n ? z[8 * i + j] : 0.0f;
    mpfc_cnn_math::gelu8(zz, gg);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (8 * i + j < n) g[8 * i + j] = gg[j];
  }
}
}  // namespace

extern "C" int mpfc_probe_gelu(const float* d_z, float* d_g, float* d_dg, int n, void* cuda_stream) {
  if (!d_z || !d_g || !d_dg || n < 0) return MPFC_ERR_INVALID;
  if (n == 0) return MPFC_OK;
  k_gelu<<<(n + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(d_z, d_g, d_dg, n);
  return cudaGetLastError() == cudaSuccess ? MPFC_OK : MPFC_ERR_CUDA;
}

extern "C" int mpfc_probe_gelu8(const float* d_z, float* d_g, int n, void* cuda_stream) {
  if (!d_z || !d_g || n < 0) return MPFC_ERR_INVALID;
  if (n == 0) return MPFC_OK;
  const int threads = (n + 7) / 8;
  k_gelu8<<<(threads + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(d_z, d_g, n);
  return cudaGetLastError() == cudaSuccess ? MPFC_OK : MPFC_ERR_CUDA;
}
