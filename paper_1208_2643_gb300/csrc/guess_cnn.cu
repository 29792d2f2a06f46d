// Learned initial guess inside the solver (MPFC_GUESS_LEARNED): before each step's
// V-cycles, the network of mpfc_cnn.h predicts the error of the linear extrapolation
// from phi^k, phi^{k-1}, phi^{k-2}, and its output, scaled back, is added to the
// extrapolated phi^(0).  mu^(0), kappa^(0) then follow from phi^(0) as for the other
// guesses, and the V-cycles run to the same tolerance.
#include <cuda_bf16.h>
#include <string.h>

#include <vector>

#include "../../include/mpfc.h"
#include "../../include/mpfc_cnn.h"
#include "cnn_math.cuh"
#include "mpfc_internal.h"

int mpfc_cnn_conv_guess(const void* x, int H, int W, int cin_p, const void* wk, const float* bias, double* phi0,
                        double scale, cudaStream_t s);
int mpfc_cnn_conv_layer(const void* x, int H, int W, int cin_p, const void* wk, const float* bias, int cout,
                        void* y_bf16, cudaStream_t s);

namespace {
// (cin, cout, cin_p, cout_p) of the five layers
const int kLayers[5][4] = {{3, 32, 4, 32}, {32, 32, 32, 32}, {32, 32, 32, 32}, {32, 32, 32, 32}, {32, 1, 32, 8}};
int kpad_of(int cin_p) { return (9 * cin_p + 15) / 16 * 16; }

// Output tiles of the two inference kernels: 32 x 8 pixels, one per thread.
constexpr int kGX = 32, kGY = 8;

__device__ __forceinline__ int gwrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }
__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// First layer of the inference, with its input: the three normalised features of each
// pixel of the tile and its one-pixel periodic halo (x0 = (phi^k - mean)/s0,
// x1 = (phi^k - phi^{k-1})/s1, x2 = (phi^k - 2 phi^{k-1} + phi^{k-2})/s2, differences
// in FP64, rounded to bf16 like the training input), then the 3 -> 32 convolution in
// FP32 multiply-adds of those bf16 values with the bf16 weights (exact products, as on
// the tensor cores), bias, GELU, and the 32 channels as bf16 (64 bytes per pixel).
__global__ void __launch_bounds__(kGX * kGY) k_guess_in(const __grid_constant__ GuessInArgs P,
                                                        const double* __restrict__ pk, const double* __restrict__ pkm1,
                                                        const double* __restrict__ pkm2, const double* __restrict__ mean_p,
                                                        int m, int n, __nv_bfloat16* __restrict__ act) {
  __shared__ float feat[3][kGY + 2][kGX + 2];
  mpfc::pdl_enter();
  const int x0 = blockIdx.x * kGX, y0 = blockIdx.y * kGY;
  const double mean = *mean_p;
  for (int t = threadIdx.x; t < (kGX + 2) * (kGY + 2); t += kGX * kGY) {
    const int ty = t / (kGX + 2), tx = t - ty * (kGX + 2);
    const size_t g = (size_t)gwrap(y0 + ty - 1, n) * m + gwrap(x0 + tx - 1, m);
    const double a = pk[g], c1 = pkm1[g], c2 = pkm2[g];
    feat[0][ty][tx] = bf16_round(mpfc::f64_to_f32_rn((a - mean) * P.inv[0]));
    feat[1][ty][tx] = bf16_round(mpfc::f64_to_f32_rn((a - c1) * P.inv[1]));
    feat[2][ty][tx] = bf16_round(mpfc::f64_to_f32_rn(((a - c1) - (c1 - c2)) * P.inv[2]));
  }
  __syncthreads();
  const int tx = threadIdx.x % kGX, ty = threadIdx.x / kGX;
  const int x = x0 + tx, y = y0 + ty;
  if (x >= m || y >= n) return;
  float acc[32];
#pragma unroll
  for (int co = 0; co < 32; ++co) acc[co] = 0.f;
#pragma unroll
  for (int tap = 0; tap < 9; ++tap)
#pragma unroll
    for (int ci = 0; ci < 3; ++ci) {
      const float v = feat[ci][ty + tap / 3][tx + tap % 3];
#pragma unroll
      for (int co = 0; co < 32; ++co) acc[co] = fmaf(v, P.w[tap * 3 + ci][co], acc[co]);
    }
  uint32_t packed[16];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    float z[8], g8[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) z[c] = acc[8 * h + c] + P.b[8 * h + c];
    mpfc_cnn_math::gelu8(z, g8);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      __nv_bfloat162 v2 = __floats2bfloat162_rn(g8[2 * c], g8[2 * c + 1]);
      packed[4 * h + c] = *reinterpret_cast<uint32_t*>(&v2);
    }
  }
  uint4* dst = reinterpret_cast<uint4*>(act + ((size_t)y * m + x) * 32);
#pragma unroll
  for (int q = 0; q < 4; ++q) dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
}

// Last layer of the inference: the 32 -> 1 convolution of the bf16 activations (a tile
// with its periodic halo staged in shared memory by 16-byte asynchronous copies, 80
// bytes per pixel so that a warp's 16-byte reads of consecutive pixels fall in
// distinct banks), FP32 multiply-adds with the bf16 weights, bias, and the result
// scaled back and added to the FP64 field: phi0 += sy (acc + b).
constexpr int kGS = 40;   // staged pixel stride (bf16)
__global__ void __launch_bounds__(kGX * kGY) k_guess_out(const __grid_constant__ GuessOutArgs P,
                                                         const __nv_bfloat16* __restrict__ act, int m, int n,
                                                         double* __restrict__ phi0) {
  __shared__ __align__(16) __nv_bfloat16 at[kGY + 2][kGX + 2][kGS];
  mpfc::pdl_enter();
  const int x0 = blockIdx.x * kGX, y0 = blockIdx.y * kGY;
  for (int t = threadIdx.x; t < (kGX + 2) * (kGY + 2) * 4; t += kGX * kGY) {
    const int p = t >> 2, c = t & 3;
    const int ty = p / (kGX + 2), tx = p - ty * (kGX + 2);
    const size_t g = (size_t)gwrap(y0 + ty - 1, n) * m + gwrap(x0 + tx - 1, m);
    const unsigned sa = (unsigned)__cvta_generic_to_shared(&at[ty][tx][8 * c]);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(act + g * 32 + 8 * c) : "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int tx = threadIdx.x % kGX, ty = threadIdx.x / kGX;
  const int x = x0 + tx, y = y0 + ty;
  if (x >= m || y >= n) return;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};   // one partial sum per 8-channel chunk
#pragma unroll
  for (int tap = 0; tap < 9; ++tap)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint4 v = *reinterpret_cast<const uint4*>(&at[ty + tap / 3][tx + tap % 3][8 * c]);
      const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float lo = __uint_as_float(u[j] << 16), hi = __uint_as_float(u[j] & 0xFFFF0000u);
        acc[c] = fmaf(lo, P.w[tap][8 * c + 2 * j], acc[c]);
        acc[c] = fmaf(hi, P.w[tap][8 * c + 2 * j + 1], acc[c]);
      }
    }
  const float out = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + P.b;
  phi0[(size_t)y * m + x] += P.scale * (double)out;
}

// Host-side rounding to bf16, nearest even (the weights are finite).
float host_bf16(float v) {
  uint32_t u;
  memcpy(&u, &v, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

// The whole inference on the handle's state, its scaled output added to `phi0`.
void enqueue_guess_network(mpfc_s* H, double* phi0, cudaStream_t s) {
  const MpfcGuess& g = H->guess;
  const int m = H->p.m, n = H->p.n;
  const dim3 grid((m + kGX - 1) / kGX, (n + kGY - 1) / kGY), blk(kGX * kGY);
  mpfc_cnn_mean(H->phik, (long long)m * n, g.mean, s);
  mpfc_launch(H->shape, k_guess_in, grid, blk, 0, s, g.in_args, (const double*)H->phik, (const double*)H->phikm1,
              (const double*)g.phikm2, (const double*)g.mean, m, n, (__nv_bfloat16*)g.act[0]);
  // the 32 -> 32 layers (GELU, bf16 out): tcgen05 where the width allows, else mma.sync;
  // layer biases follow each layer's weights in the parameter blob
  size_t off = 4 + 9 * 3 * 32 + 32;
  for (int l = 1; l < 4; ++l) {
    const float* bias = g.params + off + 9 * 32 * 32;
    mpfc_cnn_conv_layer(g.act[(l - 1) & 1], n, m, 32, g.wk[l], bias, 32, g.act[l & 1], s);
    off += 9 * 32 * 32 + 32;
  }
  mpfc_launch(H->shape, k_guess_out, grid, blk, 0, s, g.out_args, (const __nv_bfloat16*)g.act[1], m, n, phi0);
}
}  // namespace

size_t mpfc_guess_carve(mpfc_s* H, const mpfc_params* p, size_t* off, char* base) {
  if (p->guess != MPFC_GUESS_LEARNED) return 0;
  size_t start = *off;
  auto take = [&](size_t bytes) -> char* {
    char* ptr = base ? base + *off : nullptr;
    *off = (*off + bytes + 255) & ~(size_t)255;
    return ptr;
  };
  size_t G = (size_t)p->m * p->n;
  MpfcGuess g;
  g.params = (float*)take(sizeof(float) * MPFC_CNN_PARAM_COUNT);
  for (int l = 0; l < 5; ++l) g.wk[l] = take(2 * (size_t)kLayers[l][3] * kpad_of(kLayers[l][2]));
  g.act[0] = take(2 * G * 32);
  g.act[1] = take(2 * G * 32);
  g.phikm2 = (double*)take(sizeof(double) * G);
  g.mean = (double*)take(sizeof(double) * 129);
  g.loaded = false;
  if (H && base) H->guess = g;
  return *off - start;
}

bool mpfc_has_guess_model(const mpfc_s* H) { return H && H->p.guess == MPFC_GUESS_LEARNED && H->guess.loaded; }

void mpfc_enqueue_learned_guess(mpfc_s* H, cudaStream_t s) { enqueue_guess_network(H, H->lev[0].phi, s); }

extern "C" int mpfc_set_guess_model(mpfc_t* H, const float* params, size_t count) {
  if (!H || !params || count != MPFC_CNN_PARAM_COUNT || H->p.guess != MPFC_GUESS_LEARNED) return MPFC_ERR_INVALID;
  cudaStream_t s = H->stream;
  cudaError_t e = cudaMemcpyAsync(H->guess.params, params, sizeof(float) * count, cudaMemcpyDefault, s);
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "guess params", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  size_t off = 4;
  for (int l = 0; l < 5; ++l) {
    int rc = mpfc_cnn_pack_weights(H->guess.params + off, kLayers[l][0], kLayers[l][1], kLayers[l][2],
                                   kLayers[l][3], 0, H->guess.wk[l], s);
    if (rc != MPFC_OK) return rc;
    off += 9 * (size_t)kLayers[l][0] * kLayers[l][1] + kLayers[l][1];
  }
  std::vector<float> blob(count);
  e = cudaMemcpyAsync(blob.data(), H->guess.params, sizeof(float) * count, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "guess pack", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  MpfcGuess& g = H->guess;
  for (int i = 0; i < 4; ++i) g.norms_host[i] = blob[i];
  // first and last layers as kernel arguments (bf16-rounded weights, as the network
  // computes with them; the normalisation as in the training features)
  const float* w1 = blob.data() + 4;
  for (int k = 0; k < 27; ++k)
    for (int co = 0; co < 32; ++co) g.in_args.w[k][co] = host_bf16(w1[k * 32 + co]);
  for (int co = 0; co < 32; ++co) g.in_args.b[co] = w1[27 * 32 + co];
  for (int i = 0; i < 3; ++i) g.in_args.inv[i] = 1.0 / (double)blob[i];
  const float* w5 = blob.data() + count - (9 * 32 + 1);
  for (int k = 0; k < 9; ++k)
    for (int ci = 0; ci < 32; ++ci) g.out_args.w[k][ci] = host_bf16(w5[k * 32 + ci]);
  g.out_args.b = w5[9 * 32];
  g.out_args.scale = (double)blob[3];
  // step graphs bake the first and last layers into kernel arguments: rebuild them
  mpfc_drop_graphs(H);
  H->guess.loaded = true;
  return MPFC_OK;
}

extern "C" int mpfc_op_learned_guess(mpfc_t* H) {
  if (!mpfc_has_guess_model(H)) return MPFC_ERR_INVALID;
  mpfc_enqueue_learned_guess(H, H->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "learned guess", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  return MPFC_OK;
}

extern "C" int mpfc_guess_correction(mpfc_t* H, double* d_out) {
  if (!mpfc_has_guess_model(H) || !d_out) return MPFC_ERR_INVALID;
  cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(double) * (size_t)H->p.m * H->p.n, H->stream);
  if (e == cudaSuccess) {
    enqueue_guess_network(H, d_out, H->stream);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "learned guess correction", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  return MPFC_OK;
}
