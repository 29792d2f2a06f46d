// Learned initial guess inside the solver (MPFC_GUESS_LEARNED): before each step's
// V-cycles, the network of mpfc_cnn.h predicts the error of the linear extrapolation
// from phi^k, phi^{k-1}, phi^{k-2}, and its output, scaled back, is added to the
// extrapolated phi^(0).  mu^(0), kappa^(0) then follow from phi^(0) as for the other
// guesses, and the V-cycles run to the same tolerance.
#include <cuda_bf16.h>
#include <string.h>

#include "../../include/mpfc.h"
#include "../../include/mpfc_cnn.h"
#include "mpfc_internal.h"

int mpfc_cnn_conv_guess(const void* x, int H, int W, int cin_p, const void* wk, const float* bias, double* phi0,
                        double scale, cudaStream_t s);
int mpfc_cnn_conv_layer(const void* x, int H, int W, int cin_p, const void* wk, const float* bias, int cout,
                        void* y_bf16, cudaStream_t s);

namespace {
// (cin, cout, cin_p, cout_p) of the five layers
const int kLayers[5][4] = {{3, 32, 4, 32}, {32, 32, 32, 32}, {32, 32, 32, 32}, {32, 32, 32, 32}, {32, 1, 32, 8}};
int kpad_of(int cin_p) { return (9 * cin_p + 15) / 16 * 16; }
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
  g.x = take(2 * G * 4);
  g.act[0] = take(2 * G * 32);
  g.act[1] = take(2 * G * 32);
  g.phikm2 = (double*)take(sizeof(double) * G);
  g.mean = (double*)take(sizeof(double) * 129);
  g.loaded = false;
  if (H && base) H->guess = g;
  return *off - start;
}

bool mpfc_has_guess_model(const mpfc_s* H) { return H && H->p.guess == MPFC_GUESS_LEARNED && H->guess.loaded; }

void mpfc_enqueue_learned_guess(mpfc_s* H, cudaStream_t s) {
  const MpfcGuess& g = H->guess;
  const int m = H->p.m, n = H->p.n;
  const float* prm = g.params;
  mpfc_cnn_features(H->phik, H->phikm1, g.phikm2, nullptr, 1, n, m, prm, g.mean, g.x, nullptr, s);
  // layer biases follow each layer's weights in the parameter blob
  size_t off = 4;
  const void* in = g.x;
  int cin_p = 4;
  for (int l = 0; l < 4; ++l) {
    size_t wcount = 9 * (size_t)kLayers[l][0] * kLayers[l][1];
    const float* bias = prm + off + wcount;
    mpfc_cnn_conv_layer(in, n, m, cin_p, g.wk[l], bias, kLayers[l][1], g.act[l & 1], s);
    off += wcount + kLayers[l][1];
    in = g.act[l & 1];
    cin_p = 32;
  }
  const float* bias5 = prm + off + 9 * 32;
  mpfc_cnn_conv_guess(in, n, m, 32, g.wk[4], bias5, H->lev[0].phi, (double)g.norms_host[3], s);
}

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
  e = cudaMemcpyAsync(H->guess.norms_host, H->guess.params, sizeof(float) * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "guess pack", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  // step graphs bake the output scale into a kernel argument: rebuild them
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
