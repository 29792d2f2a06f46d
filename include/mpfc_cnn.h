/*
 * mpfc_cnn.h -- kernels of the learned initial guess (no counterpart in the paper:
 * the paper starts each step's multigrid solve from the previous state).
 *
 * A 5-layer periodic 3x3 CNN (3 -> 32 -> 32 -> 32 -> 32 -> 1 channels, GELU after the
 * first four) maps the last three fields phi^k, phi^{k-1}, phi^{k-2} to the error of
 * the linear extrapolation 2 phi^k - phi^{k-1} of phi^{k+1}.  The solver adds the
 * prediction to its initial guess (MPFC_GUESS_LEARNED) and still iterates to the full
 * tolerance, so the network only changes how many V-cycles a step takes.
 *
 * Tensors: NHWC, bf16 activations with channels padded to cin_p / cout_p, fp32
 * gradients and master weights, fp64 fields; images are periodic.  FP32 master
 * weights of a layer are [tap][c_in][c_out] with tap = (dy+1)*3 + (dx+1) and the
 * output at p summing w[tap][ci][co] * x[p + (dy, dx)][ci]; the kernels use packed
 * bf16 copies made by mpfc_cnn_pack_weights.  All calls are asynchronous on `stream`
 * (a cudaStream_t) and return 0 or a negative MPFC_ERR_* status.
 */
#ifndef MPFC_CNN_H
#define MPFC_CNN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of fp32 values of a model parameter blob: 4 normalisation scales
 * (s0, s1, s2, sy) then, for each layer, weights [9][c_in][c_out] and bias [c_out]. */
#define MPFC_CNN_PARAM_COUNT 28933

/* Network input x (B x H x W x 4 bf16) from three fields per sample (B stacked m*n
 * double arrays) and, if phikp1 and y_f32 are given, the target y (B x H x W fp32);
 * `means` is B * 129 doubles of scratch; its first B entries receive the per-sample
 * means of phi^k (deterministic two-pass reduction). */
int mpfc_cnn_features(const double* phik, const double* phikm1, const double* phikm2, const double* phikp1, int B,
                      int H, int W, const float* norms, double* means, void* x_bf16, float* y_f32, void* stream);

/* Packs fp32 master weights w [9][cin][cout] into the bf16 layout of the forward kernel
 * (transposed = 0: [cout_p][K], K = 9 cin_p rounded up to 16) or of the data-gradient
 * kernel (transposed = 1: taps flipped, channels swapped: [cin_p][9 cout_p rounded]).
 * cin_p, cout_p: padded channel counts (cin_p in {4, 8, 16, 32}; cout_p a multiple of 8,
 * at most 32; for transposed packing cout_p must be in {4, 8, 16, 32}). */
int mpfc_cnn_pack_weights(const float* w, int cin, int cout, int cin_p, int cout_p, int transposed, void* wk,
                          void* stream);

/* Forward periodic 3x3 convolution on BF16 tensor cores (implicit GEMM, FP32
 * accumulation): acc[p][co] = sum_tap,ci x[p + off(tap)][ci] w[tap][ci][co].
 * mode 0: y_bf16 = gelu(acc + bias) (exact-erf GELU) and, if z_f32 is given, the
 * pre-activation acc + bias (fp32, for the backward pass); mode 1: y_f32 = acc + bias.
 * Outputs have cout_p channels (padding channels written as 0). */
int mpfc_cnn_conv_forward(const void* x, int B, int H, int W, int cin_p, const void* wk, const float* bias, int cout,
                          int cout_p, int mode, void* y_bf16, float* y_f32, float* z_f32, void* stream);

/* Data gradient through one layer and the GELU before it, on tensor cores:
 * dzprev[p][ci] = gelu'(z_prev[p][ci]) * sum_tap,co dz[p - off(tap)][co] w[tap][ci][co],
 * with wk_t packed transposed; dz is bf16 with cout_p channels, z_prev fp32 with cin_p.
 * Writes bf16 and fp32 copies of dzprev. */
int mpfc_cnn_conv_backward_data(const void* dz, int B, int H, int W, int cout_p, const void* wk_t, int cin, int cin_p,
                                const float* z_prev, void* dzprev_bf16, float* dzprev_f32, void* stream);

/* Scratch bytes mpfc_cnn_conv_backward_weight needs for a B x H x W batch. */
size_t mpfc_cnn_wgrad_scratch_bytes(int B, int H, int W);

/* Weight and bias gradients on CUDA cores, FP32 accumulation, deterministic (per-chunk
 * partials summed in chunk order): dw[tap][ci][co] = sum_p x[p + off(tap)][ci] dz[p][co],
 * db[co] = sum_p dz[p][co].  x: bf16 with cin_p channels; dz: fp32 with cout_p. */
int mpfc_cnn_conv_backward_weight(const void* x, int B, int H, int W, int cin, int cin_p, const float* dz, int cout,
                                  int cout_p, float* dw, float* db, void* scratch, void* stream);

/* Mean squared error of yhat (channel 0 of an fp32 tensor with `yhat_stride` channels)
 * against y (n values): dy = 2 (yhat - y)/n into channel 0 of dy_f32 / dy_bf16 (stride
 * dy_stride, other channels zeroed); per-block squared-error sums in loss_partials
 * (nblocks <= 4096 entries). */
int mpfc_cnn_mse(const float* yhat, int yhat_stride, const float* y, long long n, float* dy_f32, void* dy_bf16,
                 int dy_stride, float* loss_partials, int nblocks, void* stream);

/* Adam update (Kingma & Ba) of n fp32 parameters at step t >= 1, bias-corrected. */
int mpfc_cnn_adam(float* param, const float* grad, float* m, float* v, int n, float lr, float beta1, float beta2,
                  float eps, int t, void* stream);

/* Chooses the tensor-core path of the 32 -> 32 channel convolutions (forward and data
 * gradient, image width a multiple of 128): 1 = tcgen05 MMAs with the accumulator in
 * tensor memory (default), 0 = warp-level mma.sync.  Other shapes always use mma.sync.
 * Process-wide; applies to convolutions launched, and step graphs captured, afterwards. */
int mpfc_cnn_set_tensor_path(int use_tcgen05);

/* Test hook of the tcgen05 convolution's failure handling (no counterpart in the paper;
 * for tests of the bounded waits without a GPU fault).  withhold = 1: in every following
 * tcgen05 convolution, CTA 0 skips the tensor copy of its first input row (it touches
 * no memory out of bounds), so the MMA issuer's wait on that row runs out after
 * spin_cycles clock cycles; the CTA then stops all its roles, waits (bounded) for the
 * copies and MMAs it already issued, frees its tensor memory and returns, and the launch
 * leaves that CTA's tiles unwritten; mpfc_cnn_tensor_path_status then reports the
 * failure.  withhold = 0, spin_cycles = 0 restore normal operation (waits limited to
 * about 0.1 s).  Process-wide, synchronous.  MPFC_ERR_INVALID for other values. */
int mpfc_cnn_test_withhold_load(int withhold, long long spin_cycles);

/* Reports (and clears) whether a tcgen05 convolution gave up waiting for its MMAs
 * since the last call: MPFC_OK if none did, MPFC_ERR_NOT_CONVERGED if one did (its
 * output is then incomplete), MPFC_ERR_CUDA on a CUDA error.  Synchronous. */
int mpfc_cnn_tensor_path_status(void);

#ifdef __cplusplus
}
#endif

#endif
