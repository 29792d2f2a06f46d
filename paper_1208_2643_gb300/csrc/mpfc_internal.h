// Internal handle layout of libmpfc, shared by the translation units of the CUDA path.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "../../include/mpfc.h"
#include "mpfc_common.cuh"

// FP32 copy of one level for the inner V-cycles of the mixed-precision form.
struct Lev32 {
  int m, n;
  int nyn;                   // homogeneous Neumann in y (ghost row = boundary row), 0: periodic
  float h;
  float *ephi, *emu, *eka;   // correction e = (e_phi, e_mu, e_kappa)
  float *r1, *r2, *r3;       // source of the correction equation (restricted defect)
  float* q;                  // gam + g'(phi) of the FP64 iterate, restricted
  float *xphi, *xmu, *xka;   // second copy of e for out-of-place sweeps (nullptr: none)
};

// Inference-kernel arguments of the learned guess's first and last layers: the
// weights, rounded to bf16 as the network computes with them, travel as kernel
// parameters, so the multiply-adds read them from the constant bank.
struct GuessInArgs {
  float w[27][32];   // [tap * 3 + channel][output channel]
  float b[32];
  double inv[3];     // 1 / (s0, s1, s2), the input normalisation
};
struct GuessOutArgs {
  float w[9][32];    // [tap][input channel]
  float b;
  double scale;      // sy: the output's scale back to phi
};

// Learned-guess buffers in the workspace (MPFC_GUESS_LEARNED).
struct MpfcGuess {
  float* params = nullptr;     // fp32 model blob (normalisation, weights, biases)
  void* wk[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // packed bf16 weights
  void* act[2] = {nullptr, nullptr};   // activations, bf16 [m*n][32]
  double* phikm2 = nullptr;    // phi^{k-2}
  double* mean = nullptr;
  float norms_host[4] = {1.f, 1.f, 1.f, 1.f};   // host copy of the normalisation scales
  GuessInArgs in_args;         // first layer (with the input features), host copy
  GuessOutArgs out_args;       // last layer, host copy
  bool loaded = false;
};

// Launch shapes of the per-cell kernels of the FP64 time step (mpfc_set_launch_shape).
struct mpfc_launch_shape {
  int rows;          // blocks of 32 x rows threads for launches of at least small_cells cells
  int small_cells;   // smaller launches: one-warp blocks (32 x 1), spread over the SMs
  int pdl_blocks;    // programmatic dependent launch for grids of at most this many blocks
  int tail_cells;    // levels of at most this many cells run in one cluster launch (0: none)
  int tail_ctas;     // CTAs of that cluster (8, or 16 where the GPU allows it)
  int split_cells;   // FP64 transfers onto or from fine levels of at most this many cells:
                     // four threads per coarse cell (restriction), one per fine cell (prolongation)
};

struct mpfc_s {
  mpfc_params p;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t body_stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int nlev = 0;
  mpfc::Lev lev[mpfc::kMaxLevels];
  mpfc::Coef coef[2][mpfc::kMaxLevels];
  mpfc::Coef coefb[2][mpfc::kMaxLevels];   // cell systems of Neumann boundary rows (3 neighbours)
  double* phik = nullptr;
  double* phikm1 = nullptr;
  double* psik = nullptr;
  mpfc::Ctl* ctl = nullptr;
  double* partials = nullptr;
  double* bpart = nullptr;   // per-warp residual sums of the finest level's last half sweep
  int nbpart = 0;
  // learned guess (FP64 handles): the network corrects the extrapolated guess only when
  // that guess's scaled residual is at least guess_gate (0: on every step)
  double guess_gate = 0.0;
  mpfc::StepRecord* info = nullptr;
  float* K3[2] = {nullptr, nullptr};    // coarsest grid, per scheme: I - c theta L^3 then c L (FP32)
  double* px[mpfc::kMaxLevels];
  double* pf[mpfc::kMaxLevels];
  cudaGraphExec_t exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaGraphConditionalHandle cur_handle = 0;   // handle of the graph being captured
  int launch_mode = MPFC_LAUNCH_GRAPH;
  // set by mpfc_create from the precision (mpfc_default_launch_shape)
  mpfc_launch_shape shape = {1, 0, 0, 0, 8};
  // mixed precision
  Lev32 lev32[mpfc::kMaxLevels];
  float* K3f[2] = {nullptr, nullptr};
  int sweep_tile_rows = 16;                     // FP32 one-launch sweeps: tile height (0: two launches per sweep)
  long long sweep_tile_cells = 2048LL * 2048;   // ... on levels of at least this many cells
  int outer_max = 0;
  // learned initial guess
  MpfcGuess guess;
  // pinning (Sec. 4.6): weight per level and the finest-level target, carved when
  // p.pinning; active once mpfc_set_pinning gave a weight
  double* pinW[mpfc::kMaxLevels] = {};
  double* pinhat = nullptr;
  int pin_active = 0;
};

// Block shape of the per-cell V-cycle kernels on an X x Y launch.  GB300's FP64 unit
// is narrow: a warp-wide FP64 instruction takes about 64 cycles whatever the number of
// active lanes, and an SM saturates at about four warps issuing FP64.  A half sweep of
// ~33 FP64 instructions per cell therefore costs ~1 us per warp however few cells it
// has, so small launches use one-warp blocks spread over as many SMs as possible, and
// large ones blocks of 32 x rows threads (the grid then also balances over the SMs in
// finer steps).
inline dim3 mpfc_blk_for(const mpfc_launch_shape& sh, int X, int Y) {
  if ((long long)X * Y >= sh.small_cells) return dim3(32, sh.rows);
  return dim3(X < 32 ? X : 32, 1);
}
inline dim3 mpfc_grid_of(const mpfc_launch_shape& sh, int X, int Y) {
  dim3 b = mpfc_blk_for(sh, X, Y);
  return dim3((X + b.x - 1) / b.x, (Y + b.y - 1) / b.y);
}

// Launch on s, with programmatic stream serialization when the grid has at most
// sh.pdl_blocks blocks: the kernel may then be scheduled while its predecessor still
// runs and waits for it in pdl_enter() (every kernel of the time step starts with that
// call), which overlaps the launch latency of the chain of small kernels that a
// V-cycle is.  A launch error is left for cudaGetLastError.
template <typename... KArgs, typename... Args>
inline void mpfc_launch(const mpfc_launch_shape& sh, void (*kern)(KArgs...), dim3 g, dim3 b, size_t smem,
                        cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = ((long long)g.x * g.y * g.z <= sh.pdl_blocks) ? 1 : 0;
  (void)cudaLaunchKernelEx(&cfg, kern, args...);
}

// NVTX range for profiler timelines (a no-op unless a tool is attached): a time step
// around its graph launch; in MPFC_LAUNCH_STREAM mode also each V-cycle and each
// level's launches, which then show the device work they enqueue.
struct MpfcRange {
  explicit MpfcRange(const char* name) { nvtxRangePushA(name); }
  ~MpfcRange() { nvtxRangePop(); }
  MpfcRange(const MpfcRange&) = delete;
  MpfcRange& operator=(const MpfcRange&) = delete;
};
// "level 0" .. "level 15" (static names for the per-level ranges)
const char* mpfc_level_name(int l);

void mpfc_set_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void mpfc_drop_graphs(mpfc_s* H);
int mpfc_num_levels(int m, int n, int coarsest);
mpfc::Coef mpfc_coef(const mpfc_params* p, int scheme, double h, int nb);
void mpfc_build_K3(const mpfc::Lev& C, const mpfc::Coef& k, std::vector<double>& K3);
void mpfc_coarse_block(const mpfc::Lev& C, const mpfc::Coef& k, std::vector<float>& out);
int mpfc_reduce_blocks(size_t G);
int mpfc_tail_max_ctas();
mpfc_launch_shape mpfc_default_launch_shape(int precision);
void mpfc_abort_capture(cudaStream_t s);
int mpfc_capture_while(mpfc_s* H, cudaStream_t cs, cudaGraphConditionalHandle hnd,
                       void (*body_fn)(mpfc_s*, int, cudaStream_t), int scheme);
// The same for a conditional node of any type (IF for the learned guess's gate).
int mpfc_capture_conditional(mpfc_s* H, cudaStream_t cs, cudaGraphConditionalHandle hnd, cudaGraphConditionalNodeType type,
                             void (*body_fn)(mpfc_s*, int, cudaStream_t), int scheme);
void mpfc_enqueue_prologue(mpfc_s* H, int scheme, cudaStream_t s);
void mpfc_enqueue_commit(mpfc_s* H, int scheme, cudaStream_t s);

// mixed-precision form (fp32_inner.cu)
size_t mpfc_fp32_carve(mpfc_s* H, const mpfc_params* p, size_t* off, char* base, int nlev);
int mpfc_fp32_init(mpfc_s* H);
void mpfc_fp32_destroy(mpfc_s* H);
int mpfc_fp32_enqueue_step(mpfc_s* H, int scheme, cudaStream_t cs, cudaGraphConditionalHandle hnd);
int mpfc_fp32_step_stream(mpfc_s* H, int scheme);
int mpfc_host_continue(const mpfc::Ctl* c);

// learned initial guess (guess_cnn.cu, cnn.cu)
void mpfc_cnn_mean(const double* phik, long long G, double* means, cudaStream_t s);
size_t mpfc_guess_carve(mpfc_s* H, const mpfc_params* p, size_t* off, char* base);
bool mpfc_has_guess_model(const mpfc_s* H);
void mpfc_enqueue_learned_guess(mpfc_s* H, cudaStream_t s);
