// libmpfc: host driver and C ABI (see include/mpfc.h).
//
// A handle carves every device array out of the caller's workspace, builds one
// CUDA graph per scheme for a whole time step (source, guess, a conditional WHILE
// node that runs V-cycles until the device-side residual test fails, and the psi
// update), and replays it once per step.  No host synchronisation happens inside a
// step; the residual test, cycle counting and divergence detection run on the GPU.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "../../include/mpfc.h"
#include "fp64_kernels.cuh"
#include "mpfc_internal.h"

using namespace mpfc;

#define CK(call)                                              \
  do {                                                        \
    cudaError_t err_ = (call);                                \
    if (err_ != cudaSuccess) {                                \
      mpfc_set_cuda_error(err_, #call, __FILE__, __LINE__);   \
      return MPFC_ERR_CUDA;                                   \
    }                                                         \
  } while (0)

// As CK, inside a stream capture: an error first ends the capture on `stream` (see
// mpfc_abort_capture), so that the caller's stream is not left capturing.
#define CKCAP(call, stream)                                   \
  do {                                                        \
    cudaError_t err_ = (call);                                \
    if (err_ != cudaSuccess) {                                \
      mpfc_set_cuda_error(err_, #call, __FILE__, __LINE__);   \
      mpfc_abort_capture(stream);                             \
      return MPFC_ERR_CUDA;                                   \
    }                                                         \
  } while (0)

static char g_last_cuda_error[512];

const char* mpfc_level_name(int l) {
  static const char* const names[kMaxLevels] = {"level 0",  "level 1",  "level 2",  "level 3",  "level 4",  "level 5",
                                                "level 6",  "level 7",  "level 8",  "level 9",  "level 10", "level 11",
                                                "level 12", "level 13", "level 14", "level 15"};
  return (l >= 0 && l < kMaxLevels) ? names[l] : "level";
}

namespace mpfc {
int sm_count() {
  constexpr int kDevs = 64;
  static std::atomic<int> cache[kDevs];   // 0: not queried yet
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  if (dev < kDevs)
    if (int c = cache[dev].load()) return c;
  int c = 0;
  if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c < 1) {
    (void)cudaGetLastError();
    return 1;   // grids stay correct (every sized kernel strides over its work), only smaller
  }
  if (dev < kDevs) cache[dev].store(c);
  return c;
}
}  // namespace mpfc

void mpfc_set_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

extern "C" const char* mpfc_last_cuda_error(void) { return g_last_cuda_error; }

// ---------------------------------------------------------------------------
// Parameters, hierarchy, coefficients
// ---------------------------------------------------------------------------
extern "C" void mpfc_default_params(mpfc_params* p) {
  memset(p, 0, sizeof(*p));
  p->m = 64;
  p->n = 64;
  p->h = 0.5;
  p->M = 1.0;
  p->epsilon = 0.025;
  p->beta = 0.9;
  p->dt = 0.01;
  p->nu1 = 2;
  p->nu2 = 2;
  p->coarsest = 4;
  p->omega = 0.8;
  p->tol = 1e-10;
  p->max_cycles = 100;
  p->precision = MPFC_FP64;
  p->guess = MPFC_GUESS_EXTRAP;
}

// Halve while both sides stay even and keep at least `coarsest` cells.
int mpfc_num_levels(int m, int n, int coarsest) {
  int L = 1;
  while (L < kMaxLevels && m % 2 == 0 && n % 2 == 0 && m / 2 >= coarsest && n / 2 >= coarsest && (m / 2) % 2 == 0 &&
         (n / 2) % 2 == 0) {
    m /= 2;
    n /= 2;
    ++L;
  }
  return L;
}

static bool params_valid(const mpfc_params* p) {
  if (!p) return false;
  if (p->m < 4 || p->n < 4 || p->m % 2 || p->n % 2) return false;
  if (!(p->h > 0) || !(p->M > 0) || !(p->beta >= 0) || !(p->dt > 0) || !(p->epsilon <= 1.0)) return false;
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 < 1 || p->coarsest < 2) return false;
  if (!(p->omega > 0 && p->omega <= 1.0)) return false;
  if (!(p->tol >= 0) || p->max_cycles < 1) return false;
  if (p->precision != MPFC_FP64 && p->precision != MPFC_FP32_INNER) return false;
  if (p->guess < MPFC_GUESS_PREV || p->guess > MPFC_GUESS_LEARNED) return false;
  if (p->inner_cycles < 0 || p->inner_cycles > 64) return false;
  if (p->bc != MPFC_BC_PERIODIC && p->bc != MPFC_BC_NEUMANN_Y) return false;
  if (p->pinning != 0 && p->pinning != 1) return false;
  if (p->model != MPFC_MODEL_MPFC && p->model != MPFC_MODEL_PFC) return false;
  if (p->pinning && p->guess == MPFC_GUESS_LEARNED) return false;
  // the mixed conditions are built for the FP64 and FP32-inner paths with the analytic guesses
  if (p->bc == MPFC_BC_NEUMANN_Y && p->guess == MPFC_GUESS_LEARNED) return false;
  int L = mpfc_num_levels(p->m, p->n, p->coarsest);
  int mc = p->m >> (L - 1), nc = p->n >> (L - 1);
  if (mc * nc > kMaxCoarseCells) return false;
  // the kernels index cells and stride their grid loops in 32-bit ints: at most 2^30
  // cells keeps every index, every cell count and every index-plus-stride below 2^31
  if ((size_t)p->m * (size_t)p->n > ((size_t)1 << 30)) return false;
  // the per-cell launches put the rows on the grid's y dimension (at most 65535 blocks)
  if (p->n > 65535) return false;
  return true;
}

// nb: face neighbours that are not ghosts (4, or 3 next to a Neumann boundary, whose
// ghost is the cell's own unknown and so joins the diagonal).
Coef mpfc_coef(const mpfc_params* p, int scheme, double h, int nb) {
  Coef k;
  double alpha = 1.0 - p->epsilon;
  if (scheme == 1) {
    k.c = p->dt * p->M / (p->beta + 1.0 / p->dt);
    k.gam = alpha;
    k.theta = 1.0;
  } else {
    k.c = p->dt * p->M / (p->beta + 2.0 / p->dt);
    k.gam = 0.5 * alpha;
    k.theta = 0.5;
  }
  if (p->model == MPFC_MODEL_PFC) k.c = p->dt * p->M;   // (phi - phi^k)/s = M Delta_h mu
  k.omega = p->omega;
  double h2 = h * h;
  k.cmu = k.c / h2;
  k.a = nb * k.c / h2;
  k.ih2 = 1.0 / h2;
  k.b = nb / h2;
  k.b3 = nb * k.theta / h2;
  k.th2 = k.theta / h2;
  k.D0 = 1.0 + k.a * k.gam + k.a * k.b * k.b3;
  k.Q0 = k.gam + k.b * k.b3;
  k.a3 = 3.0 * k.a;
  k.omw = 1.0 - k.omega;
  k.D0w = k.D0 / k.omega;
  k.aw = k.a / k.omega;
  k.a3w = k.a3 / k.omega;
  k.relax = (k.omega != 1.0);
  k.pad = 0;
  return k;
}

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carver {
  char* base;
  size_t off;
  template <typename T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off = align256(off + count * sizeof(T));
    return p;
  }
};

// Default gate of the learned guess, as a multiple of the tolerance: on the headline
// workload (1024^2, tol 1e-10) the extrapolated guess needs four or more V-cycles exactly
// when its scaled residual is at least 2.6e-6, and the network's own error floor (a
// scaled residual near 7e-7) still leaves three, so only those steps gain a cycle.
constexpr double kGuessGateTolMultiple = 2.6e4;

// Walks the layout; with base == nullptr only computes the size.
static size_t carve(mpfc_s* H, const mpfc_params* p, char* base) {
  Carver c{base, 0};
  int L = mpfc_num_levels(p->m, p->n, p->coarsest);
  size_t G0 = (size_t)p->m * p->n;
  Ctl* ctl = c.take<Ctl>(1);
  double* partials = c.take<double>((size_t)kMaxSums * kMaxPartials);
  // per-warp residual sums of the finest level's last half sweep (k_smooth_res)
  const int nbpart = ((p->m / 2 + 31) / 32) * p->n;
  double* bpart = c.take<double>((size_t)nbpart);
  StepRecord* info = c.take<StepRecord>(kInfoCap);
  double* phik = c.take<double>(G0);
  double* phikm1 = c.take<double>(G0);
  double* psik = c.take<double>(G0);
  int m = p->m, n = p->n;
  double h = p->h;
  Lev lev[kMaxLevels];
  double *px[kMaxLevels], *pf[kMaxLevels], *pw[kMaxLevels];
  for (int l = 0; l < L; ++l) {
    size_t G = (size_t)m * n;
    Lev& v = lev[l];
    v.m = m;
    v.n = n;
    v.nyn = p->bc == MPFC_BC_NEUMANN_Y;
    v.W = nullptr;
    v.h = h;
    v.phi = c.take<double>(G);
    v.mu = c.take<double>(G);
    v.ka = c.take<double>(G);
    v.S1 = c.take<double>(G);
    v.S2 = c.take<double>(G);
    v.S3 = c.take<double>(G);
    if (l > 0) {
      v.b1 = c.take<double>(G);
      v.b2 = c.take<double>(G);
      v.b3 = c.take<double>(G);
      v.pk = c.take<double>(G);
    } else {
      v.b1 = v.b2 = v.b3 = nullptr;
      v.pk = phik;
    }
    px[l] = c.take<double>(G);
    pf[l] = c.take<double>(G);
    pw[l] = p->pinning ? c.take<double>(G) : nullptr;
    m /= 2;
    n /= 2;
    h *= 2.0;
  }
  double* pinhat = p->pinning ? c.take<double>(G0) : nullptr;
  int Gc = lev[L - 1].m * lev[L - 1].n;
  float* K3a = c.take<float>(2 * (size_t)Gc * Gc);   // K3 and c L of scheme 1 (mpfc_coarse_block)
  float* K3b = c.take<float>(2 * (size_t)Gc * Gc);
  mpfc_fp32_carve(H, p, &c.off, base, L);
  mpfc_guess_carve(H, p, &c.off, base);
  if (H && base) {
    H->nlev = L;
    H->ctl = ctl;
    H->partials = partials;
    H->bpart = bpart;
    H->nbpart = nbpart;
    H->info = info;
    H->phik = phik;
    H->phikm1 = phikm1;
    H->psik = psik;
    for (int l = 0; l < L; ++l) {
      H->lev[l] = lev[l];
      H->px[l] = px[l];
      H->pf[l] = pf[l];
      H->pinW[l] = pw[l];
    }
    H->pinhat = pinhat;
    H->pin_active = 0;
    H->K3[0] = K3a;
    H->K3[1] = K3b;
  }
  return c.off;
}

extern "C" size_t mpfc_workspace_bytes(const mpfc_params* p) {
  if (!params_valid(p)) return 0;
  return carve(nullptr, p, nullptr);
}

// K3 = I - c theta L^3 on the coarsest grid (dense, row-major G x G).
void mpfc_build_K3(const Lev& C, const Coef& k, std::vector<double>& K3) {
  int m = C.m, n = C.n, G = m * n;
  std::vector<double> Lm((size_t)G * G, 0.0), L2((size_t)G * G, 0.0), L3((size_t)G * G, 0.0);
  double ih2 = 1.0 / (C.h * C.h);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) {
      int r = j * m + i;
      Lm[(size_t)r * G + r] -= 4.0 * ih2;
      // a Neumann ghost row is the boundary row itself, which folds it into the diagonal
      int js = C.nyn ? (j > 0 ? j - 1 : 0) : (j + n - 1) % n, jn = C.nyn ? (j < n - 1 ? j + 1 : n - 1) : (j + 1) % n;
      int nb[4] = {j * m + (i + m - 1) % m, j * m + (i + 1) % m, js * m + i, jn * m + i};
      for (int t = 0; t < 4; ++t) Lm[(size_t)r * G + nb[t]] += ih2;
    }
  for (int r = 0; r < G; ++r)
    for (int t = 0; t < G; ++t) {
      double a = Lm[(size_t)r * G + t];
      if (a == 0.0) continue;
      for (int c2 = 0; c2 < G; ++c2) L2[(size_t)r * G + c2] += a * Lm[(size_t)t * G + c2];
    }
  for (int r = 0; r < G; ++r)
    for (int t = 0; t < G; ++t) {
      double a = L2[(size_t)r * G + t];
      if (a == 0.0) continue;
      for (int c2 = 0; c2 < G; ++c2) L3[(size_t)r * G + c2] += a * Lm[(size_t)t * G + c2];
    }
  K3.assign((size_t)G * G, 0.0);
  for (int r = 0; r < G; ++r)
    for (int c2 = 0; c2 < G; ++c2)
      K3[(size_t)r * G + c2] = (r == c2 ? 1.0 : 0.0) - k.c * k.theta * L3[(size_t)r * G + c2];
}

// Default launch shapes, from interleaved timings on GB300 (V-cycle at 1024^2):
//   FP64: one-warp blocks everywhere and programmatic launch only for grids of at most
//     16 blocks (the coarse tail, the coarsest levels' one-warp launches): 341 steps/s
//     at 1024^2 (scheme 1) against 328 with programmatic launch up to 4 x SMs blocks and
//     315 for every grid; 756 against 689 at 512^2, 662 against 613 for scheme 2 at
//     512^2, 111 against 109 at 2048^2; only grids of about 128^2 gain from it (1466
//     against 1501 steps/s there).  (An earlier driver favoured 4 x SMs: 743 against
//     822 us per V-cycle with 32 x 8 blocks and none.)
//   FP32 inner cycles (memory-latency bound, they want occupancy): 32 x 4 blocks and the
//     same programmatic launch, 472 us per outer iteration against 479 (32 x 8, none)
//     and 725 with one-warp blocks;
//   the FP64 levels of at most 16 x 16 cells as one single-CTA launch: 701 us per
//     V-cycle at 1024^2 against 721 without (a 16-CTA cluster: 719; at 64^2: 138, 162,
//     155); larger tails were slower, their phases being bound by the FP64 instruction
//     latency of the cell updates, not by launches;
//   the FP32 inner cycles' levels of at most 32 x 32 cells in one CTA with the levels in
//     shared memory: 430 us per outer iteration at 1024^2 against 475 (64 x 64: 457).
mpfc_launch_shape mpfc_default_launch_shape(int precision) {
  if (precision == MPFC_FP32_INNER) return mpfc_launch_shape{4, 0, 4 * mpfc::sm_count(), 32 * 32, 1, 0};
  // split transfers up to 256^2 fine cells: 2.917 against 2.975 ms per step at 1024^2
  // (0: 2.975, 64^2: 2.934, 128^2: 2.920, 512^2: 2.962, 1024^2: 3.160); with them,
  // programmatic launch up to 128 blocks (the split kernels' grids on levels up to 64^2):
  // 2.916 against 2.926 ms with 16 blocks, 3.003 with 256 (the 128^2 sweeps), and 1.853
  // against 1.864 ms for scheme 2 at 512^2; tails from 8^2 and 32^2 stay slower
  return mpfc_launch_shape{1, 0, 128, 256, 1, 256 * 256};
}

// The coarsest grid's matrices for one scheme as the FP32 block the coarse solves read:
// K3 = I - c theta L^3 (G x G, row-major), then c L (G x G), L the five-point Laplacian
// with the level's boundary rule.
void mpfc_coarse_block(const Lev& C, const Coef& k, std::vector<float>& out) {
  std::vector<double> K3;
  mpfc_build_K3(C, k, K3);
  const int m = C.m, n = C.n, G = m * n;
  const double ih2 = 1.0 / (C.h * C.h);
  std::vector<double> cL((size_t)G * G, 0.0);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) {
      const int r = j * m + i;
      cL[(size_t)r * G + r] -= 4.0 * k.c * ih2;
      const int js = C.nyn ? (j > 0 ? j - 1 : 0) : (j + n - 1) % n, jn = C.nyn ? (j < n - 1 ? j + 1 : n - 1) : (j + 1) % n;
      const int nb[4] = {j * m + (i + m - 1) % m, j * m + (i + 1) % m, js * m + i, jn * m + i};
      for (int t = 0; t < 4; ++t) cL[(size_t)r * G + nb[t]] += k.c * ih2;
    }
  out.assign(K3.begin(), K3.end());
  out.insert(out.end(), cL.begin(), cL.end());
}

extern "C" int mpfc_create(const mpfc_params* p, void* d_workspace, size_t bytes, void* cuda_stream, mpfc_t** out) {
  if (!out) return MPFC_ERR_INVALID;
  *out = nullptr;
  if (!params_valid(p)) return MPFC_ERR_INVALID;
  size_t need = carve(nullptr, p, nullptr);
  if (!d_workspace || bytes < need || ((uintptr_t)d_workspace & 255)) return MPFC_ERR_WORKSPACE;
  mpfc_s* H = new mpfc_s();
  H->p = *p;
  H->shape = mpfc_default_launch_shape(p->precision);
  H->guess_gate = kGuessGateTolMultiple * p->tol;
  H->stream = (cudaStream_t)cuda_stream;
  H->ws = (char*)d_workspace;
  H->ws_bytes = bytes;
  carve(H, p, (char*)d_workspace);
  for (int s = 0; s < 2; ++s)
    for (int l = 0; l < H->nlev; ++l) {
      H->coef[s][l] = mpfc_coef(p, s + 1, H->lev[l].h, 4);
      H->coefb[s][l] = mpfc_coef(p, s + 1, H->lev[l].h, 3);
    }
  int rc = MPFC_OK;
  do {
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&H->body_stream, cudaStreamNonBlocking)) != cudaSuccess) {
      mpfc_set_cuda_error(e, "cudaStreamCreate", __FILE__, __LINE__);
      rc = MPFC_ERR_CUDA;
      break;
    }
    Ctl c0;
    memset(&c0, 0, sizeof(c0));
    c0.tol = p->tol;
    c0.max_cycles = p->max_cycles;
    size_t G0 = (size_t)p->m * p->n;
    const Lev& C = H->lev[H->nlev - 1];
    if ((e = cudaMemcpyAsync(H->ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, H->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(H->phik, 0, G0 * sizeof(double), H->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(H->phikm1, 0, G0 * sizeof(double), H->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(H->psik, 0, G0 * sizeof(double), H->stream)) != cudaSuccess) {
      mpfc_set_cuda_error(e, "initialise workspace", __FILE__, __LINE__);
      rc = MPFC_ERR_CUDA;
      break;
    }
    for (int s = 0; s < 2 && rc == MPFC_OK; ++s) {
      std::vector<float> K3f;
      mpfc_coarse_block(C, H->coef[s][H->nlev - 1], K3f);
      if ((e = cudaMemcpyAsync(H->K3[s], K3f.data(), K3f.size() * sizeof(float), cudaMemcpyHostToDevice, H->stream)) !=
              cudaSuccess ||
          (e = cudaStreamSynchronize(H->stream)) != cudaSuccess) {
        mpfc_set_cuda_error(e, "upload coarse matrix", __FILE__, __LINE__);
        rc = MPFC_ERR_CUDA;
      }
    }
    if (rc == MPFC_OK) rc = mpfc_fp32_init(H);
  } while (0);
  if (rc != MPFC_OK) {
    mpfc_destroy(H);
    return rc;
  }
  *out = H;
  return MPFC_OK;
}

void mpfc_drop_graphs(mpfc_s* H) {
  for (int s = 0; s < 2; ++s)
    for (int v = 0; v < 2; ++v)
      if (H->exec[s][v]) {
        cudaGraphExecDestroy(H->exec[s][v]);
        H->exec[s][v] = nullptr;
      }
}

extern "C" void mpfc_destroy(mpfc_t* H) {
  if (!H) return;
  mpfc_drop_graphs(H);
  mpfc_fp32_destroy(H);
  if (H->cap_stream) cudaStreamDestroy(H->cap_stream);
  if (H->body_stream) cudaStreamDestroy(H->body_stream);
  delete H;
}

extern "C" int mpfc_levels(const mpfc_t* H) { return H ? H->nlev : 0; }

extern "C" int mpfc_level_size(const mpfc_t* H, int level, int* m, int* n, double* hl) {
  if (!H || level < 0 || level >= H->nlev) return MPFC_ERR_INVALID;
  if (m) *m = H->lev[level].m;
  if (n) *n = H->lev[level].n;
  if (hl) *hl = H->lev[level].h;
  return MPFC_OK;
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
static dim3 grid_for(int X, int Y, dim3 b) { return dim3((X + b.x - 1) / b.x, (Y + b.y - 1) / b.y); }
static const dim3 kBlk2d(32, 8);

int mpfc_reduce_blocks(size_t G) {
  size_t b = (G + 255) / 256;
  if (b > (size_t)kMaxPartials) b = kMaxPartials;
  if (b < 1) b = 1;
  return (int)b;
}

// `sweeps` red-black sweeps; with bpart, the last half sweep is k_smooth_res, which also
// leaves the residual sums of the cells it updates (the finest level's last sweep).
template <int SCH>
static void launch_smooth(const mpfc_launch_shape& sh, const Lev& L, const Coef& k, const Coef& kb, int sweeps,
                          cudaStream_t s, double* bpart = nullptr) {
  dim3 b = mpfc_blk_for(sh, L.m / 2, L.n), g = mpfc_grid_of(sh, L.m / 2, L.n);
  for (int sw = 0; sw < sweeps; ++sw) {
    mpfc_launch(sh, k_smooth<SCH>, g, b, 0, s, L, k, kb, 0);
    if (bpart && sw == sweeps - 1)
      mpfc_launch(sh, k_smooth_res<SCH>, dim3((L.m / 2 + 31) / 32, L.n), dim3(32), 0, s, L, k, kb, bpart);
    else
      mpfc_launch(sh, k_smooth<SCH>, g, b, 0, s, L, k, kb, 1);
  }
}

static size_t coarse_smem(const Lev& C) {
  int G = C.m * C.n;
  return sizeof(double) * 7 * (size_t)G + sizeof(float) * ((size_t)G * (G + 1) + (size_t)G);
}

// Largest tail cluster this GPU runs: 16 CTAs where a non-portable cluster of that size
// can be resident (one query, then cached), else the portable 8.
int mpfc_tail_max_ctas() {
  static std::atomic<int> cached{0};   // 0: not queried yet (concurrent first calls agree)
  if (int c = cached.load()) return c;
  int best = 8;
  if (cudaFuncSetAttribute(k_tail<1, kLdL2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(k_tail<2, kLdL2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = coarse_smem(Lev{8, 8});
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = 16;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_tail<1, kLdL2>, &cfg) == cudaSuccess && n > 0) best = 16;
  }
  (void)cudaGetLastError();
  cached.store(best);
  return best;
}

template <int SCH>
static void launch_coarse(mpfc_s* H, const Lev& C, const Coef& k, cudaStream_t s) {
  mpfc_launch(H->shape, k_coarse_solve<SCH>, dim3(1), dim3(32), coarse_smem(C), s, C, k, (const float*)H->K3[SCH - 1]);
}

// First level run by the tail kernel: the finest level of at most shape.tail_cells
// cells, leaving at least one level above the coarsest and at most kMaxTail levels in
// the tail; nlev when no tail is used.
static int tail_first_level(const mpfc_s* H) {
  const int L = H->nlev;
  if (H->shape.tail_cells <= 0 || L < 2) return L;
  int lt = L - 1;
  while (lt > 0 && (long long)H->lev[lt - 1].m * H->lev[lt - 1].n <= H->shape.tail_cells) --lt;
  if (lt > L - 2) return L;
  if (L - lt > kMaxTail) lt = L - kMaxTail;
  return lt;
}

// Whether a V-cycle ends with k_smooth_res on the finest level (which then runs by
// per-level launches and has post-sweeps), so that its residual test is k_resnorm_red.
static bool vcycle_fuses_norm(const mpfc_s* H) {
  const int L = H->nlev, lt = tail_first_level(H);
  const int down = lt < L ? lt : L - 1;
  return down >= 1 && H->p.nu2 >= 1;
}

// Levels lt .. nlev-1 as one launch (k_tail): one CTA, or a cluster of tail_ctas CTAs.
template <int SCH>
static void launch_tail(mpfc_s* H, int lt, cudaStream_t s) {
  TailArgs A;
  A.nlev = H->nlev - lt;
  A.nu1 = H->p.nu1;
  A.nu2 = H->p.nu2;
  A.K3f = H->K3[SCH - 1];
  for (int i = 0; i < A.nlev; ++i) {
    A.lv[i].L = H->lev[lt + i];
    A.lv[i].k = H->coef[SCH - 1][lt + i];
    A.lv[i].kb = H->coefb[SCH - 1][lt + i];
  }
  const int nc = H->shape.tail_ctas;
  const size_t smem = coarse_smem(H->lev[H->nlev - 1]);
  if (nc == 1) {   // one CTA: __syncthreads between the phases, plain (L1) loads
    mpfc_launch(H->shape, k_tail<SCH, kLdPlain>, dim3(1), dim3(kTailThreads), smem, s, A);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = nc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = (nc <= H->shape.pdl_blocks) ? 2 : 1;
  (void)cudaLaunchKernelEx(&cfg, k_tail<SCH, kLdL2>, A);
}

template <int SCH>
static void enqueue_vcycle(mpfc_s* H, cudaStream_t s) {
  const mpfc_params& p = H->p;
  const mpfc_launch_shape& sh = H->shape;
  const int L = H->nlev;
  const int lt = tail_first_level(H);
  const int down = lt < L ? lt : L - 1;   // levels smoothed and restricted by per-level launches
  for (int l = 0; l < down; ++l) {
    MpfcRange range(mpfc_level_name(l));
    const Lev& F = H->lev[l];
    const Lev& C = H->lev[l + 1];
    launch_smooth<SCH>(sh, F, H->coef[SCH - 1][l], H->coefb[SCH - 1][l], p.nu1, s);
    if ((long long)F.m * F.n <= sh.split_cells)
      mpfc_launch(sh, k_resid_restrict4<SCH>, dim3((4 * C.m + 31) / 32, C.n), dim3(32), 0, s, F, C,
                  H->coef[SCH - 1][l], 1);
    else
      mpfc_launch(sh, k_resid_restrict<SCH>, mpfc_grid_of(sh, C.m, C.n), mpfc_blk_for(sh, C.m, C.n), 0, s, F, C,
                  H->coef[SCH - 1][l], 1);
    mpfc_launch(sh, k_tau<SCH>, mpfc_grid_of(sh, C.m, C.n), mpfc_blk_for(sh, C.m, C.n), 0, s, C, H->coef[SCH - 1][l + 1]);
  }
  {
    MpfcRange range(lt < L ? "coarse tail" : "coarsest solve");
    if (lt < L) launch_tail<SCH>(H, lt, s);
    else launch_coarse<SCH>(H, H->lev[L - 1], H->coef[SCH - 1][L - 1], s);
  }
  for (int l = down - 1; l >= 0; --l) {
    MpfcRange range(mpfc_level_name(l));
    const Lev& F = H->lev[l];
    const Lev& C = H->lev[l + 1];
    ProlongArgs A{C.phi, C.mu, C.ka, C.b1, C.b2, C.b3, F.phi, F.mu, F.ka, C.m, C.n, C.nyn};
    if ((long long)F.m * F.n <= sh.split_cells)
      mpfc_launch(sh, k_prolong_fine, mpfc_grid_of(sh, F.m, F.n), mpfc_blk_for(sh, F.m, F.n), 0, s, A);
    else
      mpfc_launch(sh, k_prolong, grid_for(C.m, C.n, kBlk2d), kBlk2d, 0, s, A);
    launch_smooth<SCH>(sh, F, H->coef[SCH - 1][l], H->coefb[SCH - 1][l], p.nu2, s,
                       (l == 0 && vcycle_fuses_norm(H)) ? H->bpart : nullptr);
  }
}

// The learned guess's gate: sets the condition of the step graph's IF node that holds
// the network's correction from the scaled residual of the extrapolated guess.
__global__ void k_guess_gate(const Ctl* ctl, double threshold, cudaGraphConditionalHandle h) {
  pdl_enter();
  if (threadIdx.x == 0) cudaGraphSetConditional(h, (ctl->status == 0 && ctl->res0 >= threshold) ? 1u : 0u);
}

// Whether the step runs the learned guess behind its gate (FP64 handles).
static bool guess_gated(const mpfc_s* H) {
  return H->p.guess == MPFC_GUESS_LEARNED && H->p.precision == MPFC_FP64 && H->guess_gate > 0.0;
}

// The prologue: source and extrapolated guess; with `network`, the learned correction
// of the guess (always, where no gate decides); then kappa and mu consistent with phi.
template <int SCH>
static void enqueue_prologue(mpfc_s* H, cudaStream_t s, bool network = true) {
  const mpfc_params& p = H->p;
  const Lev& L0 = H->lev[0];
  mpfc_launch(H->shape, k_step_begin, dim3(1), dim3(32), 0, s, H->ctl);
  SourceArgs A;
  A.phik = H->phik;
  A.phikm1 = H->phikm1;
  A.psik = H->psik;
  A.psi_coef = (p.model == MPFC_MODEL_PFC) ? 0.0 : (SCH == 1) ? 1.0 / (p.beta + 1.0 / p.dt) : 2.0 / (p.beta + 2.0 / p.dt);
  A.half_alpha = 0.5 * (1.0 - p.epsilon);
  A.W = H->pin_active ? H->pinW[0] : nullptr;
  A.phihat = H->pinhat;
  A.guess = (p.guess == MPFC_GUESS_PREV) ? 0 : 1;   // the learned guess corrects the extrapolation
  dim3 g0 = grid_for(L0.m, L0.n, kBlk2d);
  mpfc_launch(H->shape, k_source_guess<SCH>, g0, kBlk2d, 0, s, L0, A);
  if (p.guess == MPFC_GUESS_LEARNED && network) mpfc_enqueue_learned_guess(H, s);
  if (SCH == 2)
    for (int l = 1; l < H->nlev; ++l) {
      const Lev& C = H->lev[l];
      mpfc_launch(H->shape, k_restrict_plane, grid_for(C.m, C.n, kBlk2d), kBlk2d, 0, s, (const double*)H->lev[l - 1].pk, C.pk,
                 C.m, C.n);
    }
  mpfc_launch(H->shape, k_guess_kappa, g0, kBlk2d, 0, s, L0, H->coef[SCH - 1][0]);
  mpfc_launch(H->shape, k_guess_mu<SCH>, g0, kBlk2d, 0, s, L0, H->coef[SCH - 1][0]);
}

template <int SCH>
static void enqueue_commit(mpfc_s* H, cudaStream_t s) {
  size_t G = (size_t)H->p.m * H->p.n;
  int blocks = (int)((G + 255) / 256);
  if (blocks > 16 * mpfc::sm_count()) blocks = 16 * mpfc::sm_count();
  mpfc_launch(H->shape, k_commit<SCH>, dim3(blocks), dim3(256), 0, s, (const double*)H->lev[0].phi, H->phik, H->phikm1, H->psik,
             H->guess.phikm2, (int)G, 1.0 / H->p.dt, (int)(H->p.model == MPFC_MODEL_PFC), H->ctl, H->info);
}

template <int SCH>
static void enqueue_resnorm(mpfc_s* H, int mode, cudaGraphConditionalHandle hnd, int set_cond, cudaStream_t s) {
  const Lev& L0 = H->lev[0];
  if (mode == 1 && vcycle_fuses_norm(H)) {   // after a V-cycle that ended with k_smooth_res
    int blocks = mpfc_reduce_blocks((size_t)L0.m * L0.n / 2);
    mpfc_launch(H->shape, k_resnorm_red<SCH>, dim3(blocks), dim3(256), 0, s, L0, H->coef[SCH - 1][0], H->ctl,
                H->partials, (const double*)H->bpart, H->nbpart, hnd, set_cond);
    return;
  }
  int blocks = mpfc_reduce_blocks((size_t)L0.m * L0.n);
  if (mode == 0)   // right after the initial guess: rows 2 and 3 hold by construction
    mpfc_launch(H->shape, k_resnorm<SCH, true>, dim3(blocks), dim3(256), 0, s, L0, H->coef[SCH - 1][0], H->ctl,
                H->partials, mode, hnd, set_cond);
  else
    mpfc_launch(H->shape, k_resnorm<SCH>, dim3(blocks), dim3(256), 0, s, L0, H->coef[SCH - 1][0], H->ctl, H->partials,
                mode, hnd, set_cond);
}

// Body of the FP64 WHILE node: one V-cycle, then the residual test that sets the
// loop condition.
// The gated learned correction: the network adds its correction to the extrapolated
// guess, kappa and mu are formed again from the corrected phi, and the residual test of
// the guess runs again (it sets the V-cycle loop's condition).
template <int SCH>
static void enqueue_learned_correction(mpfc_s* H, cudaGraphConditionalHandle hnd, int set_cond, cudaStream_t s) {
  const Lev& L0 = H->lev[0];
  dim3 g0 = grid_for(L0.m, L0.n, kBlk2d);
  mpfc_enqueue_learned_guess(H, s);
  mpfc_launch(H->shape, k_guess_kappa, g0, kBlk2d, 0, s, L0, H->coef[SCH - 1][0]);
  mpfc_launch(H->shape, k_guess_mu<SCH>, g0, kBlk2d, 0, s, L0, H->coef[SCH - 1][0]);
  enqueue_resnorm<SCH>(H, 0, hnd, set_cond, s);
}

static void learned_body(mpfc_s* H, int scheme, cudaStream_t s) {
  if (scheme == 1) enqueue_learned_correction<1>(H, H->cur_handle, 1, s);
  else enqueue_learned_correction<2>(H, H->cur_handle, 1, s);
}

static void fp64_body(mpfc_s* H, int scheme, cudaStream_t s) {
  cudaGraphConditionalHandle hnd = H->cur_handle;
  if (scheme == 1) {
    enqueue_vcycle<1>(H, s);
    enqueue_resnorm<1>(H, 1, hnd, 1, s);
  } else {
    enqueue_vcycle<2>(H, s);
    enqueue_resnorm<2>(H, 1, hnd, 1, s);
  }
}

// Builds the step graph of one scheme:
//   prologue -> resnorm(mode 0, sets cond) -> WHILE(cond){ V-cycle; resnorm(mode 1) } -> commit
template <int SCH>
static int build_step_graph(mpfc_s* H) {
  cudaStream_t cs = H->cap_stream;
  cudaGraph_t graph = nullptr;
  cudaGraphConditionalHandle hnd;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CKCAP(cudaStreamGetCaptureInfo(cs, &st, nullptr, &graph, &deps, nullptr, &ndeps), cs);
  CKCAP(cudaGraphConditionalHandleCreate(&hnd, graph, 0, 0), cs);
  H->cur_handle = hnd;
  int rc;
  if (H->p.precision == MPFC_FP32_INNER) {
    rc = mpfc_fp32_enqueue_step(H, SCH, cs, hnd);
  } else {
    const bool gated = guess_gated(H);
    enqueue_prologue<SCH>(H, cs, !gated);
    enqueue_resnorm<SCH>(H, 0, hnd, 1, cs);
    rc = MPFC_OK;
    if (gated) {   // IF(res0 >= gate){ network; kappa, mu; resnorm(mode 0, sets cond) }
      cudaGraphConditionalHandle hif;
      CKCAP(cudaGraphConditionalHandleCreate(&hif, graph, 0, 0), cs);
      mpfc_launch(H->shape, k_guess_gate, dim3(1), dim3(32), 0, cs, (const Ctl*)H->ctl, H->guess_gate, hif);
      rc = mpfc_capture_conditional(H, cs, hif, cudaGraphCondTypeIf, &learned_body, SCH);
    }
    if (rc == MPFC_OK) rc = mpfc_capture_while(H, cs, hnd, &fp64_body, SCH);
    if (rc == MPFC_OK) enqueue_commit<SCH>(H, cs);
  }
  if (rc != MPFC_OK) {
    mpfc_abort_capture(cs);
    return rc;
  }
  CK(cudaStreamEndCapture(cs, &graph));
  cudaGraphExec_t exec;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "cudaGraphInstantiate(step graph)", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  H->exec[SCH - 1][0] = exec;
  return MPFC_OK;
}

// Ends a capture on s that an error interrupted, so that the stream can be used again.
// The partial graph is left undestroyed: after a failed capture into a conditional
// node's body, that body's state is not one the runtime documents as safe to destroy,
// and an error path that loses a graph is better than one that can crash the process.
void mpfc_abort_capture(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess || st == cudaStreamCaptureStatusNone) {
    (void)cudaGetLastError();
    return;
  }
  cudaGraph_t g = nullptr;
  (void)cudaStreamEndCapture(s, &g);
  (void)cudaGetLastError();   // the invalidated capture's error is reported by the caller
}

int mpfc_capture_while(mpfc_s* H, cudaStream_t cs, cudaGraphConditionalHandle hnd, void (*body_fn)(mpfc_s*, int, cudaStream_t),
                       int scheme) {
  return mpfc_capture_conditional(H, cs, hnd, cudaGraphCondTypeWhile, body_fn, scheme);
}

int mpfc_capture_conditional(mpfc_s* H, cudaStream_t cs, cudaGraphConditionalHandle hnd, cudaGraphConditionalNodeType type,
                             void (*body_fn)(mpfc_s*, int, cudaStream_t), int scheme) {
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamGetCaptureInfo(cs, &st, nullptr, &graph, &deps, nullptr, &ndeps));
  std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = hnd;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  CK(cudaGraphAddNode(&cnode, graph, dv.data(), nullptr, dv.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  CK(cudaStreamBeginCaptureToGraph(H->body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  body_fn(H, scheme, H->body_stream);
  CKCAP(cudaStreamEndCapture(H->body_stream, &body), H->body_stream);
  return MPFC_OK;
}

// Shared pieces used by the FP32-inner driver.
void mpfc_enqueue_prologue(mpfc_s* H, int scheme, cudaStream_t s) {
  if (scheme == 1) enqueue_prologue<1>(H, s);
  else enqueue_prologue<2>(H, s);
}
void mpfc_enqueue_commit(mpfc_s* H, int scheme, cudaStream_t s) {
  if (scheme == 1) enqueue_commit<1>(H, s);
  else enqueue_commit<2>(H, s);
}

// Host mirror of the device-side loop decision of k_resnorm.
static bool host_continue(const Ctl& c) {
  if (c.skip || c.status != 0) return false;
  if (c.fixed_cycles > 0) return c.cycles < c.fixed_cycles;
  return c.res > c.tol && c.cycles < c.max_cycles;
}

// One step launched kernel by kernel on the stream, with the loop decision read
// back after every residual test (same kernels, same order as the graph).
static int step_stream_mode(mpfc_s* H, int scheme) {
  MpfcRange range("mpfc step");
  cudaStream_t s = H->stream;
  if (H->p.precision == MPFC_FP32_INNER) return mpfc_fp32_step_stream(H, scheme);
  const bool gated = guess_gated(H);
  if (scheme == 1) {
    enqueue_prologue<1>(H, s, !gated);
    enqueue_resnorm<1>(H, 0, 0, 0, s);
  } else {
    enqueue_prologue<2>(H, s, !gated);
    enqueue_resnorm<2>(H, 0, 0, 0, s);
  }
  if (gated) {   // the gate read on the host
    Ctl c;
    CK(cudaMemcpyAsync(&c, H->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (c.status == 0 && c.res0 >= H->guess_gate) {
      if (scheme == 1) enqueue_learned_correction<1>(H, 0, 0, s);
      else enqueue_learned_correction<2>(H, 0, 0, s);
    }
  }
  for (;;) {
    Ctl c;
    CK(cudaMemcpyAsync(&c, H->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!host_continue(c)) break;
    MpfcRange vrange("V-cycle");
    if (scheme == 1) {
      enqueue_vcycle<1>(H, s);
      enqueue_resnorm<1>(H, 1, 0, 0, s);
    } else {
      enqueue_vcycle<2>(H, s);
      enqueue_resnorm<2>(H, 1, 0, 0, s);
    }
  }
  if (scheme == 1) enqueue_commit<1>(H, s);
  else enqueue_commit<2>(H, s);
  CK(cudaGetLastError());
  return MPFC_OK;
}

int mpfc_host_continue(const Ctl* c) { return host_continue(*c) ? 1 : 0; }

static int launch_steps(mpfc_s* H, int scheme, int nsteps) {
  if (H->launch_mode == MPFC_LAUNCH_STREAM) {
    for (int k = 0; k < nsteps; ++k) {
      int rc = step_stream_mode(H, scheme);
      if (rc != MPFC_OK) return rc;
    }
    return MPFC_OK;
  }
  for (int k = 0; k < nsteps; ++k) {
    MpfcRange range("mpfc step");
    CK(cudaGraphLaunch(H->exec[scheme - 1][0], H->stream));
  }
  return MPFC_OK;
}

extern "C" int mpfc_set_launch_shape(mpfc_t* H, int rows, int small_cells, int pdl_blocks, int tail_cells,
                                     int tail_ctas) {
  if (!H || (rows != 1 && rows != 2 && rows != 4 && rows != 8) || small_cells < 0 || pdl_blocks < 0 ||
      tail_cells < 0 || (tail_ctas != 1 && tail_ctas != 8 && tail_ctas != 16))
    return MPFC_ERR_INVALID;
  if (tail_ctas > mpfc_tail_max_ctas()) return MPFC_ERR_INVALID;
  H->shape = mpfc_launch_shape{rows, small_cells, pdl_blocks, tail_cells, tail_ctas, H->shape.split_cells};
  mpfc_drop_graphs(H);
  return MPFC_OK;
}

extern "C" int mpfc_set_transfer_split(mpfc_t* H, int fine_cells) {
  if (!H || fine_cells < 0) return MPFC_ERR_INVALID;
  H->shape.split_cells = fine_cells;
  mpfc_drop_graphs(H);
  return MPFC_OK;
}

extern "C" int mpfc_set_guess_gate(mpfc_t* H, double res0_threshold) {
  if (!H || H->p.guess != MPFC_GUESS_LEARNED || H->p.precision != MPFC_FP64 || !(res0_threshold >= 0.0))
    return MPFC_ERR_INVALID;
  H->guess_gate = res0_threshold;
  mpfc_drop_graphs(H);
  return MPFC_OK;
}

extern "C" int mpfc_launch_counts(const mpfc_t* H, int scheme, int* per_step, int* per_cycle) {
  if (!H || (scheme != 1 && scheme != 2) || H->p.precision != MPFC_FP64 || H->p.guess == MPFC_GUESS_LEARNED)
    return MPFC_ERR_INVALID;
  const mpfc_params& p = H->p;
  const int L = H->nlev, lt = tail_first_level(H);
  const int down = lt < L ? lt : L - 1;   // levels run by per-level launches
  // per level: nu1 + nu2 sweeps of two colours, restriction, tau, prolongation
  const int per_level = 2 * p.nu1 + 2 * p.nu2 + 3;
  // + the tail launch or the coarsest solve, + the residual test
  if (per_cycle) *per_cycle = down * per_level + 2;
  // step begin, source and guess, kappa, mu, [phi^k onto the coarse levels], residual test, commit
  if (per_step) *per_step = 6 + (scheme == 2 ? L - 1 : 0);
  return MPFC_OK;
}

extern "C" int mpfc_set_launch_mode(mpfc_t* H, int mode) {
  if (!H || (mode != MPFC_LAUNCH_GRAPH && mode != MPFC_LAUNCH_STREAM)) return MPFC_ERR_INVALID;
  H->launch_mode = mode;
  return MPFC_OK;
}

static int ensure_graph(mpfc_s* H, int scheme) {
  if (H->launch_mode == MPFC_LAUNCH_STREAM) return MPFC_OK;
  if (H->exec[scheme - 1][0]) return MPFC_OK;
  return scheme == 1 ? build_step_graph<1>(H) : build_step_graph<2>(H);
}

// ---------------------------------------------------------------------------
// State and stepping
// ---------------------------------------------------------------------------
extern "C" int mpfc_set_state(mpfc_t* H, const double* phi, const double* phi_prev, const double* psi) {
  if (!H || !phi) return MPFC_ERR_INVALID;
  size_t bytes = (size_t)H->p.m * H->p.n * sizeof(double);
  CK(cudaMemcpyAsync(H->phik, phi, bytes, cudaMemcpyDefault, H->stream));
  CK(cudaMemcpyAsync(H->phikm1, phi_prev ? phi_prev : phi, bytes, cudaMemcpyDefault, H->stream));
  if (psi) CK(cudaMemcpyAsync(H->psik, psi, bytes, cudaMemcpyDefault, H->stream));
  else CK(cudaMemsetAsync(H->psik, 0, bytes, H->stream));
  if (H->guess.phikm2)
    CK(cudaMemcpyAsync(H->guess.phikm2, phi_prev ? phi_prev : phi, bytes, cudaMemcpyDefault, H->stream));
  k_ctl_reset<<<1, 32, 0, H->stream>>>(H->ctl, 0);
  CK(cudaGetLastError());
  return MPFC_OK;
}

extern "C" int mpfc_get_state(mpfc_t* H, double* phi, double* phi_prev, double* psi) {
  if (!H) return MPFC_ERR_INVALID;
  size_t bytes = (size_t)H->p.m * H->p.n * sizeof(double);
  if (phi) CK(cudaMemcpyAsync(phi, H->phik, bytes, cudaMemcpyDefault, H->stream));
  if (phi_prev) CK(cudaMemcpyAsync(phi_prev, H->phikm1, bytes, cudaMemcpyDefault, H->stream));
  if (psi) CK(cudaMemcpyAsync(psi, H->psik, bytes, cudaMemcpyDefault, H->stream));
  CK(cudaStreamSynchronize(H->stream));
  return MPFC_OK;
}

static int run_steps(mpfc_s* H, int scheme, int nsteps, int fixed_cycles, mpfc_step_info* per_step) {
  if (!H || (scheme != 1 && scheme != 2) || nsteps < 0) return MPFC_ERR_INVALID;
  if (H->pin_active && scheme != 2) return MPFC_ERR_INVALID;   // pinning is a second-order-scheme term
  if (H->p.guess == MPFC_GUESS_LEARNED && !mpfc_has_guess_model(H)) return MPFC_ERR_INVALID;
  int rc = ensure_graph(H, scheme);
  if (rc != MPFC_OK) return rc;
  std::vector<StepRecord> rec(kInfoCap);
  int done = 0;
  int first_err = MPFC_OK;
  while (done < nsteps && first_err == MPFC_OK) {
    int chunk = nsteps - done < kInfoCap ? nsteps - done : kInfoCap;
    k_ctl_reset<<<1, 32, 0, H->stream>>>(H->ctl, fixed_cycles);
    CK(cudaGetLastError());
    rc = launch_steps(H, scheme, chunk);
    if (rc != MPFC_OK) return rc;
    CK(cudaMemcpyAsync(rec.data(), H->info, chunk * sizeof(StepRecord), cudaMemcpyDeviceToHost, H->stream));
    CK(cudaStreamSynchronize(H->stream));
    for (int k = 0; k < chunk; ++k) {
      const StepRecord& r = rec[k];
      if (per_step) {
        per_step[done + k].cycles = r.cycles;
        per_step[done + k].status = r.status;
        per_step[done + k].res0 = r.res0;
        per_step[done + k].res_final = r.res_final;
      }
      if (r.status != 0 && first_err == MPFC_OK) {
        first_err = r.status;
        // later records of this chunk were skipped steps; mark them
        for (int q = k + 1; q < chunk && per_step; ++q) {
          per_step[done + q].cycles = 0;
          per_step[done + q].status = r.status;
          per_step[done + q].res0 = per_step[done + q].res_final = 0.0;
        }
        break;
      }
    }
    done += chunk;
  }
  if (first_err != MPFC_OK && per_step)
    for (int q = done; q < nsteps; ++q) {
      per_step[q].cycles = 0;
      per_step[q].status = first_err;
      per_step[q].res0 = per_step[q].res_final = 0.0;
    }
  return first_err;
}

extern "C" int mpfc_step(mpfc_t* H, int scheme, int nsteps, mpfc_step_info* per_step) {
  return run_steps(H, scheme, nsteps, 0, per_step);
}

extern "C" int mpfc_step_async(mpfc_t* H, int scheme, int nsteps) {
  if (!H || (scheme != 1 && scheme != 2) || nsteps < 0) return MPFC_ERR_INVALID;
  if (H->pin_active && scheme != 2) return MPFC_ERR_INVALID;
  if (H->p.guess == MPFC_GUESS_LEARNED && !mpfc_has_guess_model(H)) return MPFC_ERR_INVALID;
  int rc = ensure_graph(H, scheme);
  if (rc != MPFC_OK) return rc;
  return launch_steps(H, scheme, nsteps);
}

extern "C" int mpfc_records(mpfc_t* H, mpfc_step_info* out, int max_records, int* count) {
  if (!H || max_records < 0) return MPFC_ERR_INVALID;
  Ctl c;
  CK(cudaMemcpyAsync(&c, H->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, H->stream));
  CK(cudaStreamSynchronize(H->stream));
  int n = c.slot < kInfoCap ? c.slot : kInfoCap;
  if (n > max_records) n = max_records;
  std::vector<StepRecord> rec(n > 0 ? n : 1);
  if (n > 0) CK(cudaMemcpyAsync(rec.data(), H->info, n * sizeof(StepRecord), cudaMemcpyDeviceToHost, H->stream));
  k_ctl_reset<<<1, 32, 0, H->stream>>>(H->ctl, 0);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(H->stream));
  int first = MPFC_OK;
  for (int k = 0; k < n; ++k) {
    if (out) {
      out[k].cycles = rec[k].cycles;
      out[k].status = rec[k].status;
      out[k].res0 = rec[k].res0;
      out[k].res_final = rec[k].res_final;
    }
    if (rec[k].status != 0 && first == MPFC_OK) first = rec[k].status;
  }
  if (count) *count = c.slot;
  return first;
}

extern "C" int mpfc_step_cycles(mpfc_t* H, int scheme, int ncycles, mpfc_step_info* info) {
  if (ncycles < 1) return MPFC_ERR_INVALID;
  return run_steps(H, scheme, 1, ncycles, info);
}

// ---------------------------------------------------------------------------
// Diagnostics
// ---------------------------------------------------------------------------
static int read_sums(mpfc_s* H, double* out, int count) {
  double tmp[kMaxSums];
  CK(cudaMemcpyAsync(tmp, H->ctl->sums, sizeof(double) * kMaxSums, cudaMemcpyDeviceToHost, H->stream));
  CK(cudaStreamSynchronize(H->stream));
  for (int i = 0; i < count; ++i) out[i] = tmp[i];
  return MPFC_OK;
}

extern "C" int mpfc_mass(mpfc_t* H, double* out) {
  if (!H || !out) return MPFC_ERR_INVALID;
  size_t G = (size_t)H->p.m * H->p.n;
  k_sum1<<<mpfc_reduce_blocks(G), 256, 0, H->stream>>>(H->phik, (int)G, H->ctl, H->partials);
  CK(cudaGetLastError());
  double s;
  int rc = read_sums(H, &s, 1);
  if (rc) return rc;
  *out = H->p.h * H->p.h * s;
  return MPFC_OK;
}

// Periodic Poisson multigrid: -Delta_h x = f (f mean-zero), V(2,2) red-black
// cycles until ||r|| <= 1e-13 ||f|| (at most 60).  Result in H->px[0].
static int poisson_solve(mpfc_s* H, const double* rhs) {
  int L = H->nlev;
  size_t G0 = (size_t)H->p.m * H->p.n;
  cudaStream_t s = H->stream;
  k_sum1<<<mpfc_reduce_blocks(G0), 256, 0, s>>>(rhs, (int)G0, H->ctl, H->partials);
  k_sub_mean<<<mpfc_reduce_blocks(G0), 256, 0, s>>>(rhs, H->pf[0], (int)G0, H->ctl);
  CK(cudaMemsetAsync(H->px[0], 0, G0 * sizeof(double), s));
  for (int cyc = 0; cyc < 60; ++cyc) {
    for (int l = 0; l < L - 1; ++l) {
      const Lev& F = H->lev[l];
      dim3 g = grid_for(F.m / 2, F.n, kBlk2d);
      for (int sw = 0; sw < 2; ++sw)
        for (int c = 0; c < 2; ++c) k_pois_smooth<<<g, kBlk2d, 0, s>>>(H->px[l], H->pf[l], F.m, F.n, F.nyn, F.h * F.h, c);
      const Lev& C = H->lev[l + 1];
      k_pois_restrict<<<grid_for(C.m, C.n, kBlk2d), kBlk2d, 0, s>>>(H->px[l], H->pf[l], H->pf[l + 1], H->px[l + 1],
                                                                     C.m, C.n, C.nyn, 1.0 / (F.h * F.h));
    }
    const Lev& Cc = H->lev[L - 1];
    k_pois_coarse<<<1, 128, sizeof(double) * (Cc.m * Cc.n + 1), s>>>(H->px[L - 1], H->pf[L - 1], Cc.m, Cc.n,
                                                                      Cc.nyn, Cc.h * Cc.h, 200);
    for (int l = L - 2; l >= 0; --l) {
      const Lev& F = H->lev[l];
      const Lev& C = H->lev[l + 1];
      k_pois_prolong<<<grid_for(C.m, C.n, kBlk2d), kBlk2d, 0, s>>>(H->px[l + 1], H->px[l], C.m, C.n, C.nyn);
      dim3 g = grid_for(F.m / 2, F.n, kBlk2d);
      for (int sw = 0; sw < 2; ++sw)
        for (int c = 0; c < 2; ++c) k_pois_smooth<<<g, kBlk2d, 0, s>>>(H->px[l], H->pf[l], F.m, F.n, F.nyn, F.h * F.h, c);
    }
    const Lev& F0 = H->lev[0];
    k_pois_resnorm<<<mpfc_reduce_blocks(G0), 256, 0, s>>>(H->px[0], H->pf[0], F0.m, F0.n, F0.nyn,
                                                          1.0 / (F0.h * F0.h), H->ctl, H->partials);
    CK(cudaGetLastError());
    double v[2];
    int rc = read_sums(H, v, 2);
    if (rc) return rc;
    if (!(v[0] == v[0])) return MPFC_ERR_DIVERGED;
    if (v[0] <= 1e-26 * v[1] || v[1] == 0.0) break;
  }
  return MPFC_OK;
}

extern "C" int mpfc_energy(mpfc_t* H, mpfc_energy_t* out) {
  if (!H || !out) return MPFC_ERR_INVALID;
  int rc = poisson_solve(H, H->psik);
  if (rc) return rc;
  size_t G = (size_t)H->p.m * H->p.n;
  k_energy_sums<<<mpfc_reduce_blocks(G), 256, 0, H->stream>>>(
      H->phik, H->phikm1, H->psik, H->px[0], H->p.m, H->p.n, H->lev[0].nyn, H->pin_active ? H->pinW[0] : nullptr,
      H->pinhat, H->ctl, H->partials);
  CK(cudaGetLastError());
  double v[7];
  rc = read_sums(H, v, 7);
  if (rc) return rc;
  double h = H->p.h, h2 = h * h, alpha = 1.0 - H->p.epsilon;
  double F = 0.25 * h2 * v[0] + 0.5 * alpha * h2 * v[1] - v[2] + 0.5 * h2 * v[3] / (h2 * h2);
  double m1 = h2 * v[4];
  out->F = F;
  out->pseudoF = H->p.model == MPFC_MODEL_PFC ? F : F + m1 / (2.0 * H->p.M);
  out->tildeF = out->pseudoF + 0.5 * v[5];
  out->pinning = h2 * v[6];
  return MPFC_OK;
}

extern "C" int mpfc_set_pinning(mpfc_t* H, const double* weight, const double* target) {
  if (!H || !H->p.pinning || (weight && !target)) return MPFC_ERR_INVALID;
  mpfc_drop_graphs(H);   // the levels' weight pointers are part of the captured kernels
  if (!weight) {
    H->pin_active = 0;
    for (int l = 0; l < H->nlev; ++l) H->lev[l].W = nullptr;
    return MPFC_OK;
  }
  size_t G = (size_t)H->p.m * H->p.n;
  CK(cudaMemcpyAsync(H->pinW[0], weight, G * sizeof(double), cudaMemcpyDefault, H->stream));
  CK(cudaMemcpyAsync(H->pinhat, target, G * sizeof(double), cudaMemcpyDefault, H->stream));
  for (int l = 1; l < H->nlev; ++l) {
    const Lev& C = H->lev[l];
    k_restrict_plane<<<grid_for(C.m, C.n, kBlk2d), kBlk2d, 0, H->stream>>>(H->pinW[l - 1], H->pinW[l], C.m, C.n);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(H->stream));
  H->pin_active = 1;
  for (int l = 0; l < H->nlev; ++l) H->lev[l].W = H->pinW[l];
  return MPFC_OK;
}

extern "C" const char* mpfc_strerror(int status) {
  switch (status) {
    case MPFC_OK: return "ok";
    case MPFC_ERR_INVALID: return "invalid argument or parameters";
    case MPFC_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
    case MPFC_ERR_CUDA: return g_last_cuda_error[0] ? g_last_cuda_error : "CUDA error";
    case MPFC_ERR_NOT_CONVERGED: return "V-cycle limit reached before the tolerance";
    case MPFC_ERR_DIVERGED: return "residual became non-finite or grew beyond 1e10 times its start";
    case MPFC_ERR_TOO_LARGE: return "grid exceeds the 2048 x 2048 cells the static scratch of mpfc_mass_noalloc allows";
    default: return "unknown status";
  }
}

// ---------------------------------------------------------------------------
// Component entry points
// ---------------------------------------------------------------------------
static bool level_ok(const mpfc_s* H, int level) { return H && level >= 0 && level < H->nlev; }

extern "C" int mpfc_op_source(mpfc_t* H, int scheme, const double* phik, const double* phikm1, const double* psik,
                              double* S1, double* S2, double* S3) {
  if (!H || (scheme != 1 && scheme != 2) || !phik || !phikm1 || !psik || !S1 || !S2 || !S3) return MPFC_ERR_INVALID;
  const mpfc_params& p = H->p;
  Lev L = H->lev[0];
  L.S1 = S1;
  L.S2 = S2;
  L.S3 = S3;
  L.phi = nullptr;
  SourceArgs A{phik, phikm1, psik, H->pin_active ? H->pinW[0] : nullptr, H->pinhat,
               p.model == MPFC_MODEL_PFC ? 0.0
               : scheme == 1             ? 1.0 / (p.beta + 1.0 / p.dt)
                                         : 2.0 / (p.beta + 2.0 / p.dt),
               0.5 * (1.0 - p.epsilon), 2};
  dim3 g = grid_for(L.m, L.n, kBlk2d);
  if (scheme == 1) k_source_guess<1><<<g, kBlk2d, 0, H->stream>>>(L, A);
  else k_source_guess<2><<<g, kBlk2d, 0, H->stream>>>(L, A);
  CK(cudaGetLastError());
  return MPFC_OK;
}

static Lev user_level(const mpfc_s* H, int level, double* phi, double* mu, double* ka, const double* S1,
                      const double* S2, const double* S3, const double* pk) {
  Lev L = H->lev[level];
  L.phi = phi;
  L.mu = mu;
  L.ka = ka;
  L.S1 = const_cast<double*>(S1);
  L.S2 = const_cast<double*>(S2);
  L.S3 = const_cast<double*>(S3);
  L.pk = const_cast<double*>(pk);
  L.b1 = L.b2 = L.b3 = nullptr;
  return L;
}

extern "C" int mpfc_op_smooth(mpfc_t* H, int scheme, int level, double* phi, double* mu, double* kappa,
                              const double* S1, const double* S2, const double* S3, const double* phik, int sweeps) {
  if (!level_ok(H, level) || (scheme != 1 && scheme != 2) || sweeps < 0 || (scheme == 2 && !phik))
    return MPFC_ERR_INVALID;
  Lev L = user_level(H, level, phi, mu, kappa, S1, S2, S3, phik);
  if (scheme == 1) launch_smooth<1>(H->shape, L, H->coef[0][level], H->coefb[0][level], sweeps, H->stream);
  else launch_smooth<2>(H->shape, L, H->coef[1][level], H->coefb[1][level], sweeps, H->stream);
  CK(cudaGetLastError());
  return MPFC_OK;
}

extern "C" int mpfc_op_residual(mpfc_t* H, int scheme, int level, const double* phi, const double* mu,
                                const double* kappa, const double* S1, const double* S2, const double* S3,
                                const double* phik, double* r1, double* r2, double* r3) {
  if (!level_ok(H, level) || (scheme != 1 && scheme != 2) || (scheme == 2 && !phik)) return MPFC_ERR_INVALID;
  Lev L = user_level(H, level, const_cast<double*>(phi), const_cast<double*>(mu), const_cast<double*>(kappa), S1, S2,
                     S3, phik);
  dim3 g = grid_for(L.m, L.n, kBlk2d);
  if (scheme == 1) k_residual<1><<<g, kBlk2d, 0, H->stream>>>(L, H->coef[0][level], r1, r2, r3);
  else k_residual<2><<<g, kBlk2d, 0, H->stream>>>(L, H->coef[1][level], r1, r2, r3);
  CK(cudaGetLastError());
  return MPFC_OK;
}

extern "C" int mpfc_op_restrict(mpfc_t* H, int scheme, int level, const double* phi, const double* mu,
                                const double* kappa, const double* S1, const double* S2, const double* S3,
                                const double* phik, const double* phik_c, double* phi_c, double* mu_c,
                                double* kappa_c, double* S1_c, double* S2_c, double* S3_c) {
  if (!level_ok(H, level) || level + 1 >= H->nlev || (scheme != 1 && scheme != 2) ||
      (scheme == 2 && (!phik || !phik_c)))
    return MPFC_ERR_INVALID;
  Lev F = user_level(H, level, const_cast<double*>(phi), const_cast<double*>(mu), const_cast<double*>(kappa), S1, S2,
                     S3, phik);
  Lev C = user_level(H, level + 1, phi_c, mu_c, kappa_c, S1_c, S2_c, S3_c, phik_c);
  dim3 g = grid_for(C.m, C.n, kBlk2d);
  if (scheme == 1) {
    k_resid_restrict<1><<<g, kBlk2d, 0, H->stream>>>(F, C, H->coef[0][level], 0);
    k_tau<1><<<g, kBlk2d, 0, H->stream>>>(C, H->coef[0][level + 1]);
  } else {
    k_resid_restrict<2><<<g, kBlk2d, 0, H->stream>>>(F, C, H->coef[1][level], 0);
    k_tau<2><<<g, kBlk2d, 0, H->stream>>>(C, H->coef[1][level + 1]);
  }
  CK(cudaGetLastError());
  return MPFC_OK;
}

extern "C" int mpfc_op_prolong(mpfc_t* H, int level, const double* phi_c_new, const double* mu_c_new,
                               const double* kappa_c_new, const double* phi_c_old, const double* mu_c_old,
                               const double* kappa_c_old, double* phi, double* mu, double* kappa) {
  if (!level_ok(H, level) || level + 1 >= H->nlev) return MPFC_ERR_INVALID;
  const Lev& C = H->lev[level + 1];
  ProlongArgs A{phi_c_new, mu_c_new, kappa_c_new, phi_c_old, mu_c_old, kappa_c_old, phi, mu, kappa, C.m, C.n, C.nyn};
  k_prolong<<<grid_for(C.m, C.n, kBlk2d), kBlk2d, 0, H->stream>>>(A);
  CK(cudaGetLastError());
  return MPFC_OK;
}

extern "C" int mpfc_op_coarse_solve(mpfc_t* H, int scheme, double* phi, double* mu, double* kappa, const double* S1,
                                    const double* S2, const double* S3, const double* phik) {
  if (!H || (scheme != 1 && scheme != 2) || (scheme == 2 && !phik)) return MPFC_ERR_INVALID;
  int l = H->nlev - 1;
  Lev C = user_level(H, l, phi, mu, kappa, S1, S2, S3, phik);
  if (scheme == 1) launch_coarse<1>(H, C, H->coef[0][l], H->stream);
  else launch_coarse<2>(H, C, H->coef[1][l], H->stream);
  CK(cudaGetLastError());
  return MPFC_OK;
}
