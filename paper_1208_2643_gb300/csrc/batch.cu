// Batched ensemble: many independent MPFC instances (uneven grid sizes and
// parameters) advanced together.  Every kernel of the FAS V-cycle runs as one
// persistent launch per multigrid level over a work list of (instance, tile) items,
// so the latency-bound coarse levels of all instances share launches.  Instances are
// aligned at their coarsest grid: global level GL-1 is every instance's coarsest, and
// an instance with L levels joins the descent at global level GL-L.  Each instance has
// its own residual test; converged instances drop out of the work (their items are
// skipped) while the others continue, and the whole step is one CUDA graph with a
// conditional WHILE node that runs while any instance is active.
#include <string.h>

#include <algorithm>
#include <vector>

#include "fp64_kernels.cuh"
#include "mpfc_internal.h"

using namespace mpfc;

namespace {

struct BItem {
  int inst, level, x0, y0;   // tile origin in the kernel's iteration domain
};

struct BCtl {                // per instance
  double res0, res;
  int cycles, status, active, halted;
  int total_cycles, steps, first_error, pad;
};

struct BGlobal {
  unsigned int counter;
  int fixed_cycles, max_cycles, any_active;
  double tol;
};

constexpr int kBlocksPerSM = 8;   // persistent launches: this many blocks per SM

// Sum over a block of any shape (linear thread index); the total is valid in thread 0.
__device__ __forceinline__ double block_total2d(double v, double* red) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = (blockDim.x * blockDim.y) >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double x = 0.0;
  if (wid == 0) {
    x = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  }
  __syncthreads();
  return x;
}

int grid_for_items(int n) { return std::max(1, std::min(n, kBlocksPerSM * mpfc::sm_count())); }

// ---------------------------------------------------------------------------
// Batched kernels (grid-stride over work items; one item = one tile of one level of
// one instance).  Lev / Coef tables are indexed [instance * kMaxLevels + level].
// ---------------------------------------------------------------------------
template <int SCH>
__global__ void kb_smooth(const BItem* __restrict__ items, int n, const Lev* __restrict__ levs,
                          const Coef* __restrict__ coefs, const BCtl* __restrict__ ctl, int color) {
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    BItem w = items[it];
    if (!ctl[w.inst].active) continue;
    const int id = w.inst * kMaxLevels + w.level;
    Lev L = levs[id];
    int x = w.x0 + threadIdx.x, j = w.y0 + threadIdx.y;
    if (x < (L.m >> 1) && j < L.n) smooth_cell<SCH>(L, coefs[id], coefs[id], 2 * x + ((j + color) & 1), j);
  }
}

// items over coarse levels (level >= 1): restriction from level-1 and tau
template <int SCH>
__global__ void kb_restrict(const BItem* __restrict__ items, int n, const Lev* __restrict__ levs,
                            const Coef* __restrict__ coefs, const BCtl* __restrict__ ctl) {
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    BItem w = items[it];
    if (!ctl[w.inst].active) continue;
    const int idc = w.inst * kMaxLevels + w.level;
    Lev C = levs[idc], F = levs[idc - 1];
    int I = w.x0 + threadIdx.x, J = w.y0 + threadIdx.y;
    if (I < C.m && J < C.n) resid_restrict_cell<SCH>(F, C, coefs[idc - 1], 1, I, J);
  }
}

template <int SCH>
__global__ void kb_tau(const BItem* __restrict__ items, int n, const Lev* __restrict__ levs,
                       const Coef* __restrict__ coefs, const BCtl* __restrict__ ctl) {
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    BItem w = items[it];
    if (!ctl[w.inst].active) continue;
    const int idc = w.inst * kMaxLevels + w.level;
    Lev C = levs[idc];
    int i = w.x0 + threadIdx.x, j = w.y0 + threadIdx.y;
    if (i < C.m && j < C.n) tau_cell<SCH>(C, coefs[idc], i, j);
  }
}

__global__ void __launch_bounds__(kPTX * kPTY) kb_prolong(const BItem* __restrict__ items, int n,
                                                          const Lev* __restrict__ levs, const BCtl* __restrict__ ctl) {
  __shared__ ProlongTile E;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    BItem w = items[it];
    if (!ctl[w.inst].active) continue;   // uniform over the block
    const int idc = w.inst * kMaxLevels + w.level;
    Lev C = levs[idc], F = levs[idc - 1];
    ProlongArgs A{C.phi, C.mu, C.ka, C.b1, C.b2, C.b3, F.phi, F.mu, F.ka, C.m, C.n};
    prolong_tile(A, E, w.x0, w.y0);
    __syncthreads();   // E is restaged for the next item
  }
}

__global__ void kb_restrict_pk(const BItem* __restrict__ items, int n, const Lev* __restrict__ levs,
                               const BCtl* __restrict__ ctl) {
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    BItem w = items[it];
    if (ctl[w.inst].halted) continue;
    const int idc = w.inst * kMaxLevels + w.level;
    Lev C = levs[idc], F = levs[idc - 1];
    int I = w.x0 + threadIdx.x, J = w.y0 + threadIdx.y;
    if (I < C.m && J < C.n) {
      size_t a = (size_t)(2 * J) * F.m + 2 * I, b = a + F.m;
      C.pk[(size_t)J * C.m + I] = 0.25 * ((F.pk[a] + F.pk[a + 1]) + (F.pk[b] + F.pk[b + 1]));
    }
  }
}

template <int SCH>
__global__ void kb_coarse(const Lev* __restrict__ levs, const Coef* __restrict__ coefs, const int* __restrict__ nlev,
                          const float* __restrict__ K3, const long long* __restrict__ K3off,
                          const BCtl* __restrict__ ctl) {
  int inst = blockIdx.x;
  if (!ctl[inst].active) return;
  int id = inst * kMaxLevels + nlev[inst] - 1;
  coarse_solve_block<SCH>(levs[id], coefs[id], K3 + K3off[inst]);
}

// finest-level work (items with level 0, grouped by instance)
template <int SCH>
__global__ void kb_source(const BItem* __restrict__ items, int n, const Lev* __restrict__ levs,
                          const SourceArgs* __restrict__ src, const BCtl* __restrict__ ctl) {
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    BItem w = items[it];
    if (ctl[w.inst].halted) continue;
    Lev L = levs[w.inst * kMaxLevels];
    int i = w.x0 + threadIdx.x, j = w.y0 + threadIdx.y;
    if (i < L.m && j < L.n) source_cell<SCH>(L, src[w.inst], i, j);
  }
}

template <int SCH>
__global__ void kb_guess(const BItem* __restrict__ items, int n, const Lev* __restrict__ levs,
                         const Coef* __restrict__ coefs, const BCtl* __restrict__ ctl, int stage) {
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    BItem w = items[it];
    if (ctl[w.inst].halted) continue;
    const int id = w.inst * kMaxLevels;
    Lev L = levs[id];
    int i = w.x0 + threadIdx.x, j = w.y0 + threadIdx.y;
    if (i < L.m && j < L.n) {
      if (stage == 0) guess_kappa_cell(L, coefs[id], i, j);
      else guess_mu_cell<SCH>(L, coefs[id], i, j);
    }
  }
}

__global__ void kb_step_begin(BCtl* ctl, int count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    ctl[i].cycles = 0;
    ctl[i].status = 0;
    ctl[i].active = !ctl[i].halted;
  }
}

// Per-instance scaled residual norms.  mode 0: after the guess; mode 1: after a
// V-cycle (only instances that took part are updated).  The last block reduces the
// per-item partials of each instance in item order (one warp per instance), updates
// the instance's loop state and sets the graph condition to "any instance active".
template <int SCH>
__global__ void __launch_bounds__(256) kb_resnorm(const BItem* __restrict__ items, int n,
                                                  const int* __restrict__ ibeg, int count,
                                                  const Lev* __restrict__ levs, const Coef* __restrict__ coefs,
                                                  BCtl* ctl, BGlobal* glob, double* partials, int mode,
                                                  cudaGraphConditionalHandle hnd, int set_cond) {
  __shared__ double red[32];
  __shared__ bool last;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    BItem w = items[it];
    double v = 0.0;
    bool take = (mode == 0) ? !ctl[w.inst].halted : (bool)ctl[w.inst].active;
    if (take) {
      const int id = w.inst * kMaxLevels;
      Lev L = levs[id];
      int i = w.x0 + threadIdx.x, j = w.y0 + threadIdx.y;
      if (i < L.m && j < L.n) {
        double a, b, c;
        resid_at<SCH>(L, coefs[id], i, j, a, b, c);
        v = fma(a, a, fma(b, b, c * c));
      }
    }
    double tot = block_total2d(v, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[it] = tot;
  }
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    last = (atomicAdd(&glob->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = (blockDim.x * blockDim.y) >> 5;
  for (int inst = wid; inst < count; inst += nw) {
    double s = 0.0;
    for (int it = ibeg[inst] + lane; it < ibeg[inst + 1]; it += 32) s += ((volatile double*)partials)[it];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
      BCtl& c = ctl[inst];
      Lev L = levs[inst * kMaxLevels];
      double res = sqrt(s / (3.0 * (double)L.m * (double)L.n));
      if (mode == 0) {
        if (!c.halted) {
          c.res0 = res;
          c.res = res;
          if (!(res == res) || isinf(res)) c.status = 2;
        }
      } else if (c.active) {
        c.res = res;
        c.cycles += 1;
        if (!(res == res) || isinf(res) || res > 1e10 * fmax(c.res0, glob->tol)) c.status = 2;
      }
      bool act = !c.halted && c.status == 0 &&
                 (glob->fixed_cycles > 0 ? c.cycles < glob->fixed_cycles
                                         : (c.res > glob->tol && c.cycles < glob->max_cycles));
      c.active = act ? 1 : 0;
    }
  }
  __syncthreads();
  if (tid == 0) {
    int any = 0;
    for (int inst = 0; inst < count; ++inst) any |= ctl[inst].active;
    glob->any_active = any;
    glob->counter = 0u;
    if (set_cond) cudaGraphSetConditional(hnd, any ? 1u : 0u);
  }
}

// psi update and history rotation per instance (level-0 items); a failing instance
// keeps its state and is halted for the rest of the call.
template <int SCH>
__global__ void kb_commit(const BItem* __restrict__ items, int n, const Lev* __restrict__ levs,
                          const double* __restrict__ inv_s, int pfc, double* const* __restrict__ state, BCtl* ctl,
                          const BGlobal* glob) {
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    BItem w = items[it];
    BCtl c = ctl[w.inst];
    if (c.halted) continue;
    bool ok = c.status == 0 && (glob->fixed_cycles > 0 || c.res <= glob->tol);
    if (!ok) continue;
    Lev L = levs[w.inst * kMaxLevels];
    int i = w.x0 + threadIdx.x, j = w.y0 + threadIdx.y;
    if (i < L.m && j < L.n) {
      size_t t = (size_t)j * L.m + i;
      double* phik = state[3 * w.inst];
      double* phikm1 = state[3 * w.inst + 1];
      double* psik = state[3 * w.inst + 2];
      double pn = L.phi[t], p0 = phik[t];
      double is = inv_s[w.inst];
      psik[t] = (SCH == 1 || pfc) ? (pn - p0) * is : 2.0 * is * (pn - p0) - psik[t];
      phikm1[t] = p0;
      phik[t] = pn;
    }
  }
}

__global__ void kb_step_end(BCtl* ctl, const BGlobal* glob, int count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  BCtl& c = ctl[i];
  if (c.halted) return;
  int st = 0;
  if (c.status == 2) st = MPFC_ERR_DIVERGED;
  else if (glob->fixed_cycles <= 0 && !(c.res <= glob->tol)) st = MPFC_ERR_NOT_CONVERGED;
  c.total_cycles += c.cycles;
  if (st != 0) {
    c.halted = 1;
    c.first_error = st;
  } else {
    c.steps += 1;
  }
}

__global__ void kb_reset(BCtl* ctl, BGlobal* glob, int count, int fixed_cycles) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    ctl[i].halted = 0;
    ctl[i].first_error = 0;
    ctl[i].total_cycles = 0;
    ctl[i].steps = 0;
  }
  if (i == 0) {
    glob->counter = 0u;
    glob->fixed_cycles = fixed_cycles;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct mpfc_batch_s {
  int count = 0;
  std::vector<mpfc_params> each;
  mpfc_params p0;
  cudaStream_t stream = nullptr, cap = nullptr, body = nullptr;
  int GL = 0;
  std::vector<int> nlev, gl0;
  std::vector<Lev> lev;            // [inst * kMaxLevels + l]
  std::vector<Coef> coef[2];
  std::vector<SourceArgs> src[2];
  // device tables
  Lev* d_lev = nullptr;
  Coef* d_coef[2] = {nullptr, nullptr};
  SourceArgs* d_src[2] = {nullptr, nullptr};
  int* d_nlev = nullptr;
  float* d_K3[2] = {nullptr, nullptr};
  long long* d_K3off = nullptr;
  double* d_inv_s = nullptr;
  double** d_state = nullptr;
  BCtl* d_ctl = nullptr;
  BGlobal* d_glob = nullptr;
  double* d_partials = nullptr;
  BItem* d_items = nullptr;
  int* d_ibeg = nullptr;
  size_t items_cap = 0;
  // item lists (offsets into d_items)
  std::vector<int> half_off, half_cnt, full_off, full_cnt;
  int fin_off = 0, fin_cnt = 0;
  std::vector<int> tile_x, tile_y;   // smoother tile (threads) per global level
  std::vector<double*> state;        // 3 per instance
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraphConditionalHandle hnd = 0;
  size_t ws_need = 0;
  char* ws = nullptr;
};

namespace {

#define BCK(call)                                             \
  do {                                                        \
    cudaError_t err_ = (call);                                \
    if (err_ != cudaSuccess) {                                \
      mpfc_set_cuda_error(err_, #call, __FILE__, __LINE__);   \
      return MPFC_ERR_CUDA;                                   \
    }                                                         \
  } while (0)

// As BCK, inside a stream capture: an error first ends the capture on `stream`, so
// that the stream is not left capturing (mpfc_abort_capture).
#define BCKCAP(call, stream)                                  \
  do {                                                        \
    cudaError_t err_ = (call);                                \
    if (err_ != cudaSuccess) {                                \
      mpfc_set_cuda_error(err_, #call, __FILE__, __LINE__);   \
      mpfc_abort_capture(stream);                             \
      return MPFC_ERR_CUDA;                                   \
    }                                                         \
  } while (0)

struct BCarver {
  char* base;
  size_t off;
  template <typename T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off = (off + count * sizeof(T) + 255) & ~(size_t)255;
    return p;
  }
};

bool same_solver_settings(const mpfc_params& a, const mpfc_params& b) {
  return a.nu1 == b.nu1 && a.nu2 == b.nu2 && a.coarsest == b.coarsest && a.omega == b.omega && a.tol == b.tol &&
         a.max_cycles == b.max_cycles && a.precision == b.precision && a.guess == b.guess && a.model == b.model;
}

// Work items of one iteration domain (dx x dy cells or half-cells) tiled tx x ty.
void add_items(std::vector<BItem>& v, int inst, int level, int dx, int dy, int tx, int ty) {
  for (int y = 0; y < dy; y += ty)
    for (int x = 0; x < dx; x += tx) v.push_back(BItem{inst, level, x, y});
}

// Builds every work list (with the current smoother tiles) and the device tables.
int build_items(mpfc_batch_s* B) {
  std::vector<BItem> all;
  B->half_off.assign(B->GL, 0);
  B->half_cnt.assign(B->GL, 0);
  B->full_off.assign(B->GL, 0);
  B->full_cnt.assign(B->GL, 0);
  for (int gl = 0; gl < B->GL; ++gl) {
    B->half_off[gl] = (int)all.size();
    for (int i = 0; i < B->count; ++i) {
      int l = gl - B->gl0[i];
      if (l < 0) continue;
      const Lev& L = B->lev[i * kMaxLevels + l];
      add_items(all, i, l, L.m / 2, L.n, B->tile_x[gl], B->tile_y[gl]);
    }
    B->half_cnt[gl] = (int)all.size() - B->half_off[gl];
    B->full_off[gl] = (int)all.size();
    for (int i = 0; i < B->count; ++i) {
      int l = gl - B->gl0[i];
      if (l < 1) continue;   // coarse-level items: restriction / tau / prolongation / phi^k
      const Lev& L = B->lev[i * kMaxLevels + l];
      add_items(all, i, l, L.m, L.n, kPTX, kPTY);
    }
    B->full_cnt[gl] = (int)all.size() - B->full_off[gl];
  }
  B->fin_off = (int)all.size();
  std::vector<int> ibeg(B->count + 1, 0);
  for (int i = 0; i < B->count; ++i) {
    ibeg[i] = (int)all.size() - B->fin_off;
    const Lev& L = B->lev[i * kMaxLevels];
    add_items(all, i, 0, L.m, L.n, kPTX, kPTY);
  }
  ibeg[B->count] = (int)all.size() - B->fin_off;
  B->fin_cnt = (int)all.size() - B->fin_off;
  if (all.size() > B->items_cap) return MPFC_ERR_WORKSPACE;
  BCK(cudaMemcpyAsync(B->d_items, all.data(), all.size() * sizeof(BItem), cudaMemcpyHostToDevice, B->stream));
  BCK(cudaMemcpyAsync(B->d_ibeg, ibeg.data(), ibeg.size() * sizeof(int), cudaMemcpyHostToDevice, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  return MPFC_OK;
}

// Upper bound of the number of work items for any smoother tile of >= 64 threads:
// ceil(a/tx) ceil(b/ty) <= ab/64 + a + b + 1 for the a x b half domain, plus the
// 32 x 8 tiles of the full domains (coarse-level list and the finest-level list).
size_t max_items(const std::vector<mpfc_params>& each, int coarsest) {
  size_t n = 0;
  for (const auto& p : each) {
    int L = mpfc_num_levels(p.m, p.n, coarsest);
    size_t m = p.m, nn = p.n;
    for (int l = 0; l < L; ++l) {
      size_t a = m / 2, b = nn;
      n += a * b / 64 + a + b + 1;
      n += 2 * (((m + kPTX - 1) / kPTX) * ((nn + kPTY - 1) / kPTY));
      m /= 2;
      nn /= 2;
    }
  }
  return n + 64;
}

size_t carve_batch(mpfc_batch_s* B, int count, const mpfc_params* each, char* base) {
  BCarver c{base, 0};
  int GL = 0;
  std::vector<int> nl(count);
  for (int i = 0; i < count; ++i) {
    nl[i] = mpfc_num_levels(each[i].m, each[i].n, each[i].coarsest);
    GL = std::max(GL, nl[i]);
  }
  std::vector<mpfc_params> ev(each, each + count);
  size_t nitems = max_items(ev, each[0].coarsest);
  Lev* d_lev = c.take<Lev>((size_t)count * kMaxLevels);
  Coef* d_c1 = c.take<Coef>((size_t)count * kMaxLevels);
  Coef* d_c2 = c.take<Coef>((size_t)count * kMaxLevels);
  SourceArgs* d_s1 = c.take<SourceArgs>(count);
  SourceArgs* d_s2 = c.take<SourceArgs>(count);
  int* d_nlev = c.take<int>(count);
  long long* d_K3off = c.take<long long>(count);
  double* d_inv_s = c.take<double>(count);
  double** d_state = c.take<double*>((size_t)3 * count);
  BCtl* d_ctl = c.take<BCtl>(count);
  BGlobal* d_glob = c.take<BGlobal>(1);
  double* d_partials = c.take<double>(nitems);
  BItem* d_items = c.take<BItem>(nitems);
  int* d_ibeg = c.take<int>((size_t)count + 1);
  size_t k3tot = 0;
  std::vector<long long> k3off(count);
  for (int i = 0; i < count; ++i) {
    int mc = each[i].m >> (nl[i] - 1), nc = each[i].n >> (nl[i] - 1);
    k3off[i] = (long long)k3tot;
    k3tot += 2 * (size_t)mc * nc * mc * nc;   // K3 and c L (mpfc_coarse_block)
  }
  float* d_K3a = c.take<float>(k3tot);
  float* d_K3b = c.take<float>(k3tot);
  if (B && base) {
    B->d_lev = d_lev;
    B->d_coef[0] = d_c1;
    B->d_coef[1] = d_c2;
    B->d_src[0] = d_s1;
    B->d_src[1] = d_s2;
    B->d_nlev = d_nlev;
    B->d_K3off = d_K3off;
    B->d_inv_s = d_inv_s;
    B->d_state = d_state;
    B->d_ctl = d_ctl;
    B->d_glob = d_glob;
    B->d_partials = d_partials;
    B->d_items = d_items;
    B->d_ibeg = d_ibeg;
    B->items_cap = nitems;
    B->d_K3[0] = d_K3a;
    B->d_K3[1] = d_K3b;
    B->GL = GL;
    B->nlev = nl;
    B->gl0.resize(count);
    B->lev.assign((size_t)count * kMaxLevels, Lev{});
    B->state.resize((size_t)3 * count);
    for (int i = 0; i < count; ++i) B->gl0[i] = GL - nl[i];
  }
  for (int i = 0; i < count; ++i) {
    size_t G0 = (size_t)each[i].m * each[i].n;
    double* phik = c.take<double>(G0);
    double* phikm1 = c.take<double>(G0);
    double* psik = c.take<double>(G0);
    int m = each[i].m, n = each[i].n;
    double h = each[i].h;
    for (int l = 0; l < nl[i]; ++l) {
      size_t G = (size_t)m * n;
      Lev v;
      v.m = m;
      v.n = n;
      v.nyn = 0;   // batches are periodic and unpinned
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
      if (B && base) B->lev[(size_t)i * kMaxLevels + l] = v;
      m /= 2;
      n /= 2;
      h *= 2.0;
    }
    if (B && base) {
      B->state[3 * i] = phik;
      B->state[3 * i + 1] = phikm1;
      B->state[3 * i + 2] = psik;
    }
  }
  return c.off;
}

template <int SCH>
void enqueue_batch_vcycle(mpfc_batch_s* B, cudaStream_t s) {
  const int S = SCH - 1;
  const mpfc_params& p = B->p0;
  auto smooth = [&](int gl, int sweeps) {
    int n = B->half_cnt[gl];
    if (n == 0) return;
    dim3 blk(B->tile_x[gl], B->tile_y[gl]);
    for (int sw = 0; sw < sweeps; ++sw)
      for (int color = 0; color < 2; ++color)
        kb_smooth<SCH><<<grid_for_items(n), blk, 0, s>>>(B->d_items + B->half_off[gl], n, B->d_lev, B->d_coef[S],
                                                         B->d_ctl, color);
  };
  const dim3 blk2(kPTX, kPTY);
  for (int gl = 0; gl < B->GL - 1; ++gl) {
    smooth(gl, p.nu1);
    int n = B->full_cnt[gl + 1];
    if (n) {
      kb_restrict<SCH><<<grid_for_items(n), blk2, 0, s>>>(B->d_items + B->full_off[gl + 1], n, B->d_lev,
                                                           B->d_coef[S], B->d_ctl);
      kb_tau<SCH><<<grid_for_items(n), blk2, 0, s>>>(B->d_items + B->full_off[gl + 1], n, B->d_lev, B->d_coef[S],
                                                      B->d_ctl);
    }
  }
  int Gc = 0;
  for (int i = 0; i < B->count; ++i) {
    const Lev& C = B->lev[i * kMaxLevels + B->nlev[i] - 1];
    Gc = std::max(Gc, C.m * C.n);
  }
  size_t smem = sizeof(double) * 7 * (size_t)Gc + sizeof(float) * ((size_t)Gc * (Gc + 1) + (size_t)Gc);
  kb_coarse<SCH><<<B->count, 32, smem, s>>>(B->d_lev, B->d_coef[S], B->d_nlev, B->d_K3[S], B->d_K3off, B->d_ctl);
  for (int gl = B->GL - 2; gl >= 0; --gl) {
    int n = B->full_cnt[gl + 1];
    if (n) kb_prolong<<<grid_for_items(n), blk2, 0, s>>>(B->d_items + B->full_off[gl + 1], n, B->d_lev, B->d_ctl);
    smooth(gl, p.nu2);
  }
}

template <int SCH>
void enqueue_batch_resnorm(mpfc_batch_s* B, int mode, cudaGraphConditionalHandle hnd, int set_cond, cudaStream_t s) {
  kb_resnorm<SCH><<<grid_for_items(B->fin_cnt), dim3(kPTX, kPTY), 0, s>>>(
      B->d_items + B->fin_off, B->fin_cnt, B->d_ibeg, B->count, B->d_lev, B->d_coef[SCH - 1], B->d_ctl, B->d_glob,
      B->d_partials, mode, hnd, set_cond);
}

template <int SCH>
void enqueue_batch_prologue(mpfc_batch_s* B, cudaStream_t s) {
  const dim3 blk2(kPTX, kPTY);
  int nb = (B->count + 127) / 128;
  kb_step_begin<<<nb, 128, 0, s>>>(B->d_ctl, B->count);
  const BItem* fin = B->d_items + B->fin_off;
  int g = grid_for_items(B->fin_cnt);
  kb_source<SCH><<<g, blk2, 0, s>>>(fin, B->fin_cnt, B->d_lev, B->d_src[SCH - 1], B->d_ctl);
  if (SCH == 2)
    for (int gl = 1; gl < B->GL; ++gl) {
      int n = B->full_cnt[gl];
      if (n)
        kb_restrict_pk<<<grid_for_items(n), blk2, 0, s>>>(B->d_items + B->full_off[gl], n, B->d_lev, B->d_ctl);
    }
  kb_guess<SCH><<<g, blk2, 0, s>>>(fin, B->fin_cnt, B->d_lev, B->d_coef[SCH - 1], B->d_ctl, 0);
  kb_guess<SCH><<<g, blk2, 0, s>>>(fin, B->fin_cnt, B->d_lev, B->d_coef[SCH - 1], B->d_ctl, 1);
}

template <int SCH>
void enqueue_batch_commit(mpfc_batch_s* B, cudaStream_t s) {
  const BItem* fin = B->d_items + B->fin_off;
  kb_commit<SCH><<<grid_for_items(B->fin_cnt), dim3(kPTX, kPTY), 0, s>>>(
      fin, B->fin_cnt, B->d_lev, B->d_inv_s, B->p0.model == MPFC_MODEL_PFC, B->d_state, B->d_ctl, B->d_glob);
  kb_step_end<<<(B->count + 127) / 128, 128, 0, s>>>(B->d_ctl, B->d_glob, B->count);
}

template <int SCH>
int build_batch_graph(mpfc_batch_s* B) {
  cudaStream_t cs = B->cap;
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  BCKCAP(cudaStreamGetCaptureInfo(cs, &st, nullptr, &graph, &deps, nullptr, &ndeps), cs);
  cudaGraphConditionalHandle hnd;
  BCKCAP(cudaGraphConditionalHandleCreate(&hnd, graph, 0, 0), cs);
  enqueue_batch_prologue<SCH>(B, cs);
  enqueue_batch_resnorm<SCH>(B, 0, hnd, 1, cs);
  BCKCAP(cudaStreamGetCaptureInfo(cs, &st, nullptr, &graph, &deps, nullptr, &ndeps), cs);
  std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = hnd;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  BCKCAP(cudaGraphAddNode(&cnode, graph, dv.data(), nullptr, dv.size(), &cp), cs);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  BCKCAP(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies), cs);
  BCKCAP(cudaStreamBeginCaptureToGraph(B->body, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal), cs);
  enqueue_batch_vcycle<SCH>(B, B->body);
  enqueue_batch_resnorm<SCH>(B, 1, hnd, 1, B->body);
  cudaError_t e = cudaStreamEndCapture(B->body, &body);
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "cudaStreamEndCapture(batch WHILE body)", __FILE__, __LINE__);
    mpfc_abort_capture(B->body);
    mpfc_abort_capture(cs);
    return MPFC_ERR_CUDA;
  }
  enqueue_batch_commit<SCH>(B, cs);
  BCK(cudaStreamEndCapture(cs, &graph));
  cudaGraphExec_t exec;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "cudaGraphInstantiate(batch step graph)", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  B->exec[SCH - 1] = exec;
  return MPFC_OK;
}

void drop_graphs(mpfc_batch_s* B) {
  for (int s = 0; s < 2; ++s)
    if (B->exec[s]) {
      cudaGraphExecDestroy(B->exec[s]);
      B->exec[s] = nullptr;
    }
}

}  // namespace

extern "C" size_t mpfc_batch_workspace_bytes(int count, const mpfc_params* each) {
  if (count < 1 || !each) return 0;
  for (int i = 0; i < count; ++i) {
    if (mpfc_workspace_bytes(&each[i]) == 0) return 0;
    if (!same_solver_settings(each[i], each[0]) || each[i].precision != MPFC_FP64 ||
        each[i].guess == MPFC_GUESS_LEARNED || each[i].bc != MPFC_BC_PERIODIC || each[i].pinning)
      return 0;
  }
  return carve_batch(nullptr, count, each, nullptr);
}

extern "C" int mpfc_batch_create(int count, const mpfc_params* each, void* d_workspace, size_t bytes,
                                 void* cuda_stream, mpfc_batch_t** out) {
  if (!out) return MPFC_ERR_INVALID;
  *out = nullptr;
  size_t need = mpfc_batch_workspace_bytes(count, each);
  if (need == 0) return MPFC_ERR_INVALID;
  if (!d_workspace || bytes < need || ((uintptr_t)d_workspace & 255)) return MPFC_ERR_WORKSPACE;
  mpfc_batch_s* B = new mpfc_batch_s();
  B->count = count;
  B->each.assign(each, each + count);
  B->p0 = each[0];
  B->stream = (cudaStream_t)cuda_stream;
  B->ws = (char*)d_workspace;
  B->ws_need = need;
  carve_batch(B, count, each, (char*)d_workspace);
  int rc = MPFC_OK;
  do {
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&B->body, cudaStreamNonBlocking)) != cudaSuccess) {
      mpfc_set_cuda_error(e, "cudaStreamCreate", __FILE__, __LINE__);
      rc = MPFC_ERR_CUDA;
      break;
    }
    B->tile_x.assign(B->GL, 32);
    B->tile_y.assign(B->GL, 8);
    for (int s = 0; s < 2; ++s) {
      B->coef[s].assign((size_t)count * kMaxLevels, Coef{});
      B->src[s].resize(count);
    }
    std::vector<long long> k3off(count);
    std::vector<double> inv_s(count);
    std::vector<float> K3all[2];
    long long k3tot = 0;
    for (int i = 0; i < count; ++i) {
      const mpfc_params& p = each[i];
      for (int s = 0; s < 2; ++s)
        for (int l = 0; l < B->nlev[i]; ++l)
          B->coef[s][(size_t)i * kMaxLevels + l] = mpfc_coef(&p, s + 1, B->lev[(size_t)i * kMaxLevels + l].h, 4);
      for (int s = 0; s < 2; ++s) {
        SourceArgs& A = B->src[s][i];
        A.phik = B->state[3 * i];
        A.phikm1 = B->state[3 * i + 1];
        A.psik = B->state[3 * i + 2];
        A.psi_coef = (p.model == MPFC_MODEL_PFC) ? 0.0 : (s == 0) ? 1.0 / (p.beta + 1.0 / p.dt) : 2.0 / (p.beta + 2.0 / p.dt);
        A.half_alpha = 0.5 * (1.0 - p.epsilon);
        A.W = nullptr;
        A.phihat = nullptr;
        A.guess = (p.guess == MPFC_GUESS_PREV) ? 0 : 1;
      }
      inv_s[i] = 1.0 / p.dt;
      k3off[i] = k3tot;
      const Lev& C = B->lev[(size_t)i * kMaxLevels + B->nlev[i] - 1];
      for (int s = 0; s < 2; ++s) {
        std::vector<float> blk;
        mpfc_coarse_block(C, B->coef[s][(size_t)i * kMaxLevels + B->nlev[i] - 1], blk);
        K3all[s].insert(K3all[s].end(), blk.begin(), blk.end());
      }
      k3tot += 2LL * C.m * C.n * C.m * C.n;
    }
    BGlobal g0;
    memset(&g0, 0, sizeof(g0));
    g0.max_cycles = B->p0.max_cycles;
    g0.tol = B->p0.tol;
    std::vector<BCtl> c0(count);
    memset(c0.data(), 0, sizeof(BCtl) * count);
    cudaStream_t s = B->stream;
    if ((e = cudaMemcpyAsync(B->d_lev, B->lev.data(), sizeof(Lev) * B->lev.size(), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_coef[0], B->coef[0].data(), sizeof(Coef) * B->coef[0].size(),
                             cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_coef[1], B->coef[1].data(), sizeof(Coef) * B->coef[1].size(),
                             cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_src[0], B->src[0].data(), sizeof(SourceArgs) * count, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_src[1], B->src[1].data(), sizeof(SourceArgs) * count, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_nlev, B->nlev.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_K3off, k3off.data(), sizeof(long long) * count, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_inv_s, inv_s.data(), sizeof(double) * count, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_state, B->state.data(), sizeof(double*) * 3 * count, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_ctl, c0.data(), sizeof(BCtl) * count, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_glob, &g0, sizeof(g0), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(B->d_K3[0], K3all[0].data(), sizeof(float) * K3all[0].size(), cudaMemcpyHostToDevice,
                             s)) ||
        (e = cudaMemcpyAsync(B->d_K3[1], K3all[1].data(), sizeof(float) * K3all[1].size(), cudaMemcpyHostToDevice,
                             s)) ||
        (e = cudaStreamSynchronize(s))) {
      mpfc_set_cuda_error(e, "batch tables", __FILE__, __LINE__);
      rc = MPFC_ERR_CUDA;
      break;
    }
    for (int i = 0; i < count && rc == MPFC_OK; ++i) {
      size_t bytes0 = (size_t)each[i].m * each[i].n * sizeof(double);
      for (int k = 0; k < 3; ++k)
        if ((e = cudaMemsetAsync(B->state[3 * i + k], 0, bytes0, s)) != cudaSuccess) {
          mpfc_set_cuda_error(e, "batch state", __FILE__, __LINE__);
          rc = MPFC_ERR_CUDA;
        }
    }
    if (rc == MPFC_OK) rc = build_items(B);
  } while (0);
  if (rc != MPFC_OK) {
    mpfc_batch_destroy(B);
    return rc;
  }
  *out = B;
  return MPFC_OK;
}

extern "C" void mpfc_batch_destroy(mpfc_batch_t* B) {
  if (!B) return;
  drop_graphs(B);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->body) cudaStreamDestroy(B->body);
  delete B;
}

extern "C" int mpfc_batch_set_state(mpfc_batch_t* B, int inst, const double* phi, const double* phi_prev,
                                    const double* psi) {
  if (!B || inst < 0 || inst >= B->count || !phi) return MPFC_ERR_INVALID;
  size_t bytes = (size_t)B->each[inst].m * B->each[inst].n * sizeof(double);
  BCK(cudaMemcpyAsync(B->state[3 * inst], phi, bytes, cudaMemcpyDefault, B->stream));
  BCK(cudaMemcpyAsync(B->state[3 * inst + 1], phi_prev ? phi_prev : phi, bytes, cudaMemcpyDefault, B->stream));
  if (psi) BCK(cudaMemcpyAsync(B->state[3 * inst + 2], psi, bytes, cudaMemcpyDefault, B->stream));
  else BCK(cudaMemsetAsync(B->state[3 * inst + 2], 0, bytes, B->stream));
  return MPFC_OK;
}

extern "C" int mpfc_batch_get_state(mpfc_batch_t* B, int inst, double* phi, double* phi_prev, double* psi) {
  if (!B || inst < 0 || inst >= B->count) return MPFC_ERR_INVALID;
  size_t bytes = (size_t)B->each[inst].m * B->each[inst].n * sizeof(double);
  if (phi) BCK(cudaMemcpyAsync(phi, B->state[3 * inst], bytes, cudaMemcpyDefault, B->stream));
  if (phi_prev) BCK(cudaMemcpyAsync(phi_prev, B->state[3 * inst + 1], bytes, cudaMemcpyDefault, B->stream));
  if (psi) BCK(cudaMemcpyAsync(psi, B->state[3 * inst + 2], bytes, cudaMemcpyDefault, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  return MPFC_OK;
}

static int batch_run(mpfc_batch_s* B, int scheme, int nsteps, int fixed, int* statuses, int* cycles, bool sync) {
  if (!B || (scheme != 1 && scheme != 2) || nsteps < 0) return MPFC_ERR_INVALID;
  if (!B->exec[scheme - 1]) {
    int rc = scheme == 1 ? build_batch_graph<1>(B) : build_batch_graph<2>(B);
    if (rc != MPFC_OK) return rc;
  }
  kb_reset<<<(B->count + 127) / 128, 128, 0, B->stream>>>(B->d_ctl, B->d_glob, B->count, fixed);
  BCK(cudaGetLastError());
  for (int k = 0; k < nsteps; ++k) {
    MpfcRange range("mpfc batch step");
    BCK(cudaGraphLaunch(B->exec[scheme - 1], B->stream));
  }
  if (!sync) return MPFC_OK;
  std::vector<BCtl> c(B->count);
  BCK(cudaMemcpyAsync(c.data(), B->d_ctl, sizeof(BCtl) * B->count, cudaMemcpyDeviceToHost, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  int first = MPFC_OK;
  for (int i = 0; i < B->count; ++i) {
    if (statuses) statuses[i] = c[i].first_error;
    if (cycles) cycles[i] = c[i].total_cycles;
    if (c[i].first_error != 0 && first == MPFC_OK) first = c[i].first_error;
  }
  return first;
}

extern "C" int mpfc_batch_step(mpfc_batch_t* B, int scheme, int nsteps, int* statuses, int* cycles) {
  return batch_run(B, scheme, nsteps, 0, statuses, cycles, true);
}

extern "C" int mpfc_batch_step_cycles(mpfc_batch_t* B, int scheme, int ncycles, int* statuses) {
  if (ncycles < 1) return MPFC_ERR_INVALID;
  return batch_run(B, scheme, 1, ncycles, statuses, nullptr, true);
}

extern "C" int mpfc_batch_levels(const mpfc_batch_t* B) { return B ? B->GL : 0; }

extern "C" int mpfc_batch_set_tile(mpfc_batch_t* B, int level, int tx, int ty) {
  if (!B || level < 0 || level >= B->GL || tx < 1 || ty < 1 || tx * ty > 1024 || tx * ty < 64 || (tx * ty) % 32)
    return MPFC_ERR_INVALID;
  B->tile_x[level] = tx;
  B->tile_y[level] = ty;
  drop_graphs(B);
  return build_items(B);
}

extern "C" int mpfc_batch_time_smooth(mpfc_batch_t* B, int scheme, int level, int reps, float* ms) {
  if (!B || level < 0 || level >= B->GL || reps < 1 || !ms || (scheme != 1 && scheme != 2)) return MPFC_ERR_INVALID;
  int n = B->half_cnt[level];
  *ms = 0.f;
  if (n == 0) return MPFC_OK;
  // all instances active for the measurement
  kb_step_begin<<<(B->count + 127) / 128, 128, 0, B->stream>>>(B->d_ctl, B->count);
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  dim3 blk(B->tile_x[level], B->tile_y[level]);
  const BItem* it = B->d_items + B->half_off[level];
  for (int w = 0; w < 2; ++w) {
    BCK(cudaEventRecord(e0, B->stream));
    for (int r = 0; r < reps; ++r)
      for (int color = 0; color < 2; ++color) {
        if (scheme == 1)
          kb_smooth<1><<<grid_for_items(n), blk, 0, B->stream>>>(it, n, B->d_lev, B->d_coef[0], B->d_ctl, color);
        else
          kb_smooth<2><<<grid_for_items(n), blk, 0, B->stream>>>(it, n, B->d_lev, B->d_coef[1], B->d_ctl, color);
      }
    BCK(cudaEventRecord(e1, B->stream));
    BCK(cudaEventSynchronize(e1));
  }
  BCK(cudaEventElapsedTime(ms, e0, e1));
  *ms /= reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BCK(cudaGetLastError());
  return MPFC_OK;
}
