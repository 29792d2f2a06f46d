// The coarse end of the FP64 V-cycle in one launch: one CTA (LD = kLdPlain) or one
// thread-block cluster (LD = kLdL2) runs the whole sub-cycle from a small level down to
// the coarsest solve and back up (the FAS V-cycle of App. B, in the order of the
// per-level launches: nu1 red-black sweeps, restriction with the tau correction,
// recursion, prolongation, nu2 sweeps).  Phases are separated by __syncthreads or
// cluster barriers with release/acquire semantics instead of kernel boundaries, and
// every cell is computed by the same per-cell functions as the per-level kernels, so the
// results are bit for bit those of the per-level launches.  On GB300 a small level's
// launch costs more than its work; this kernel replaces eleven launches per level.
// Included by fp64_kernels.cuh inside namespace mpfc.
#pragma once

constexpr int kMaxTail = 8;         // levels one tail launch can cover
constexpr int kTailThreads = 256;   // threads per CTA (of the CTA, or of each CTA of the cluster)

struct TailLev {
  Lev L;
  Coef k, kb;   // interior and Neumann-row cell systems of the level
};

struct TailArgs {
  int nlev;        // levels covered, the last one the coarsest
  int nu1, nu2;    // pre- and post-sweeps
  const float* K3f;
  TailLev lv[kMaxTail];
};

// LD == kLdL2: all threads of all CTAs of the cluster, after this thread's writes:
// release them to the cluster and acquire those of the others (the loads that follow go
// to L2).  LD == kLdPlain: one CTA, __syncthreads.
template <int LD>
__device__ __forceinline__ void tail_barrier() {
  if (LD == kLdL2) asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
  else __syncthreads();
}

template <int SCH, int LD>
__device__ __forceinline__ void tail_half_sweep(const TailLev& T, int color, int tid, int nth) {
  const int half = T.L.m >> 1, cells = half * T.L.n;
  for (int t = tid; t < cells; t += nth) {
    const int j = t / half, x = t - j * half;
    smooth_cell<SCH, LD>(T.L, T.k, T.kb, 2 * x + ((j + color) & 1), j);
  }
}

// Every thread of the launch runs the same sequence of barriers: no thread leaves
// early, and the coarsest solve (one warp of CTA 0) sits between two barriers.
template <int SCH, int LD>
__global__ void __launch_bounds__(kTailThreads, 1) k_tail(const __grid_constant__ TailArgs A) {
  extern __shared__ double tail_sm[];
  pdl_enter();
  const int nth = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int l = 0; l < A.nlev - 1; ++l) {
    const TailLev& F = A.lv[l];
    const TailLev& C = A.lv[l + 1];
    for (int sw = 0; sw < A.nu1; ++sw)
      for (int color = 0; color < 2; ++color) {
        tail_half_sweep<SCH, LD>(F, color, tid, nth);
        tail_barrier<LD>();
      }
    const int cc = C.L.m * C.L.n;
    for (int t = tid; t < cc; t += nth) resid_restrict_cell<SCH, LD>(F.L, C.L, F.k, 1, t % C.L.m, t / C.L.m);
    tail_barrier<LD>();
    for (int t = tid; t < cc; t += nth) tau_cell<SCH, LD>(C.L, C.k, t % C.L.m, t / C.L.m);
    tail_barrier<LD>();
  }
  const TailLev& Cc = A.lv[A.nlev - 1];
  if (blockIdx.x == 0 && threadIdx.x < 32) coarse_solve_warp<SCH, LD>(Cc.L, Cc.k, A.K3f, tail_sm);
  tail_barrier<LD>();
  for (int l = A.nlev - 2; l >= 0; --l) {
    const TailLev& F = A.lv[l];
    const Lev& C = A.lv[l + 1].L;
    const int fc = F.L.m * F.L.n;
    for (int t = tid; t < fc; t += nth) {
      const int fi = t % F.L.m, fj = t / F.L.m;
      prolong_fine_plane<LD>(C.phi, C.b1, F.L.phi, C.m, C.n, C.nyn, fi, fj);
      prolong_fine_plane<LD>(C.mu, C.b2, F.L.mu, C.m, C.n, C.nyn, fi, fj);
      prolong_fine_plane<LD>(C.ka, C.b3, F.L.ka, C.m, C.n, C.nyn, fi, fj);
    }
    tail_barrier<LD>();
    for (int sw = 0; sw < A.nu2; ++sw)
      for (int color = 0; color < 2; ++color) {
        tail_half_sweep<SCH, LD>(F, color, tid, nth);
        tail_barrier<LD>();
      }
  }
}
