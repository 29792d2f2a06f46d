// FP64 kernels of the FAS V-cycle for the MPFC convex-splitting schemes.
//
// Every kernel works on one level of SoA planes (row-major [n][m], periodic wrap by
// index arithmetic, App. A (A.8)-(A.9)).  On GB300 the FP64 pipe issues about 1.6
// DFMA per clock per SM, so these kernels are bound by FP64 instruction issue, not
// by HBM: they keep loads simple (L1-cached neighbour reads) and spend their effort
// on the FP64 instruction count per cell.
#pragma once

#include "mpfc_common.cuh"

namespace mpfc {
// Non-template kernels are static: several translation units include this header.

// ---------------------------------------------------------------------------
// Source S and initial guess (App. B.1 / B.2; guess: extrapolation of phi, then
// kappa and mu chosen so that rows 2 and 3 of N(u) = S hold exactly).
// ---------------------------------------------------------------------------
struct SourceArgs {
  const double* phik;
  const double* phikm1;
  const double* psik;
  const double* W;       // pinning weight (scheme 2), nullptr: none
  const double* phihat;  // pinning target
  double psi_coef;   // 1/(beta+1/s) (scheme 1) or 2/(beta+2/s) (scheme 2)
  double half_alpha; // alpha/2 (scheme 2)
  int guess;         // 0 prev, 1 extrapolated, 2 given in L.phi already
};

template <int SCH>
__device__ __forceinline__ void source_cell(const Lev& L, const SourceArgs& A, int i, int j) {
  int m = L.m;
  int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, L.n, L.nyn), jp = ywrap(j + 1, L.n, L.nyn);
  size_t c = (size_t)j * m + i;
  size_t w = (size_t)j * m + im, e = (size_t)j * m + ip, s = (size_t)jm * m + i, nn = (size_t)jp * m + i;
  double ih2 = 1.0 / (L.h * L.h);
  const double* pk = A.phik;
  double p0 = pk[c];
  double lap_k = ((pk[w] + pk[e]) + (pk[s] + pk[nn]) - 4.0 * p0) * ih2;
  double q0 = A.phikm1[c];
  if (SCH == 1) {
    L.S1[c] = p0 + A.psi_coef * A.psik[c];
    L.S2[c] = 2.0 * lap_k;
    L.S3[c] = 0.0;
  } else {
    const double* pm = A.phikm1;
    // phitilde = (3 phik - phikm1)/2 at the five points, then Delta_h of it
    double t0 = 0.5 * (3.0 * p0 - q0);
    double tw = 0.5 * (3.0 * pk[w] - pm[w]), te = 0.5 * (3.0 * pk[e] - pm[e]);
    double ts = 0.5 * (3.0 * pk[s] - pm[s]), tn = 0.5 * (3.0 * pk[nn] - pm[nn]);
    double lap_t = ((tw + te) + (ts + tn) - 4.0 * t0) * ih2;
    L.S1[c] = p0 + A.psi_coef * A.psik[c];
    // pinning (Sec. 4.6): 2 W (phi^{k+1/2} - phihat) minus its part W phi in N gives W (phi^k - 2 phihat)
    L.S2[c] = A.half_alpha * p0 + 2.0 * lap_t + (A.W ? A.W[c] * (p0 - 2.0 * A.phihat[c]) : 0.0);
    L.S3[c] = 0.5 * lap_k;
  }
  if (A.guess == 0) L.phi[c] = p0;
  else if (A.guess == 1) L.phi[c] = 2.0 * p0 - q0;
}

template <int SCH>
__global__ void k_source_guess(Lev L, SourceArgs A) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= L.m || j >= L.n) return;
  source_cell<SCH>(L, A, i, j);
}

// kappa0 = S3 + theta Delta_h phi0
__device__ __forceinline__ void guess_kappa_cell(const Lev& L, const Coef& k, int i, int j) {
  int m = L.m;
  int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, L.n, L.nyn), jp = ywrap(j + 1, L.n, L.nyn);
  size_t c = (size_t)j * m + i;
  const double* f = L.phi;
  double sum = (f[(size_t)j * m + im] + f[(size_t)j * m + ip]) + (f[(size_t)jm * m + i] + f[(size_t)jp * m + i]);
  L.ka[c] = L.S3[c] + k.th2 * (sum - 4.0 * f[c]);
}

static __global__ void k_guess_kappa(Lev L, Coef k) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= L.m || j >= L.n) return;
  guess_kappa_cell(L, k, i, j);
}

// mu0 = S2 + g(phi0) + gam phi0 + Delta_h kappa0
template <int SCH>
__device__ __forceinline__ void guess_mu_cell(const Lev& L, const Coef& k, int i, int j) {
  int m = L.m;
  int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, L.n, L.nyn), jp = ywrap(j + 1, L.n, L.nyn);
  size_t c = (size_t)j * m + i;
  const double* f = L.ka;
  double sum = (f[(size_t)j * m + im] + f[(size_t)j * m + ip]) + (f[(size_t)jm * m + i] + f[(size_t)jp * m + i]);
  double p = L.phi[c];
  double pk = (SCH == 2) ? L.pk[c] : 0.0;
  double gam = (SCH == 2 && L.W) ? k.gam + L.W[c] : k.gam;   // pinning weight joins gam (Sec. 4.6)
  L.mu[c] = L.S2[c] + g_of<SCH>(p, pk) + gam * p + k.ih2 * (sum - 4.0 * f[c]);
}

template <int SCH>
__global__ void k_guess_mu(Lev L, Coef k) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= L.m || j >= L.n) return;
  guess_mu_cell<SCH>(L, k, i, j);
}

#include "fp64_smooth.cuh"

// ---------------------------------------------------------------------------
// Residual r = S - N(u) at one cell (App. B.1 / B.2 operator N).
// ---------------------------------------------------------------------------
template <int SCH>
__device__ __forceinline__ void resid_at(const Lev& L, const Coef& k, int i, int j, double& r1, double& r2,
                                         double& r3) {
  int m = L.m;
  int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, L.n, L.nyn), jp = ywrap(j + 1, L.n, L.nyn);
  size_t c = (size_t)j * m + i;
  size_t w = (size_t)j * m + im, e = (size_t)j * m + ip, s = (size_t)jm * m + i, nn = (size_t)jp * m + i;
  const double* phi = L.phi;
  const double* mu = L.mu;
  const double* ka = L.ka;
  double p = __ldg(phi + c), u = __ldg(mu + c), v = __ldg(ka + c);
  double smu = (__ldg(mu + w) + __ldg(mu + e)) + (__ldg(mu + s) + __ldg(mu + nn));
  double ska = (__ldg(ka + w) + __ldg(ka + e)) + (__ldg(ka + s) + __ldg(ka + nn));
  double sph = (__ldg(phi + w) + __ldg(phi + e)) + (__ldg(phi + s) + __ldg(phi + nn));
  double pk = (SCH == 2) ? __ldg(L.pk + c) : 0.0;
  // r1 = S1 - phi + c Delta_h mu
  r1 = fma(k.cmu, fma(-4.0, u, smu), __ldg(L.S1 + c) - p);
  // r2 = S2 - mu + g(phi) + gam phi + Delta_h kappa
  double gam = (SCH == 2 && L.W) ? k.gam + __ldg(L.W + c) : k.gam;
  r2 = fma(k.ih2, fma(-4.0, v, ska), fma(gam, p, __ldg(L.S2 + c) - u) + g_of<SCH>(p, pk));
  // r3 = S3 - kappa + theta Delta_h phi
  r3 = fma(k.th2, fma(-4.0, p, sph), __ldg(L.S3 + c) - v);
}

template <int SCH>
__global__ void k_residual(Lev L, Coef k, double* r1, double* r2, double* r3) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= L.m || j >= L.n) return;
  double a, b, c;
  resid_at<SCH>(L, k, i, j, a, b, c);
  size_t id = (size_t)j * L.m + i;
  r1[id] = a;
  r2[id] = b;
  r3[id] = c;
}

// ---------------------------------------------------------------------------
// FAS restriction, part 1: per coarse cell, the 2x2 averages of u and of the
// fine residual.  u_c = R u (also kept in b), S_c = R r (part 2 adds N_c(u_c)).
// ---------------------------------------------------------------------------
// Summed over a 2x2 block B of fine cells, the five-point Laplacian needs no per-cell
// evaluation: each cell of B is an inner neighbour of two others, so
//   sum_{c in B} Delta_h f(c) = (sum of the 8 cells bordering B - 2 sum_{c in B} f) / h^2.
// The restricted residual R r = (1/4) sum_B (S - N(u)) therefore takes the block sums
// of S, u and of the Laplacians, plus the per-cell nonlinear term (and the pinning
// term), instead of four full residual evaluations.
template <int SCH, int LD = kLdNC>
__device__ __forceinline__ void resid_restrict_cell(const Lev& F, const Lev& C, const Coef& kf, int keep_b, int I,
                                                    int J) {
  const int m = F.m, i0 = 2 * I, j0 = 2 * J;
  const int iw = wrapm(i0 - 1, m), ie = wrapm(i0 + 2, m);
  const int js = ywrap(j0 - 1, F.n, F.nyn), jn = ywrap(j0 + 2, F.n, F.nyn);
  const size_t r0 = (size_t)j0 * m, r1 = r0 + m, rs = (size_t)js * m, rn = (size_t)jn * m;
  // block sum and the sum over the 8 bordering cells of one field
  auto sums = [&](const double* f, double& blk, double& outer) {
    blk = (ldv<LD>(f + r0 + i0) + ldv<LD>(f + r0 + i0 + 1)) + (ldv<LD>(f + r1 + i0) + ldv<LD>(f + r1 + i0 + 1));
    outer = ((ldv<LD>(f + r0 + iw) + ldv<LD>(f + r1 + iw)) + (ldv<LD>(f + r0 + ie) + ldv<LD>(f + r1 + ie))) +
            ((ldv<LD>(f + rs + i0) + ldv<LD>(f + rs + i0 + 1)) + (ldv<LD>(f + rn + i0) + ldv<LD>(f + rn + i0 + 1)));
  };
  double sp, op, sm, om, sk, ok;
  sums(F.phi, sp, op);
  sums(F.mu, sm, om);
  sums(F.ka, sk, ok);
  double gs = 0.0;   // sum of the per-cell nonlinear term (and pinning term) of row 2
#pragma unroll
  for (int dj = 0; dj < 2; ++dj)
#pragma unroll
    for (int di = 0; di < 2; ++di) {
      const size_t id = (dj ? r1 : r0) + i0 + di;
      const double p = ldv<LD>(F.phi + id);
      const double pk = (SCH == 2) ? ldv<LD>(F.pk + id) : 0.0;
      gs += g_of<SCH>(p, pk);
      if (SCH == 2 && F.W) gs = fma(ldv<LD>(F.W + id), p, gs);
    }
  const double ss1 = (ldv<LD>(F.S1 + r0 + i0) + ldv<LD>(F.S1 + r0 + i0 + 1)) +
                     (ldv<LD>(F.S1 + r1 + i0) + ldv<LD>(F.S1 + r1 + i0 + 1));
  const double ss2 = (ldv<LD>(F.S2 + r0 + i0) + ldv<LD>(F.S2 + r0 + i0 + 1)) +
                     (ldv<LD>(F.S2 + r1 + i0) + ldv<LD>(F.S2 + r1 + i0 + 1));
  const double ss3 = (ldv<LD>(F.S3 + r0 + i0) + ldv<LD>(F.S3 + r0 + i0 + 1)) +
                     (ldv<LD>(F.S3 + r1 + i0) + ldv<LD>(F.S3 + r1 + i0 + 1));
  // sum_B r1 = sum S1 - sum phi + c sum Delta_h mu, and likewise rows 2 and 3
  const double sr1 = fma(kf.cmu, fma(-2.0, sm, om), ss1 - sp);
  const double sr2 = fma(kf.ih2, fma(-2.0, sk, ok), fma(kf.gam, sp, ss2 - sm) + gs);
  const double sr3 = fma(kf.th2, fma(-2.0, sp, op), ss3 - sk);
  size_t cid = (size_t)J * C.m + I;
  double up = 0.25 * sp, um = 0.25 * sm, uk = 0.25 * sk;
  C.phi[cid] = up;
  C.mu[cid] = um;
  C.ka[cid] = uk;
  if (keep_b) {
    C.b1[cid] = up;
    C.b2[cid] = um;
    C.b3[cid] = uk;
  }
  C.S1[cid] = 0.25 * sr1;
  C.S2[cid] = 0.25 * sr2;
  C.S3[cid] = 0.25 * sr3;
}

template <int SCH>
__global__ void k_resid_restrict(Lev F, Lev C, Coef kf, int keep_b) {
  pdl_enter();
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= C.m || J >= C.n) return;
  resid_restrict_cell<SCH>(F, C, kf, keep_b, I, J);
}

// The same restriction with four threads per coarse cell, for small levels, where a
// launch lasts about the FP64 latency of one thread's chain (a warp-wide FP64
// instruction holds its sub-partition's pipe for some 80 cycles, however many lanes are
// active).  Lanes 4c .. 4c+3 of a warp serve one coarse cell: lane q < 3 forms the block
// and border sums of field q (phi, mu, kappa) and the block sum of S_{q+1}; lane q loads
// the values of fine cell q = 2 dj + di of the block, and every lane sums the nonlinear
// term of the four in order; the partner lanes' sums, shuffled in, then give lane q row
// q + 1 of the restricted residual.  Each sum keeps the association of
// resid_restrict_cell, so the bits are the same.  Blocks are one warp (32 x 1); lane 3
// and quads past the grid compute on clamped indices and write nothing (the shuffles
// take the whole warp).
template <int SCH>
__global__ void __launch_bounds__(32) k_resid_restrict4(Lev F, Lev C, Coef kf, int keep_b) {
  pdl_enter();
  const unsigned FULL = 0xffffffffu;
  const int q = threadIdx.x & 3, base = threadIdx.x & ~3;
  const int Iq = (blockIdx.x * 32 + threadIdx.x) >> 2, J = blockIdx.y;
  const bool live = Iq < C.m && q < 3;
  const int I = Iq < C.m ? Iq : C.m - 1;
  const int m = F.m, i0 = 2 * I, j0 = 2 * J;
  const int iw = wrapm(i0 - 1, m), ie = wrapm(i0 + 2, m);
  const int js = ywrap(j0 - 1, F.n, F.nyn), jn = ywrap(j0 + 2, F.n, F.nyn);
  const size_t r0 = (size_t)j0 * m, r1 = r0 + m, rs = (size_t)js * m, rn = (size_t)jn * m;
  const double* f = q == 1 ? F.mu : q == 2 ? F.ka : F.phi;
  const double* S = q == 1 ? F.S2 : q == 2 ? F.S3 : F.S1;
  const double blk = (__ldg(f + r0 + i0) + __ldg(f + r0 + i0 + 1)) + (__ldg(f + r1 + i0) + __ldg(f + r1 + i0 + 1));
  const double outer = ((__ldg(f + r0 + iw) + __ldg(f + r1 + iw)) + (__ldg(f + r0 + ie) + __ldg(f + r1 + ie))) +
                       ((__ldg(f + rs + i0) + __ldg(f + rs + i0 + 1)) + (__ldg(f + rn + i0) + __ldg(f + rn + i0 + 1)));
  const double ss = (__ldg(S + r0 + i0) + __ldg(S + r0 + i0 + 1)) + (__ldg(S + r1 + i0) + __ldg(S + r1 + i0 + 1));
  // the nonlinear sum written exactly as in resid_restrict_cell (an addition of the cubic,
  // which the compiler may fuse with the cubic's last product, so the form must match),
  // from the four cells' values loaded one per lane
  const size_t idq = ((q & 2) ? r1 : r0) + i0 + (q & 1);
  const double pq = __ldg(F.phi + idq);
  const double pkq = (SCH == 2) ? __ldg(F.pk + idq) : 0.0;
  const double wq = (SCH == 2 && F.W) ? __ldg(F.W + idq) : 0.0;
  double gs = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double p = __shfl_sync(FULL, pq, base + c);
    const double pk = (SCH == 2) ? __shfl_sync(FULL, pkq, base + c) : 0.0;
    gs += g_of<SCH>(p, pk);
    if (SCH == 2 && F.W) gs = fma(__shfl_sync(FULL, wq, base + c), p, gs);
  }
  // row q + 1 takes the block and border sums of field (q + 1) mod 3, row 2 also phi's
  // block sum:
  //   sr1 = cmu (om - 2 sm) + (ss1 - sp)
  //   sr2 = ih2 (ok - 2 sk) + ((gam sp + (ss2 - sm)) + gs)
  //   sr3 = th2 (op - 2 sp) + (ss3 - sk)
  const int nxt = base + (q == 0 ? 1 : q == 1 ? 2 : 0);
  const double X = __shfl_sync(FULL, blk, nxt), Y = __shfl_sync(FULL, outer, nxt);
  const double sp = __shfl_sync(FULL, blk, base);
  const double z0 = ss - blk;
  const double Z = (q == 1) ? fma(kf.gam, sp, z0) + gs : z0;
  const double cq = q == 0 ? kf.cmu : q == 1 ? kf.ih2 : kf.th2;
  const double sr = fma(cq, fma(-2.0, X, Y), Z);
  if (!live) return;
  const size_t cid = (size_t)J * C.m + I;
  const double u = 0.25 * blk;
  (q == 0 ? C.phi : q == 1 ? C.mu : C.ka)[cid] = u;
  if (keep_b) (q == 0 ? C.b1 : q == 1 ? C.b2 : C.b3)[cid] = u;
  (q == 0 ? C.S1 : q == 1 ? C.S2 : C.S3)[cid] = 0.25 * sr;
}

// FAS restriction, part 2: S_c += N_c(u_c).
template <int SCH, int LD = kLdNC>
__device__ __forceinline__ void tau_cell(const Lev& C, const Coef& k, int i, int j) {
  int m = C.m;
  int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, C.n, C.nyn), jp = ywrap(j + 1, C.n, C.nyn);
  size_t c = (size_t)j * m + i;
  size_t w = (size_t)j * m + im, e = (size_t)j * m + ip, s = (size_t)jm * m + i, nn = (size_t)jp * m + i;
  const double* phi = C.phi;
  const double* mu = C.mu;
  const double* ka = C.ka;
  double p = ldown<LD>(phi + c), u = ldown<LD>(mu + c), v = ldown<LD>(ka + c);
  double smu = (ldown<LD>(mu + w) + ldown<LD>(mu + e)) + (ldown<LD>(mu + s) + ldown<LD>(mu + nn));
  double ska = (ldown<LD>(ka + w) + ldown<LD>(ka + e)) + (ldown<LD>(ka + s) + ldown<LD>(ka + nn));
  double sph = (ldown<LD>(phi + w) + ldown<LD>(phi + e)) + (ldown<LD>(phi + s) + ldown<LD>(phi + nn));
  double pk = (SCH == 2) ? ldown<LD>(C.pk + c) : 0.0;
  double N1 = fma(-k.cmu, fma(-4.0, u, smu), p);
  double gam = (SCH == 2 && C.W) ? k.gam + ldown<LD>(C.W + c) : k.gam;
  double N2 = fma(-k.ih2, fma(-4.0, v, ska), fma(-gam, p, u) - g_of<SCH>(p, pk));
  double N3 = fma(-k.th2, fma(-4.0, p, sph), v);
  C.S1[c] = ldown<LD>(C.S1 + c) + N1;
  C.S2[c] = ldown<LD>(C.S2 + c) + N2;
  C.S3[c] = ldown<LD>(C.S3 + c) + N3;
}

template <int SCH>
__global__ void k_tau(Lev C, Coef k) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= C.m || j >= C.n) return;
  tau_cell<SCH>(C, k, i, j);
}

// Plain 2x2 average of one plane (phi^k onto the coarse levels, scheme 2).
static __global__ void k_restrict_plane(const double* __restrict__ f, double* __restrict__ c, int mc, int nc) {
  pdl_enter();
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= mc || J >= nc) return;
  int mf = 2 * mc;
  size_t a = (size_t)(2 * J) * mf + 2 * I, b = a + mf;
  c[(size_t)J * mc + I] = 0.25 * ((f[a] + f[a + 1]) + (f[b] + f[b + 1]));
}

// ---------------------------------------------------------------------------
// FAS correction: u_f += P(u_c - b_c), P the cell-centred bilinear stencil
// (9, 3, 3, 1)/16.  One thread per coarse cell writes its 2x2 fine children.
// ---------------------------------------------------------------------------
struct ProlongArgs {
  const double *cphi, *cmu, *cka;   // coarse u after the coarse solve
  const double *ophi, *omu, *oka;   // coarse R u_f before it
  double *fphi, *fmu, *fka;         // fine u (in/out)
  int mc, nc;
  int nyn;                          // Neumann rule in y (ghost coarse row = boundary row)
};

// One thread per coarse cell; the block first stages e = u_c - b_c of all three
// components on its (32+2) x (8+2) coarse tile (periodic halo) in shared memory, so
// each difference is formed once and the three tiles load together, then writes the
// bilinear correction into its 2x2 fine children.
constexpr int kPTX = 32, kPTY = 8;
using ProlongTile = double[3][kPTY + 2][kPTX + 2];

__device__ __forceinline__ void prolong_apply(double (*E)[kPTX + 2], double* __restrict__ f, int mc, int I, int J) {
  int x = threadIdx.x + 1, y = threadIdx.y + 1;
  double e00 = E[y][x];
  double eW = E[y][x - 1], eE = E[y][x + 1], eS = E[y - 1][x], eN = E[y + 1][x];
  double eSW = E[y - 1][x - 1], eSE = E[y - 1][x + 1], eNW = E[y + 1][x - 1], eNE = E[y + 1][x + 1];
  const double w9 = 9.0 / 16.0, w3 = 3.0 / 16.0, w1 = 1.0 / 16.0;
  int mf = 2 * mc;
  size_t f00 = (size_t)(2 * J) * mf + 2 * I;
  size_t f01 = f00 + mf;
  double c9 = w9 * e00;
  f[f00] += fma(w3, eW + eS, fma(w1, eSW, c9));
  f[f00 + 1] += fma(w3, eE + eS, fma(w1, eSE, c9));
  f[f01] += fma(w3, eW + eN, fma(w1, eNW, c9));
  f[f01 + 1] += fma(w3, eE + eN, fma(w1, eNE, c9));
}

// The block's (kPTX x kPTY) coarse tile at (I0, J0): all three components.  A caller
// that stages another tile into E afterwards synchronises the block first.
__device__ __forceinline__ void prolong_tile(const ProlongArgs& A, ProlongTile& E, int I0, int J0) {
  for (int t = threadIdx.y * kPTX + threadIdx.x; t < (kPTX + 2) * (kPTY + 2); t += kPTX * kPTY) {
    int ty = t / (kPTX + 2), tx = t % (kPTX + 2);
    int I = wrapm(I0 + tx - 1, A.mc), J = ywrap(J0 + ty - 1, A.nc, A.nyn);
    if (I0 + tx - 1 < A.mc + 1 && J0 + ty - 1 < A.nc + 1) {
      size_t id = (size_t)J * A.mc + I;
      E[0][ty][tx] = __ldg(A.cphi + id) - __ldg(A.ophi + id);
      E[1][ty][tx] = __ldg(A.cmu + id) - __ldg(A.omu + id);
      E[2][ty][tx] = __ldg(A.cka + id) - __ldg(A.oka + id);
    }
  }
  __syncthreads();
  int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
  if (I < A.mc && J < A.nc) {
    prolong_apply(E[0], A.fphi, A.mc, I, J);
    prolong_apply(E[1], A.fmu, A.mc, I, J);
    prolong_apply(E[2], A.fka, A.mc, I, J);
  }
}

static __global__ void __launch_bounds__(kPTX * kPTY) k_prolong(ProlongArgs A) {
  pdl_enter();
  __shared__ ProlongTile E;
  prolong_tile(A, E, blockIdx.x * kPTX, blockIdx.y * kPTY);
}

// The same correction at one fine cell (fi, fj), for kernels without the shared-memory
// tile: the four coarse differences it needs are formed in place, and the weights are
// applied in the tile version's order, so both give the same bits.
template <int LD>
__device__ __forceinline__ void prolong_fine_plane(const double* cn, const double* co, double* f, int mc, int nc, int nyn,
                                                   int fi, int fj) {
  const int I = fi >> 1, J = fj >> 1;
  const int Ix = wrapm(I + ((fi & 1) ? 1 : -1), mc), Jy = ywrap(J + ((fj & 1) ? 1 : -1), nc, nyn);
  const size_t c00 = (size_t)J * mc + I, cx = (size_t)J * mc + Ix, cy = (size_t)Jy * mc + I, cxy = (size_t)Jy * mc + Ix;
  const double e00 = ldown<LD>(cn + c00) - ldown<LD>(co + c00), ex = ldown<LD>(cn + cx) - ldown<LD>(co + cx);
  const double ey = ldown<LD>(cn + cy) - ldown<LD>(co + cy), exy = ldown<LD>(cn + cxy) - ldown<LD>(co + cxy);
  const double w9 = 9.0 / 16.0, w3 = 3.0 / 16.0, w1 = 1.0 / 16.0;
  const size_t id = (size_t)fj * (2 * mc) + fi;
  f[id] = ldown<LD>(f + id) + fma(w3, ex + ey, fma(w1, exy, w9 * e00));
}

// The correction with one thread per fine cell (its three components), for small levels:
// a thread's chain is about half the FP64 instructions of a coarse cell's thread in
// k_prolong, over four times the threads.  Same bits as k_prolong.
static __global__ void k_prolong_fine(ProlongArgs A) {
  pdl_enter();
  const int fi = blockIdx.x * blockDim.x + threadIdx.x, fj = blockIdx.y * blockDim.y + threadIdx.y;
  if (fi >= 2 * A.mc || fj >= 2 * A.nc) return;
  prolong_fine_plane<kLdPlain>(A.cphi, A.ophi, A.fphi, A.mc, A.nc, A.nyn, fi, fj);
  prolong_fine_plane<kLdPlain>(A.cmu, A.omu, A.fmu, A.mc, A.nc, A.nyn, fi, fj);
  prolong_fine_plane<kLdPlain>(A.cka, A.oka, A.fka, A.mc, A.nc, A.nyn, fi, fj);
}

// ---------------------------------------------------------------------------
// Coarsest level: Newton on the eliminated equation for phi,
//   F(phi) = phi - c L (S2 + g(phi) + gam phi + L (S3 + theta L phi)) - S1 = 0,
// with Jacobian J = K3 - c L diag(gam + g'(phi)), K3 = I - c theta L^3 and c L built
// on the host (mpfc_coarse_block).  FP32 elimination on one warp (registers up to 31
// cells, shared memory up to 64).  Stops once the applied update is below
// 1e-15 (1 + |phi|_inf); at most 40 iterations.  mu and kappa are then recovered from
// rows 3 and 2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double nbsum_s(const double* f, int m, int n, int t, int nyn) {
  int i = t % m, j = t / m;
  return (f[j * m + wrapm(i - 1, m)] + f[j * m + wrapm(i + 1, m)]) +
         (f[ywrap(j - 1, n, nyn) * m + i] + f[ywrap(j + 1, n, nyn) * m + i]);
}

// Gauss-Jordan elimination with implicit partial pivoting, one column of the augmented
// matrix per lane held in registers (R register rows, R >= G; lanes past the augmented
// columns hold zeros).  Column col (col < G): the lane that holds it picks the unused
// row of largest magnitude, every lane divides its entry of that row by the pivot and
// subtracts multiples of it from all other rows.  No row is moved: afterwards row
// pivs[col] holds a 1 in column col and the lanes' other columns are transformed alike
// (pivs: G ints of shared scratch).
template <int R>
__device__ __forceinline__ void gj_eliminate(float (&a)[R], int G, int* pivs) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned used = 0u;
  for (int col = 0; col < G; ++col) {
    float best = -1.f;
    int pr = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float v = fabsf(a[r]);
      if (r < G && !((used >> r) & 1u) && v > best) {
        best = v;
        pr = r;
      }
    }
    pr = __shfl_sync(FULL, pr, col);
    float vp = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (r == pr) vp = a[r];
    const float rp = 1.f / __shfl_sync(FULL, vp, col);
    const float vn = vp * rp;   // this lane's entry of the normalised pivot row
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float f = __shfl_sync(FULL, a[r], col);
      a[r] = (r == pr) ? vn : fmaf(-f, vn, a[r]);
    }
    used |= 1u << pr;
    if (lane == 0) pivs[col] = pr;
  }
  __syncwarp();
}

// [J | rhs] with the right-hand side in lane G: eliminates and writes the solution to
// x[0..G); xr (G floats) and pivs (G ints) are shared scratch.
template <int R>
__device__ __forceinline__ void gauss_jordan_cols(float (&a)[R], int G, float* x, float* xr, int* pivs) {
  const int lane = threadIdx.x & 31;
  gj_eliminate<R>(a, G, pivs);
  if (lane == G)
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (r < G) xr[r] = a[r];
  __syncwarp();
  for (int t = lane; t < G; t += 32) x[t] = xr[pivs[t]];
  __syncwarp();
}

// The Newton iteration on the coarsest grid.  R > 0: grids of at most min(R, 31)
// cells, one Jacobian column per lane in R registers (gauss_jordan_cols); R == 0:
// up to 64 cells, Gaussian elimination with row swaps in shared memory.
template <int SCH, int R, int LD>
__device__ void coarse_newton(const Lev& C, const Coef& k, const float* __restrict__ K3f, double* sm) {
  const int m = C.m, n = C.n, G = m * n, W = G + 1;
  double* ph = sm;
  double* s1 = ph + G;
  double* s2 = s1 + G;
  double* s3 = s2 + G;
  double* pk = s3 + G;
  double* kap = pk + G;
  double* muv = kap + G;
  float* Jm = reinterpret_cast<float*>(muv + G);   // G x (G+1), last column = right-hand side
  float* d = Jm + G * W;
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  for (int t = lane; t < G; t += 32) {
    ph[t] = ldown<LD>(C.phi + t);
    s1[t] = ldown<LD>(C.S1 + t);
    s2[t] = ldown<LD>(C.S2 + t);
    s3[t] = ldown<LD>(C.S3 + t);
    pk[t] = (SCH == 2) ? ldown<LD>(C.pk + t) : 0.0;
  }
  __syncwarp();
  const float gamf = (float)k.gam;
  constexpr int RR = R > 0 ? R : 1;
  float k3c[RR], lcc[RR];   // this lane's column of K3 and of c L (register path)
  const float* cLf = K3f + G * G;   // c L, after K3 in the coarse block
  if (R > 0) {
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      k3c[r] = (lane < G && r < G) ? K3f[r * G + lane] : 0.f;
      lcc[r] = (lane < G && r < G) ? cLf[r * G + lane] : 0.f;
    }
  }
  auto kappa_at = [&](int t) { return s3[t] + k.th2 * (nbsum_s(ph, m, n, t, C.nyn) - 4.0 * ph[t]); };
  auto mu_at = [&](int t) {
    return s2[t] + g_of<SCH>(ph[t], pk[t]) + (k.gam + (C.W ? C.W[t] : 0.0)) * ph[t] +
           k.ih2 * (nbsum_s(kap, m, n, t, C.nyn) - 4.0 * kap[t]);
  };
  bool refactor = true;   // chord path: eliminate J again at this iteration
  float dprev = 0.f;
  for (int it = 0; it < 40; ++it) {
    for (int t = lane; t < G; t += 32) kap[t] = kappa_at(t);
    __syncwarp();
    for (int t = lane; t < G; t += 32) muv[t] = mu_at(t);
    __syncwarp();
    if (R == 16) {
      // Chord iteration with a lagged Jacobian (grids of at most 16 cells): Gauss-Jordan
      // on [J | I] over the 32 lanes gives X with J^-1 = rows pivs[.] of X; it is redone
      // only when the updates stop shrinking by 100x per iteration, and each iteration
      // costs an FP64 residual and a product with J^-1.  Xs (G x G) and the right-hand
      // side rh share Jm; pivs lives in d once d has been read.
      float* Xs = Jm;
      float* rh = Jm + G * G;
      int* pivs = reinterpret_cast<int*>(d);
      for (int t = lane; t < G; t += 32)
        rh[t] = (float)(s1[t] - ph[t] + k.cmu * (nbsum_s(muv, m, n, t, C.nyn) - 4.0 * muv[t]));
      if (refactor) {
        for (int t = lane; t < G; t += 32) d[t] = gamf + (float)((C.W ? C.W[t] : 0.0) + dg_of<SCH>(ph[t], pk[t]));
        __syncwarp();
        float a[16];
        const float dc = lane < G ? d[lane] : 0.f;
#pragma unroll
        for (int r = 0; r < 16; ++r)
          a[r] = lane < G ? fmaf(-lcc[r], dc, k3c[r]) : ((lane < 2 * G && lane - G == r) ? 1.f : 0.f);
        __syncwarp();   // d is free from here: pivot indices
        gj_eliminate<16>(a, G, pivs);
        if (lane >= G && lane < 2 * G)
#pragma unroll
          for (int r = 0; r < 16; ++r)
            if (r < G) Xs[r * G + (lane - G)] = a[r];
      }
      __syncwarp();
      float delta = 0.f;
      if (lane < G) {
        const float* xrow = Xs + pivs[lane] * G;
        for (int q = 0; q < G; ++q) delta = fmaf(xrow[q], rh[q], delta);
      }
      float dmax = fabsf(delta);
      double umax = 0.0;
      if (lane < G) {
        const double pn = ph[lane] + (double)delta;
        ph[lane] = pn;
        umax = fabs(pn);
      }
      for (int o = 16; o > 0; o >>= 1) {
        dmax = fmaxf(dmax, __shfl_xor_sync(FULL, dmax, o));
        umax = fmax(umax, __shfl_xor_sync(FULL, umax, o));
      }
      __syncwarp();
      if (!(dmax == dmax) || (double)dmax <= 1e-15 * (1.0 + umax)) break;
      refactor = it > 0 && !(dmax <= 0.01f * dprev);
      dprev = dmax;
      continue;
    }
    for (int t = lane; t < G; t += 32)
      Jm[t * W + G] = (float)(s1[t] - ph[t] + k.cmu * (nbsum_s(muv, m, n, t, C.nyn) - 4.0 * muv[t]));
    // the diagonal factor gam + W + g'(phi) of each column, once per column
    for (int t = lane; t < G; t += 32) d[t] = gamf + (float)((C.W ? C.W[t] : 0.0) + dg_of<SCH>(ph[t], pk[t]));
    __syncwarp();
    if (R > 0) {
      // J = K3 - c L diag(d): this lane's column, or the right-hand side in lane G
      float a[RR];
      const float dc = lane < G ? d[lane] : 0.f;
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        const float rhs = (lane == G && r < G) ? Jm[r * W + G] : 0.f;
        a[r] = lane < G ? fmaf(-lcc[r], dc, k3c[r]) : rhs;
      }
      __syncwarp();   // Jm is free from here: pivot scratch
      gauss_jordan_cols<RR>(a, G, d, Jm + G, reinterpret_cast<int*>(Jm));
    } else {
      for (int idx = lane; idx < G * G; idx += 32) {
        int r = idx / G, col = idx % G;
        Jm[r * W + col] = K3f[idx] - cLf[idx] * d[col];
      }
      __syncwarp();
      for (int col = 0; col < G; ++col) {
        float best = -1.f;
        int piv = col;
        for (int r = col + lane; r < G; r += 32) {
          float v = fabsf(Jm[r * W + col]);
          if (v > best) { best = v; piv = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          float ob = __shfl_down_sync(FULL, best, o);
          int op = __shfl_down_sync(FULL, piv, o);
          if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
        }
        piv = __shfl_sync(FULL, piv, 0);
        if (piv != col)
          for (int c2 = col + lane; c2 <= G; c2 += 32) {
            float t = Jm[col * W + c2];
            Jm[col * W + c2] = Jm[piv * W + c2];
            Jm[piv * W + c2] = t;
          }
        __syncwarp();
        float rp = 1.f / Jm[col * W + col];
        for (int r = col + 1 + lane; r < G; r += 32) {
          float f = Jm[r * W + col] * rp;
          for (int c2 = col + 1; c2 <= G; ++c2) Jm[r * W + c2] = fmaf(-f, Jm[col * W + c2], Jm[r * W + c2]);
        }
        __syncwarp();
      }
      for (int r = G - 1; r >= 0; --r) {
        float acc = 0.f;
        for (int c2 = r + 1 + lane; c2 < G; c2 += 32) acc = fmaf(Jm[r * W + c2], d[c2], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(FULL, acc, o);
        if (lane == 0) d[r] = (Jm[r * W + G] - acc) / Jm[r * W + r];
        __syncwarp();
      }
    }
    float dmax = 0.f;
    double umax = 0.0;
    for (int t = lane; t < G; t += 32) {
      double pn = ph[t] + (double)d[t];
      ph[t] = pn;
      dmax = fmaxf(dmax, fabsf(d[t]));
      umax = fmax(umax, fabs(pn));
    }
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmaxf(dmax, __shfl_xor_sync(FULL, dmax, o));
      umax = fmax(umax, __shfl_xor_sync(FULL, umax, o));
    }
    __syncwarp();
    // the update just applied was below 1e-15 (1 + |phi|_inf): converged to roundoff
    if (!(dmax == dmax) || (double)dmax <= 1e-15 * (1.0 + umax)) break;
  }
  for (int t = lane; t < G; t += 32) kap[t] = kappa_at(t);
  __syncwarp();
  for (int t = lane; t < G; t += 32) {
    muv[t] = mu_at(t);
    C.phi[t] = ph[t];
    C.ka[t] = kap[t];
    C.mu[t] = muv[t];
  }
}

// One warp.  Newton's method for F(phi) = 0 with F evaluated in FP64; the Jacobian
// is assembled, factorised and solved in FP32, i.e. Newton with iterative refinement:
// every update is computed from the FP64 residual, so the iteration converges to the
// FP64 root.  FP32 keeps the elimination off the slow FP64 pipe (on GB300 one
// warp-wide FP64 instruction occupies a sub-partition's FP64 unit for about 80 cycles).
// Called by one warp (the others of the block must not wait on it).  LD: how the
// level's planes are read (kLdL2 inside a cluster kernel).
template <int SCH, int LD = kLdPlain>
__device__ void coarse_solve_warp(const Lev& C, const Coef& k, const float* __restrict__ K3f, double* sm) {
  const int G = C.m * C.n;
  if (G <= 16) coarse_newton<SCH, 16, LD>(C, k, K3f, sm);
  else if (G <= 31) coarse_newton<SCH, 32, LD>(C, k, K3f, sm);
  else coarse_newton<SCH, 0, LD>(C, k, K3f, sm);
}

template <int SCH>
__device__ void coarse_solve_block(const Lev& C, const Coef& k, const float* __restrict__ K3f) {
  extern __shared__ double sm[];
  if (threadIdx.x >= 32) return;
  coarse_solve_warp<SCH, kLdPlain>(C, k, K3f, sm);
}

template <int SCH>
__global__ void k_coarse_solve(Lev C, Coef k, const float* __restrict__ K3f) {
  pdl_enter();
  coarse_solve_block<SCH>(C, k, K3f);
}

// ---------------------------------------------------------------------------
// Deterministic reductions: per-block partial sums (fixed tree), then the last
// block to finish adds the partials in index order.
// ---------------------------------------------------------------------------
template <int NS>
__device__ __forceinline__ void block_sum(double (&v)[NS], double* red /* NS * 32 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[s] += __shfl_down_sync(0xffffffffu, v[s], o);
  if (lane == 0)
#pragma unroll
    for (int s = 0; s < NS; ++s) red[s * 32 + wid] = v[s];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double x = lane < nw ? red[s * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[s] = x;
    }
  }
}

// Returns true in the one thread (thread 0 of the last block) that holds the
// totals in v after the call.
template <int NS>
__device__ __forceinline__ bool grid_sum(double (&v)[NS], double* partials, unsigned int* counter) {
  __shared__ double red[NS * 32];
  __shared__ bool last;
  block_sum<NS>(v, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) partials[s * kMaxPartials + blockIdx.x] = v[s];
    __threadfence();
    unsigned int done = atomicAdd(counter, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double w[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    w[s] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) w[s] += ((volatile double*)partials)[s * kMaxPartials + b];
  }
  block_sum<NS>(w, red);
  if (threadIdx.x == 0) {
    *counter = 0u;
#pragma unroll
    for (int s = 0; s < NS; ++s) v[s] = w[s];
    return true;
  }
  return false;
}

// The V-cycle loop decision from the scaled residual norm res (one thread).
// mode 0: after the initial guess (sets res0); mode 1: after a V-cycle.
__device__ __forceinline__ void resnorm_decide(Ctl* ctl, double res, int mode, cudaGraphConditionalHandle hnd,
                                               int set_cond) {
  int cond;
  if (mode == 0) {
    ctl->res0 = res;
    ctl->res = res;
    ctl->cycles = 0;
    ctl->status = 0;
  } else {
    ctl->res = res;
    ctl->cycles += 1;
    if (!(res == res) || isinf(res) || res > 1e10 * fmax(ctl->res0, ctl->tol)) ctl->status = 2;
  }
  if (ctl->skip || ctl->status != 0) cond = 0;
  else if (ctl->fixed_cycles > 0) cond = ctl->cycles < ctl->fixed_cycles;
  else cond = (res > ctl->tol) && (ctl->cycles < ctl->max_cycles);
  if (mode == 0 && (!(res == res) || isinf(res))) { ctl->status = 2; cond = 0; }
  if (set_cond) cudaGraphSetConditional(hnd, cond ? 1u : 0u);
}

// Row 1 of the residual alone, r1 = S1 - phi + c Delta_h mu (as in resid_at).
__device__ __forceinline__ double resid1_at(const Lev& L, const Coef& k, int i, int j) {
  const int m = L.m;
  const int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, L.n, L.nyn), jp = ywrap(j + 1, L.n, L.nyn);
  const size_t c = (size_t)j * m + i;
  const double* mu = L.mu;
  const double smu = (__ldg(mu + (size_t)j * m + im) + __ldg(mu + (size_t)j * m + ip)) +
                     (__ldg(mu + (size_t)jm * m + i) + __ldg(mu + (size_t)jp * m + i));
  return fma(k.cmu, fma(-4.0, __ldg(mu + c), smu), __ldg(L.S1 + c) - __ldg(L.phi + c));
}

// Scaled residual norm at the finest level, and the V-cycle loop decision.  R1ONLY:
// right after the initial guess, whose kappa and mu are defined by rows 3 and 2 of
// N(u) = S (those residuals are rounding, below the norm's resolution), only row 1.
template <int SCH, bool R1ONLY = false>
__global__ void __launch_bounds__(256) k_resnorm(Lev L, Coef k, Ctl* ctl, double* partials, int mode,
                                                 cudaGraphConditionalHandle hnd, int set_cond) {
  pdl_enter();
  double v[1] = {0.0};
  int G = L.m * L.n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < G; t += gridDim.x * blockDim.x) {
    int i = t % L.m, j = t / L.m;
    if (R1ONLY) {
      const double a = resid1_at(L, k, i, j);
      v[0] = fma(a, a, v[0]);
      continue;
    }
    double a, b, c;
    resid_at<SCH>(L, k, i, j, a, b, c);
    v[0] = fma(a, a, fma(b, b, fma(c, c, v[0])));
  }
  if (!grid_sum<1>(v, partials, &ctl->counter)) return;
  resnorm_decide(ctl, sqrt(v[0] / (3.0 * (double)G)), mode, hnd, set_cond);
}

// The same after a V-cycle whose last half sweep was k_smooth_res: the residual of the
// red cells ((i + j) even), plus the nb per-warp sums that k_smooth_res left in bpart
// for the black ones, each added by a fixed thread, so the total does not depend on
// timing.
template <int SCH>
__global__ void __launch_bounds__(256) k_resnorm_red(Lev L, Coef k, Ctl* ctl, double* partials, const double* bpart,
                                                     int nb, cudaGraphConditionalHandle hnd, int set_cond) {
  pdl_enter();
  double v[1] = {0.0};
  const int half = L.m >> 1, G = L.m * L.n, nth = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int t = tid; t < half * L.n; t += nth) {
    const int j = t / half, i = 2 * (t - j * half) + (j & 1);
    double a, b, c;
    resid_at<SCH>(L, k, i, j, a, b, c);
    v[0] = fma(a, a, fma(b, b, fma(c, c, v[0])));
  }
  for (int t = tid; t < nb; t += nth) v[0] += bpart[t];
  if (!grid_sum<1>(v, partials, &ctl->counter)) return;
  resnorm_decide(ctl, sqrt(v[0] / (3.0 * (double)G)), 1, hnd, set_cond);
}

// ---------------------------------------------------------------------------
// Step bookkeeping and the psi update.
// ---------------------------------------------------------------------------
static __global__ void k_step_begin(Ctl* ctl) {
  pdl_enter();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->skip = ctl->halt;
    ctl->cycles = 0;
    ctl->status = 0;
  }
}

static __global__ void k_ctl_reset(Ctl* ctl, int fixed_cycles) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->halt = 0;
    ctl->slot = 0;
    ctl->fixed_cycles = fixed_cycles;
    ctl->counter = 0u;
  }
}

// Final status of a step: 0 ok, -4 not converged, -5 diverged.
__device__ __forceinline__ int step_status(const Ctl* ctl) {
  if (ctl->status == 2) return -5;
  if (ctl->fixed_cycles <= 0 && !(ctl->res <= ctl->tol)) return -4;
  return 0;
}

// psi^{k+1} = (phi - phi^k)/s (scheme 1, (3.9)) or (2/s)(phi - phi^k) - psi^k
// (scheme 2, (3.15)); then phi^{k-1} <- phi^k, phi^k <- phi.  Skipped for a
// failed or skipped step, which also halts the remaining steps of the call.
template <int SCH>
// pfc: psi keeps the discrete velocity (phi^{k+1} - phi^k)/s (the PFC model has no
// velocity unknown); otherwise (3.9) / (3.15).
__global__ void k_commit(const double* __restrict__ phinew, double* phik, double* phikm1, double* psik,
                         double* phikm2, int G, double inv_s, int pfc, Ctl* ctl, StepRecord* info) {
  pdl_enter();
  int st = step_status(ctl);
  int skip = ctl->skip;
  if (blockIdx.x == 0 && threadIdx.x == 0 && !skip) {
    StepRecord r;
    r.cycles = ctl->cycles;
    r.status = st;
    r.res0 = ctl->res0;
    r.res_final = ctl->res;
    if (ctl->slot < kInfoCap) info[ctl->slot] = r;
    ctl->slot += 1;
    if (st != 0) ctl->halt = 1;
  }
  if (skip || st != 0) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < G; t += gridDim.x * blockDim.x) {
    double pn = phinew[t], p0 = phik[t];
    double ps = (SCH == 1 || pfc) ? (pn - p0) * inv_s : 2.0 * inv_s * (pn - p0) - psik[t];
    psik[t] = ps;
    if (phikm2) phikm2[t] = phikm1[t];
    phikm1[t] = p0;
    phik[t] = pn;
  }
}

// ---------------------------------------------------------------------------
// Diagnostics: mass and energy sums, Poisson multigrid for the -1 norm.
// ---------------------------------------------------------------------------
static __global__ void k_sum1(const double* __restrict__ f, int G, Ctl* ctl, double* partials) {
  double v[1] = {0.0};
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < G; t += gridDim.x * blockDim.x) v[0] += f[t];
  if (grid_sum<1>(v, partials, &ctl->counter)) ctl->sums[0] = v[0];
}

// sums: 0 phi^4, 1 phi^2, 2 |grad phi|^2 (edge differences), 3 (Delta_h phi)^2 h^4,
// 4 psi * xi, 5 |grad (phi - phi_prev)|^2, 6 W (phi - phihat)^2 (pinning, W nullable)
// With the Neumann rule the north edge of the top row has zero difference (ghost =
// boundary row) and the bottom row's south edge is never counted, as App. A's
// Neumann grid has only the n - 1 interior north-south edges.
static __global__ void k_energy_sums(const double* __restrict__ phi, const double* __restrict__ phip,
                              const double* __restrict__ psi, const double* __restrict__ xi, int m, int n, int nyn,
                              const double* __restrict__ W, const double* __restrict__ phat, Ctl* ctl,
                              double* partials) {
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  int G = m * n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < G; t += gridDim.x * blockDim.x) {
    int i = t % m, j = t / m;
    int ip = wrapm(i + 1, m), im = wrapm(i - 1, m), jp = ywrap(j + 1, n, nyn), jm = ywrap(j - 1, n, nyn);
    double p = phi[t];
    double pe = phi[j * m + ip], pw = phi[j * m + im], pn = phi[jp * m + i], ps = phi[jm * m + i];
    double p2 = p * p;
    v[0] += p2 * p2;
    v[1] += p2;
    double dx = pe - p, dy = pn - p;
    v[2] += dx * dx + dy * dy;
    double lap = (pe + pw) + (pn + ps) - 4.0 * p;
    v[3] += lap * lap;
    v[4] += psi[t] * xi[t];
    double d0 = p - phip[t];
    double ddx = (pe - phip[j * m + ip]) - d0, ddy = (pn - phip[jp * m + i]) - d0;
    v[5] += ddx * ddx + ddy * ddy;
    if (W) {
      double dp = p - phat[t];
      v[6] += W[t] * dp * dp;
    }
  }
  if (grid_sum<7>(v, partials, &ctl->counter))
    for (int s = 0; s < 7; ++s) ctl->sums[s] = v[s];
}

// x = f - mean: the right-hand side of the mean-zero Poisson problem
static __global__ void k_sub_mean(const double* __restrict__ f, double* __restrict__ out, int G, const Ctl* ctl) {
  double mean = ctl->sums[0] / (double)G;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < G; t += gridDim.x * blockDim.x) out[t] = f[t] - mean;
}

// Red-black Gauss-Seidel half sweep for -Delta_h x = f (periodic, or Neumann in y:
// a boundary row's ghost is its own unknown, so it has three neighbours).
static __global__ void k_pois_smooth(double* __restrict__ x, const double* __restrict__ f, int m, int n, int nyn,
                                     double h2, int color) {
  int xi = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (xi >= (m >> 1) || j >= n) return;
  int i = 2 * xi + ((j + color) & 1);
  int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, n, nyn), jp = ywrap(j + 1, n, nyn);
  double s = (x[j * m + im] + x[j * m + ip]) + (x[jm * m + i] + x[jp * m + i]);
  if (nyn && (j == 0 || j == n - 1)) {
    s -= x[j * m + i];
    x[j * m + i] = (s + h2 * f[j * m + i]) / 3.0;
  } else {
    x[j * m + i] = 0.25 * (s + h2 * f[j * m + i]);
  }
}

// coarse f = R (f + Delta_h x), coarse x = 0; also the sum of squared fine residuals
static __global__ void k_pois_restrict(const double* __restrict__ x, const double* __restrict__ f, double* __restrict__ fc,
                                double* __restrict__ xc, int mc, int nc, int nyn, double ih2) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= mc || J >= nc) return;
  int m = 2 * mc, n = 2 * nc;
  double acc = 0.0;
  for (int dj = 0; dj < 2; ++dj)
    for (int di = 0; di < 2; ++di) {
      int i = 2 * I + di, j = 2 * J + dj;
      int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, n, nyn), jp = ywrap(j + 1, n, nyn);
      double lap = ((x[j * m + im] + x[j * m + ip]) + (x[jm * m + i] + x[jp * m + i]) - 4.0 * x[j * m + i]) * ih2;
      acc += f[j * m + i] + lap;
    }
  fc[J * mc + I] = 0.25 * acc;
  xc[J * mc + I] = 0.0;
}

static __global__ void k_pois_prolong(const double* __restrict__ xc, double* __restrict__ x, int mc, int nc, int nyn) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= mc || J >= nc) return;
  int Im = wrapm(I - 1, mc), Ip = wrapm(I + 1, mc), Jm = ywrap(J - 1, nc, nyn), Jp = ywrap(J + 1, nc, nyn);
  auto X = [&](int a, int b) { return xc[b * mc + a]; };
  double e00 = X(I, J), eW = X(Im, J), eE = X(Ip, J), eS = X(I, Jm), eN = X(I, Jp);
  double eSW = X(Im, Jm), eSE = X(Ip, Jm), eNW = X(Im, Jp), eNE = X(Ip, Jp);
  const double w9 = 9.0 / 16.0, w3 = 3.0 / 16.0, w1 = 1.0 / 16.0;
  int mf = 2 * mc;
  size_t f00 = (size_t)(2 * J) * mf + 2 * I, f01 = f00 + mf;
  x[f00] += fma(w9, e00, fma(w3, eW + eS, w1 * eSW));
  x[f00 + 1] += fma(w9, e00, fma(w3, eE + eS, w1 * eSE));
  x[f01] += fma(w9, e00, fma(w3, eW + eN, w1 * eNW));
  x[f01 + 1] += fma(w9, e00, fma(w3, eE + eN, w1 * eNE));
}

// Coarsest Poisson level: `sweeps` red-black sweeps in one CTA, then the mean removed.
static __global__ void k_pois_coarse(double* x, const double* f, int m, int n, int nyn, double h2, int sweeps) {
  extern __shared__ double xs[];
  int G = m * n;
  for (int t = threadIdx.x; t < G; t += blockDim.x) xs[t] = x[t];
  __syncthreads();
  for (int s = 0; s < sweeps; ++s)
    for (int color = 0; color < 2; ++color) {
      for (int t = threadIdx.x; t < G; t += blockDim.x) {
        int i = t % m, j = t / m;
        if (((i + j) & 1) != color) continue;
        if (nyn && (j == 0 || j == n - 1)) xs[t] = (nbsum_s(xs, m, n, t, nyn) - xs[t] + h2 * f[t]) / 3.0;
        else xs[t] = 0.25 * (nbsum_s(xs, m, n, t, nyn) + h2 * f[t]);
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) {
    double mean = 0.0;
    for (int t = 0; t < G; ++t) mean += xs[t];
    xs[G] = mean / G;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < G; t += blockDim.x) x[t] = xs[t] - xs[G];
}

// sum of squared residuals of -Delta_h x = f, and sum of f^2
static __global__ void k_pois_resnorm(const double* __restrict__ x, const double* __restrict__ f, int m, int n, int nyn,
                               double ih2, Ctl* ctl, double* partials) {
  double v[2] = {0.0, 0.0};
  int G = m * n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < G; t += gridDim.x * blockDim.x) {
    int i = t % m, j = t / m;
    int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, n, nyn), jp = ywrap(j + 1, n, nyn);
    double lap = ((x[j * m + im] + x[j * m + ip]) + (x[jm * m + i] + x[jp * m + i]) - 4.0 * x[t]) * ih2;
    double r = f[t] + lap;
    v[0] += r * r;
    v[1] += f[t] * f[t];
  }
  if (grid_sum<2>(v, partials, &ctl->counter)) {
    ctl->sums[0] = v[0];
    ctl->sums[1] = v[1];
  }
}

#include "fp64_tail.cuh"

}  // namespace mpfc
