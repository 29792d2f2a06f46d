// The FP64 red-black nonlinear block Gauss-Seidel half sweep (App. B.1 / B.2
// smoothing schemes), kept in its own header: the DRAM traffic recorded for the
// roofline is tied to this file's contents.  Included by fp64_kernels.cuh inside
// namespace mpfc.
#pragma once

// ---------------------------------------------------------------------------
// Red-black nonlinear block Gauss-Seidel half sweep (App. B.1 / B.2 smoothing
// scheme).  Thread (x, j) visits cell i = 2x + ((j + color) & 1) of colour
// `color` (0 = red, (i+j) even).  Cells of one colour only read the other colour,
// so a half sweep is exactly parallel.
//
// The cell's 3x3 system (the cubic linearised about the current value p) is solved for
// the correction d = A^-1 r, with r = S - N(u) the cell's residual at its current values
// (rows 1 and 3 of N are linear; in row 2 the Newton term q p of the linearisation cancels,
// leaving g(p)), and u <- u + omega d.  The result is that of solving A x = R and relaxing
// towards x, but the single-precision-seeded reciprocal's error now scales the correction
// and vanishes with it, so the residual floor is the one the evaluation of r itself sets,
// as in the oracle, at any h.  (Forming kappa from the updated phi through R3 - b3 phi
// instead put the reciprocal's 2^-44 times (4/h^2)(4 theta/h^2) phi into row 2 at the
// fixed point: a residual floor near 6e-10 at h = 1/16.)
// ---------------------------------------------------------------------------
// EDGE: a row next to a Neumann boundary, where the ghost neighbour is the cell's own
// unknown (App. A, (A.7)): it leaves the neighbour sums and k holds the coefficients
// of three neighbours.
struct CellNew {
  double phi, mu, ka;      // updated values
  double R1, R3, X2;       // S1 + c h^-2 sum mu, S3 + theta h^-2 sum phi, S2 + h^-2 sum kappa
  double pk, wv;           // phi^k (scheme 2) and the pinning weight at the cell
};

template <int SCH, bool EDGE, int LD>
__device__ __forceinline__ CellNew cell_update(const Lev& L, const Coef& k, size_t c, size_t w, size_t e, size_t s,
                                               size_t nn) {
  const double* __restrict__ phi = L.phi;
  const double* __restrict__ mu = L.mu;
  const double* __restrict__ ka = L.ka;
  // neighbours belong to the other colour: read-only during this launch
  double smu = (ldv<LD>(mu + w) + ldv<LD>(mu + e)) + (ldv<LD>(mu + s) + ldv<LD>(mu + nn));
  double ska = (ldv<LD>(ka + w) + ldv<LD>(ka + e)) + (ldv<LD>(ka + s) + ldv<LD>(ka + nn));
  double sph = (ldv<LD>(phi + w) + ldv<LD>(phi + e)) + (ldv<LD>(phi + s) + ldv<LD>(phi + nn));
  const double p = ldown<LD>(phi + c), m0 = ldown<LD>(mu + c), k0 = ldown<LD>(ka + c);
  if (EDGE) {   // the ghost was read as the cell's current value: take it out again
    smu -= m0;
    ska -= k0;
    sph -= p;
  }
  CellNew o;
  o.pk = 0.0;
  o.wv = 0.0;
  o.R1 = fma(k.cmu, smu, ldv<LD>(L.S1 + c));
  o.R3 = fma(k.th2, sph, ldv<LD>(L.S3 + c));
  o.X2 = fma(k.ih2, ska, ldv<LD>(L.S2 + c));
  // residual rows: r1 = R1 - phi - a mu, r3 = R3 - b3 phi - kappa,
  // r2 = S2 + h^-2 sum kappa - mu + g(phi) + (gam + W) phi - b kappa
  const double r1 = fma(-k.a, m0, o.R1 - p);
  const double y3 = fma(-k.b3, p, o.R3);
  const double r3 = y3 - k0;
  // t = b r3 - r2 with the b kappa terms of the two rows cancelled:
  //   t = b (R3 - b3 p) + mu - (S2 + h^-2 sum kappa) - g(p) - (gam + W) p
  const double z = fma(k.b, y3, m0 - o.X2);
  // q = g'(p) (+ W) enters the determinant and the Cramer numerator of mu
  double t, detw, Qq;   // detw = det / omega
  if (SCH == 1) {
    const double p2 = p * p;
    t = fma(-k.gam, p, fma(-p2, p, z));   // g = p^3
    detw = fma(k.a3w, p2, k.D0w);         // q = 3 p^2
    Qq = fma(3.0, p2, k.Q0);
  } else {
    o.pk = ldv<LD>(L.pk + c);
    double q = dg_of<2>(p, o.pk);
    if (L.W) {   // pinning: a pointwise linear term of row 2 (gam -> gam + W)
      o.wv = ldv<LD>(L.W + c);
      q += o.wv;
    }
    t = fma(-(k.gam + o.wv), p, z - g_of<2>(p, o.pk));
    detw = fma(k.aw, q, k.D0w);
    Qq = k.Q0 + q;
  }
  // Cramer's rule on [[1, a, 0], [-(gam+q), 1, b], [b3, 0, 1]] d = r:
  //   d_phi = (r1 + a t) / det,  d_mu = ((Q0 + q) r1 - t) / det,  d_kappa = r3 - b3 d_phi;
  // wr = omega / det carries the relaxation
  const double wr = rcp_nr(detw);
  const double dphi = fma(k.a, t, r1) * wr;
  o.phi = p + dphi;
  o.mu = fma(fma(Qq, r1, -t), wr, m0);
  o.ka = fma(-k.b3, dphi, fma(k.omega, r3, k0));
  return o;
}

template <int SCH, bool EDGE, int LD>
__device__ __forceinline__ void smooth_cell_body(const Lev& L, const Coef& k, int i, int j) {
  const int m = L.m;
  const int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, L.n, L.nyn), jp = ywrap(j + 1, L.n, L.nyn);
  const size_t c = (size_t)j * m + i;
  const CellNew o = cell_update<SCH, EDGE, LD>(L, k, c, (size_t)j * m + im, (size_t)j * m + ip, (size_t)jm * m + i,
                                               (size_t)jp * m + i);
  L.phi[c] = o.phi;
  L.mu[c] = o.mu;
  L.ka[c] = o.ka;
}

// The same update, also returning the residual of the cell after it (r1^2 + r2^2 + r3^2),
// for the finest level's last half sweep of a V-cycle (k_smooth_res).  Its neighbours
// belong to the other colour and did not change, so the residual follows from the new
// values in registers and the neighbour sums already formed.
template <int SCH, bool EDGE, int LD>
__device__ __forceinline__ double smooth_cell_body_res(const Lev& L, const Coef& k, int i, int j) {
  const int m = L.m;
  const int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, L.n, L.nyn), jp = ywrap(j + 1, L.n, L.nyn);
  const size_t c = (size_t)j * m + i;
  const CellNew o = cell_update<SCH, EDGE, LD>(L, k, c, (size_t)j * m + im, (size_t)j * m + ip, (size_t)jm * m + i,
                                               (size_t)jp * m + i);
  L.phi[c] = o.phi;
  L.mu[c] = o.mu;
  L.ka[c] = o.ka;
  const double r1 = fma(-k.a, o.mu, o.R1 - o.phi);
  const double r3 = fma(-k.b3, o.phi, o.R3 - o.ka);
  const double r2 = fma(-k.b, o.ka, o.X2 - o.mu) + fma(k.gam + o.wv, o.phi, g_of<SCH>(o.phi, o.pk));
  return fma(r1, r1, fma(r2, r2, r3 * r3));
}

// Rows are warp-uniform, so the branch does not diverge; periodic levels never take
// it.  Two bodies, each reading its coefficient set at fixed parameter offsets.
template <int SCH, int LD = kLdNC>
__device__ __forceinline__ void smooth_cell(const Lev& L, const Coef& k0, const Coef& kb, int i, int j) {
  if (L.nyn && (j == 0 || j == L.n - 1)) smooth_cell_body<SCH, true, LD>(L, kb, i, j);
  else smooth_cell_body<SCH, false, LD>(L, k0, i, j);
}
template <int SCH>
__device__ __forceinline__ double smooth_cell_res(const Lev& L, const Coef& k0, const Coef& kb, int i, int j) {
  if (L.nyn && (j == 0 || j == L.n - 1)) return smooth_cell_body_res<SCH, true, kLdNC>(L, kb, i, j);
  return smooth_cell_body_res<SCH, false, kLdNC>(L, k0, i, j);
}
template <int SCH>
__global__ void __launch_bounds__(256) k_smooth(Lev L, Coef k, Coef kb, int color) {
  pdl_enter();
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= (L.m >> 1) || j >= L.n) return;
  smooth_cell<SCH>(L, k, kb, 2 * x + ((j + color) & 1), j);
}


// The finest level's last half sweep of a V-cycle (colour 1) with the residual of the
// cells it updates: each warp writes the sum of their r1^2 + r2^2 + r3^2 to
// bpart[warp] (one-warp blocks, warp = linear block index; lanes past the row add 0),
// and k_resnorm_red adds the other colour's cells.  So the V-cycle's convergence test
// evaluates the residual of half the cells from registers instead of again from memory.
template <int SCH>
__global__ void __launch_bounds__(32) k_smooth_res(Lev L, Coef k, Coef kb, double* __restrict__ bpart) {
  pdl_enter();
  const int x = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y;
  double v = 0.0;
  if (x < (L.m >> 1)) v = smooth_cell_res<SCH>(L, k, kb, 2 * x + ((j + 1) & 1), j);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) bpart[blockIdx.y * gridDim.x + blockIdx.x] = v;
}
