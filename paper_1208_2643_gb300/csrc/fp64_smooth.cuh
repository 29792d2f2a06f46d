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
// ---------------------------------------------------------------------------
// EDGE: a row next to a Neumann boundary, where the ghost neighbour is the cell's own
// unknown (App. A, (A.7)): it leaves the neighbour sums and k holds the coefficients
// of three neighbours.
template <int SCH, bool EDGE, int LD>
__device__ __forceinline__ void smooth_cell_body(const Lev& L, const Coef& k, int i, int j) {
  int m = L.m;
  int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, L.n, L.nyn), jp = ywrap(j + 1, L.n, L.nyn);
  size_t c = (size_t)j * m + i;
  size_t w = (size_t)j * m + im, e = (size_t)j * m + ip, s = (size_t)jm * m + i, nn = (size_t)jp * m + i;
  double* __restrict__ phi = L.phi;
  double* __restrict__ mu = L.mu;
  double* __restrict__ ka = L.ka;
  // neighbours belong to the other colour: read-only during this launch
  double smu = (ldv<LD>(mu + w) + ldv<LD>(mu + e)) + (ldv<LD>(mu + s) + ldv<LD>(mu + nn));
  double ska = (ldv<LD>(ka + w) + ldv<LD>(ka + e)) + (ldv<LD>(ka + s) + ldv<LD>(ka + nn));
  double sph = (ldv<LD>(phi + w) + ldv<LD>(phi + e)) + (ldv<LD>(phi + s) + ldv<LD>(phi + nn));
  double p = ldown<LD>(phi + c);
  if (EDGE) {   // the ghost was read as the cell's current value: take it out again
    smu -= ldown<LD>(mu + c);
    ska -= ldown<LD>(ka + c);
    sph -= p;
  }
  double R1 = fma(k.cmu, smu, ldv<LD>(L.S1 + c));
  double R3 = fma(k.th2, sph, ldv<LD>(L.S3 + c));
  // local Newton linearisation of the cubic about p: g ~ g(p) + g'(p)(phi - p);
  // q = g'(p) enters the determinant and the Cramer numerator of mu, and
  // e = g(p) - g'(p) p the right-hand side of row 2
  double R2, detw, Qq;   // detw = det / omega
  if (SCH == 1) {
    double p2 = p * p;
    R2 = fma(k.ih2, ska, fma(-2.0, p2 * p, ldv<LD>(L.S2 + c)));   // e = -2 p^3
    detw = fma(k.a3w, p2, k.D0w);                                   // q = 3 p^2
    Qq = fma(3.0, p2, k.Q0);
  } else {
    double pk = ldv<LD>(L.pk + c);
    double q = dg_of<2>(p, pk);
    R2 = fma(k.ih2, ska, ldv<LD>(L.S2 + c) + (g_of<2>(p, pk) - q * p));
    if (L.W) q += ldv<LD>(L.W + c);   // pinning: a pointwise linear term of row 2 (gam -> gam + W)
    detw = fma(k.aw, q, k.D0w);
    Qq = k.Q0 + q;
  }
  // Cramer's rule on [[1, a, 0], [-(gam+q), 1, b], [b3, 0, 1]] with t = b R3 - R2:
  //   phi* = (R1 + a t) / det,  mu* = ((Q0 + q) R1 - t) / det,  kappa* = R3 - b3 phi*;
  // then u <- (1 - omega) u + omega u*, with wr = omega / det
  const double wr = rcp_nr(detw);
  const double t = fma(k.b, R3, -R2);
  const double nphi = fma(k.a, t, R1);
  const double nmu = fma(Qq, R1, -t);
  if (k.relax) {
    double wphi = nphi * wr;
    double m0 = ldown<LD>(mu + c), k0 = ldown<LD>(ka + c);
    phi[c] = fma(k.omw, p, wphi);
    mu[c] = fma(k.omw, m0, nmu * wr);
    ka[c] = fma(-k.b3, wphi, fma(k.omega, R3, k.omw * k0));
  } else {
    double phin = nphi * wr;
    phi[c] = phin;
    mu[c] = nmu * wr;
    ka[c] = fma(-k.b3, phin, R3);
  }
}

// The same update, also returning the residual of the cell after it (r1^2 + r2^2 + r3^2),
// for the finest level's last half sweep of a V-cycle (k_smooth_res).
template <int SCH, bool EDGE, int LD>
__device__ __forceinline__ double smooth_cell_body_res(const Lev& L, const Coef& k, int i, int j) {
  int m = L.m;
  int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, L.n, L.nyn), jp = ywrap(j + 1, L.n, L.nyn);
  size_t c = (size_t)j * m + i;
  size_t w = (size_t)j * m + im, e = (size_t)j * m + ip, s = (size_t)jm * m + i, nn = (size_t)jp * m + i;
  double* __restrict__ phi = L.phi;
  double* __restrict__ mu = L.mu;
  double* __restrict__ ka = L.ka;
  // neighbours belong to the other colour: read-only during this launch
  double smu = (ldv<LD>(mu + w) + ldv<LD>(mu + e)) + (ldv<LD>(mu + s) + ldv<LD>(mu + nn));
  double ska = (ldv<LD>(ka + w) + ldv<LD>(ka + e)) + (ldv<LD>(ka + s) + ldv<LD>(ka + nn));
  double sph = (ldv<LD>(phi + w) + ldv<LD>(phi + e)) + (ldv<LD>(phi + s) + ldv<LD>(phi + nn));
  double p = ldown<LD>(phi + c);
  if (EDGE) {   // the ghost was read as the cell's current value: take it out again
    smu -= ldown<LD>(mu + c);
    ska -= ldown<LD>(ka + c);
    sph -= p;
  }
  double R1 = fma(k.cmu, smu, ldv<LD>(L.S1 + c));
  double R3 = fma(k.th2, sph, ldv<LD>(L.S3 + c));
  const double s2 = ldv<LD>(L.S2 + c);
  // local Newton linearisation of the cubic about p: g ~ g(p) + g'(p)(phi - p);
  // q = g'(p) enters the determinant and the Cramer numerator of mu, and
  // e = g(p) - g'(p) p the right-hand side of row 2
  double R2, detw, Qq, pk = 0.0, wv = 0.0;   // detw = det / omega
  if (SCH == 1) {
    double p2 = p * p;
    R2 = fma(k.ih2, ska, fma(-2.0, p2 * p, s2));   // e = -2 p^3
    detw = fma(k.a3w, p2, k.D0w);                  // q = 3 p^2
    Qq = fma(3.0, p2, k.Q0);
  } else {
    pk = ldv<LD>(L.pk + c);
    double q = dg_of<2>(p, pk);
    R2 = fma(k.ih2, ska, s2 + (g_of<2>(p, pk) - q * p));
    if (L.W) {   // pinning: a pointwise linear term of row 2 (gam -> gam + W)
      wv = ldv<LD>(L.W + c);
      q += wv;
    }
    detw = fma(k.aw, q, k.D0w);
    Qq = k.Q0 + q;
  }
  // Cramer's rule on [[1, a, 0], [-(gam+q), 1, b], [b3, 0, 1]] with t = b R3 - R2:
  //   phi* = (R1 + a t) / det,  mu* = ((Q0 + q) R1 - t) / det,  kappa* = R3 - b3 phi*;
  // then u <- (1 - omega) u + omega u*, with wr = omega / det
  const double wr = rcp_nr(detw);
  const double t = fma(k.b, R3, -R2);
  const double nphi = fma(k.a, t, R1);
  const double nmu = fma(Qq, R1, -t);
  double pn, un, vn;
  if (k.relax) {
    double wphi = nphi * wr;
    double m0 = ldown<LD>(mu + c), k0 = ldown<LD>(ka + c);
    pn = fma(k.omw, p, wphi);
    un = fma(k.omw, m0, nmu * wr);
    vn = fma(-k.b3, wphi, fma(k.omega, R3, k.omw * k0));
  } else {
    pn = nphi * wr;
    un = nmu * wr;
    vn = fma(-k.b3, pn, R3);
  }
  phi[c] = pn;
  mu[c] = un;
  ka[c] = vn;
  // the residual S - N(u) of the cell just updated, from the values in registers
  // (its neighbours belong to the other colour and did not change): r1 = R1 - phi - a mu,
  // r2 = S2 + h^-2 sum_nb kappa - b kappa - mu + g(phi) + (gam + W) phi,
  // r3 = R3 - kappa - b3 phi; returns r1^2 + r2^2 + r3^2
  const double r1 = fma(-k.a, un, R1 - pn);
  const double r3 = fma(-k.b3, pn, R3 - vn);
  const double r2 = fma(-k.b, vn, fma(k.ih2, ska, s2) - un) + fma(k.gam + wv, pn, g_of<SCH>(pn, pk));
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
