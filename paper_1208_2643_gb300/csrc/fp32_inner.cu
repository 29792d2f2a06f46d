// Mixed-precision form: FP64 outer defect correction around FP32 inner V-cycles.
//
// Outer iteration (FP64): r = S - N(u) with N of App. B.1/B.2, and the local Newton
// linearisation of the cubic, q = gam + g'(phi), both evaluated in double precision.
// Inner solve (FP32): the linearised correction equation J(u) e = r,
//   e_phi - c Delta_h e_mu = r1,  e_mu - q e_phi - Delta_h e_kappa = r2,
//   e_kappa - theta Delta_h e_phi = r3,
// by `inner_cycles` correction-scheme V-cycles: the same red-black block Gauss-Seidel
// cell solve as App. B (with q frozen, so no cubic), 2x2 averaging of the defect,
// bilinear prolongation of the coarse correction, and a direct FP32 solve on the
// coarsest grid.  Then u += e in FP64, and the loop test runs on the FP64 residual.
// The converged answer is therefore the FP64 solution at the FP64 tolerance; FP32
// only limits how much each outer iteration gains.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include <vector>

#include "fp64_kernels.cuh"
#include "mpfc_internal.h"

using namespace mpfc;

namespace {

struct Coef32 {
  float cmu, a, ih2, b, b3, th2, D0, Q0, omega, omw, c, theta;
  int relax;
};

Coef32 coef32_of(const Coef& k) {
  Coef32 f;
  f.cmu = (float)k.cmu;
  f.a = (float)k.a;
  f.ih2 = (float)k.ih2;
  f.b = (float)k.b;
  f.b3 = (float)k.b3;
  f.th2 = (float)k.th2;
  f.D0 = (float)(1.0 + k.a * k.b * k.b3);   // determinant without q (q includes gam here)
  f.Q0 = (float)(k.b * k.b3);
  f.omega = (float)k.omega;
  f.omw = (float)(1.0 - k.omega);
  f.c = (float)k.c;
  f.theta = (float)k.theta;
  f.relax = k.relax;
  return f;
}

const dim3 kBlk(32, 8);
dim3 grid_of(int X, int Y) { return dim3((X + kBlk.x - 1) / kBlk.x, (Y + kBlk.y - 1) / kBlk.y); }

// ---------------------------------------------------------------------------
// FP64 defect: r = S - N(u) and q = gam + g'(phi) as FP32 inputs of the inner solve,
// e = 0, and the scaled residual norm with the outer loop decision.
// ---------------------------------------------------------------------------
template <int SCH>
__global__ void __launch_bounds__(256) k_defect(Lev L, Coef k, Lev32 E, Ctl* ctl, double* partials, int mode,
                                                cudaGraphConditionalHandle hnd, int set_cond) {
  pdl_enter();
  double v[1] = {0.0};
  int G = L.m * L.n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < G; t += gridDim.x * blockDim.x) {
    int i = t % L.m, j = t / L.m;
    double a, b, c;
    resid_at<SCH>(L, k, i, j, a, b, c);
    v[0] = fma(a, a, fma(b, b, fma(c, c, v[0])));
    double p = L.phi[t];
    double pk = (SCH == 2) ? L.pk[t] : 0.0;
    // defect and linearisation handed to the FP32 solve, rounded to nearest (a
    // non-finite defect stays non-finite, so the residual test above sees it)
    E.r1[t] = f64_to_f32_rn(a);
    E.r2[t] = f64_to_f32_rn(b);
    E.r3[t] = f64_to_f32_rn(c);
    // q = gam + g'(phi), plus the pinning weight (Sec. 4.6, scheme 2: gam -> gam + W)
    const double wq = (SCH == 2 && L.W) ? L.W[t] : 0.0;
    E.q[t] = f64_to_f32_rn(k.gam + wq + dg_of<SCH>(p, pk));
    E.ephi[t] = 0.f;
    E.emu[t] = 0.f;
    E.eka[t] = 0.f;
  }
  if (!grid_sum<1>(v, partials, &ctl->counter)) return;
  double res = sqrt(v[0] / (3.0 * (double)G));
  int cond;
  if (mode == 0) {
    ctl->res0 = res;
    ctl->res = res;
    ctl->cycles = 0;
    ctl->status = 0;
    if (!(res == res) || isinf(res)) ctl->status = 2;
  } else {
    ctl->res = res;
    ctl->cycles += 1;
    if (!(res == res) || isinf(res) || res > 1e10 * fmax(ctl->res0, ctl->tol)) ctl->status = 2;
  }
  if (ctl->skip || ctl->status != 0) cond = 0;
  else if (ctl->fixed_cycles > 0) cond = ctl->cycles < ctl->fixed_cycles;
  else cond = (res > ctl->tol) && (ctl->cycles < ctl->max_cycles);
  if (set_cond) cudaGraphSetConditional(hnd, cond ? 1u : 0u);
}

// u += e (FP64 update with the FP32 correction)
__global__ void k_update(Lev L, Lev32 E) {
  pdl_enter();
  int G = L.m * L.n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < G; t += gridDim.x * blockDim.x) {
    float a = E.ephi[t], b = E.emu[t], c = E.eka[t];
    L.phi[t] += f32_to_f64(a);
    L.mu[t] += f32_to_f64(b);
    L.ka[t] += f32_to_f64(c);
  }
}

__global__ void k_restrict_q(const float* __restrict__ qf, float* __restrict__ qc, int mc, int nc) {
  pdl_enter();
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= mc || J >= nc) return;
  int mf = 2 * mc;
  size_t a = (size_t)(2 * J) * mf + 2 * I, b = a + mf;
  qc[(size_t)J * mc + I] = 0.25f * ((qf[a] + qf[a + 1]) + (qf[b] + qf[b + 1]));
}

// Loads of the FP32 cell functions: the read-only path for global planes that the
// kernel does not write, plain loads otherwise (also for planes in shared memory).
template <bool NC>
__device__ __forceinline__ float ld32(const float* p) {
  if (NC) return __ldg(p);
  return *p;
}

// The cell update of the correction equation on values: neighbour sums, q, the
// defect source r and the cell's own e (in/out).  One order of operations for every
// kernel that sweeps (global planes, shared-memory planes, temporally blocked tiles),
// so they all give the same bits.
__device__ __forceinline__ void smooth32_core(const Coef32& k, float smu, float ska, float sph, float q, float r1,
                                              float r2, float r3, float& ep, float& em, float& ek) {
  float R1 = fmaf(k.cmu, smu, r1);
  float R2 = fmaf(k.ih2, ska, r2);
  float R3 = fmaf(k.th2, sph, r3);
  float rdet = __frcp_rn(fmaf(k.a, q, k.D0));
  float nphi = fmaf(k.a, fmaf(k.b, R3, -R2), R1);
  float nmu = fmaf(k.Q0 + q, R1, fmaf(-k.b, R3, R2));
  if (k.relax) {
    float wr = k.omega * rdet;
    float wphi = nphi * wr;
    float p0 = ep, m0 = em, k0 = ek;
    ep = fmaf(k.omw, p0, wphi);
    em = fmaf(k.omw, m0, nmu * wr);
    ek = fmaf(-k.b3, wphi, fmaf(k.omega, R3, k.omw * k0));
  } else {
    float phin = nphi * rdet;
    ep = phin;
    em = nmu * rdet;
    ek = fmaf(-k.b3, phin, R3);
  }
}

// Defect rho = r - J e of the correction equation at one cell, on values.
__device__ __forceinline__ void defect32_core(const Coef32& k, float p, float u, float v, float smu, float ska, float sph,
                                              float q, float r1, float r2, float r3, float& d1, float& d2, float& d3) {
  d1 = fmaf(k.cmu, fmaf(-4.f, u, smu), r1 - p);
  d2 = fmaf(k.ih2, fmaf(-4.f, v, ska), fmaf(q, p, r2 - u));
  d3 = fmaf(k.th2, fmaf(-4.f, p, sph), r3 - v);
}

// kb: the cell system of a Neumann boundary row (three neighbours; the ghost is the
// cell's own unknown, read once through the clamped index and taken out of the sums).
template <bool NC>
__device__ __forceinline__ void smooth32_cell(const Lev32& L, const Coef32& k, const Coef32& kb, int i, int j) {
  int m = L.m;
  int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, L.n, L.nyn), jp = ywrap(j + 1, L.n, L.nyn);
  size_t c = (size_t)j * m + i;
  size_t w = (size_t)j * m + im, e = (size_t)j * m + ip, s = (size_t)jm * m + i, nn = (size_t)jp * m + i;
  float* __restrict__ ep = L.ephi;
  float* __restrict__ em = L.emu;
  float* __restrict__ ek = L.eka;
  float smu = (ld32<NC>(em + w) + ld32<NC>(em + e)) + (ld32<NC>(em + s) + ld32<NC>(em + nn));
  float ska = (ld32<NC>(ek + w) + ld32<NC>(ek + e)) + (ld32<NC>(ek + s) + ld32<NC>(ek + nn));
  float sph = (ld32<NC>(ep + w) + ld32<NC>(ep + e)) + (ld32<NC>(ep + s) + ld32<NC>(ep + nn));
  float a = ep[c], b = em[c], d = ek[c];
  const float q = ld32<NC>(L.q + c), r1 = ld32<NC>(L.r1 + c), r2 = ld32<NC>(L.r2 + c), r3 = ld32<NC>(L.r3 + c);
  // one inlined update per coefficient set (selecting between the two structs would copy
  // them through local memory)
  if (L.nyn && (j == 0 || j == L.n - 1))
    smooth32_core(kb, smu - b, ska - d, sph - a, q, r1, r2, r3, a, b, d);
  else
    smooth32_core(k, smu, ska, sph, q, r1, r2, r3, a, b, d);
  ep[c] = a;
  em[c] = b;
  ek[c] = d;
}

// ---------------------------------------------------------------------------
// FP32 red-black half sweep of the correction equation (App. B cell system with
// the frozen linearisation q = gam + g'(phi)).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_smooth32(Lev32 L, Coef32 k, Coef32 kb, int color) {
  pdl_enter();
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= (L.m >> 1) || j >= L.n) return;
  smooth32_cell<true>(L, k, kb, 2 * x + ((j + color) & 1), j);
}

// defect of the correction equation at one cell: rho = r - J e
template <bool NC>
__device__ __forceinline__ void defect32(const Lev32& L, const Coef32& k, int i, int j, float& d1, float& d2,
                                         float& d3) {
  int m = L.m;
  // a Neumann ghost reads as the cell itself, so the five-point sums are the boundary rule's
  int im = wrapm(i - 1, m), ip = wrapm(i + 1, m), jm = ywrap(j - 1, L.n, L.nyn), jp = ywrap(j + 1, L.n, L.nyn);
  size_t c = (size_t)j * m + i;
  size_t w = (size_t)j * m + im, e = (size_t)j * m + ip, s = (size_t)jm * m + i, nn = (size_t)jp * m + i;
  const float* ep = L.ephi;
  const float* em = L.emu;
  const float* ek = L.eka;
  float p = ld32<NC>(ep + c), u = ld32<NC>(em + c), v = ld32<NC>(ek + c);
  float smu = (ld32<NC>(em + w) + ld32<NC>(em + e)) + (ld32<NC>(em + s) + ld32<NC>(em + nn));
  float ska = (ld32<NC>(ek + w) + ld32<NC>(ek + e)) + (ld32<NC>(ek + s) + ld32<NC>(ek + nn));
  float sph = (ld32<NC>(ep + w) + ld32<NC>(ep + e)) + (ld32<NC>(ep + s) + ld32<NC>(ep + nn));
  defect32_core(k, p, u, v, smu, ska, sph, ld32<NC>(L.q + c), ld32<NC>(L.r1 + c), ld32<NC>(L.r2 + c),
                ld32<NC>(L.r3 + c), d1, d2, d3);
}

// coarse source = R(r - J e), coarse correction starts at zero
template <bool NC>
__device__ __forceinline__ void restrict_defect32_cell(const Lev32& F, const Lev32& C, const Coef32& kf, int I, int J) {
  float s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
  for (int dj = 0; dj < 2; ++dj)
#pragma unroll
    for (int di = 0; di < 2; ++di) {
      float a, b, c;
      defect32<NC>(F, kf, 2 * I + di, 2 * J + dj, a, b, c);
      s1 += a;
      s2 += b;
      s3 += c;
    }
  size_t cid = (size_t)J * C.m + I;
  C.r1[cid] = 0.25f * s1;
  C.r2[cid] = 0.25f * s2;
  C.r3[cid] = 0.25f * s3;
  C.ephi[cid] = 0.f;
  C.emu[cid] = 0.f;
  C.eka[cid] = 0.f;
}

__global__ void k_restrict_defect32(Lev32 F, Lev32 C, Coef32 kf) {
  pdl_enter();
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= C.m || J >= C.n) return;
  restrict_defect32_cell<true>(F, C, kf, I, J);
}

// e_f += P e_c (bilinear, shared-memory tiles of the three components of the coarse
// correction, staged together)
constexpr int kTX = 32, kTY = 8;
__device__ __forceinline__ void prolong32_apply(float (*E)[kTX + 2], float* __restrict__ ef, int mc, int I, int J) {
  int x = threadIdx.x + 1, y = threadIdx.y + 1;
  const float w9 = 9.f / 16.f, w3 = 3.f / 16.f, w1 = 1.f / 16.f;
  float c9 = w9 * E[y][x];
  int mf = 2 * mc;
  size_t f00 = (size_t)(2 * J) * mf + 2 * I, f01 = f00 + mf;
  ef[f00] += fmaf(w3, E[y][x - 1] + E[y - 1][x], fmaf(w1, E[y - 1][x - 1], c9));
  ef[f00 + 1] += fmaf(w3, E[y][x + 1] + E[y - 1][x], fmaf(w1, E[y - 1][x + 1], c9));
  ef[f01] += fmaf(w3, E[y][x - 1] + E[y + 1][x], fmaf(w1, E[y + 1][x - 1], c9));
  ef[f01 + 1] += fmaf(w3, E[y][x + 1] + E[y + 1][x], fmaf(w1, E[y + 1][x + 1], c9));
}

__global__ void __launch_bounds__(kTX * kTY) k_prolong32(Lev32 F, Lev32 C) {
  pdl_enter();
  __shared__ float E[3][kTY + 2][kTX + 2];
  const int mc = C.m, nc = C.n;
  const int I0 = blockIdx.x * kTX, J0 = blockIdx.y * kTY;
  for (int t = threadIdx.y * kTX + threadIdx.x; t < (kTX + 2) * (kTY + 2); t += kTX * kTY) {
    int ty = t / (kTX + 2), tx = t % (kTX + 2);
    if (I0 + tx - 1 < mc + 1 && J0 + ty - 1 < nc + 1) {
      size_t id = (size_t)ywrap(J0 + ty - 1, nc, C.nyn) * mc + wrapm(I0 + tx - 1, mc);
      E[0][ty][tx] = __ldg(C.ephi + id);
      E[1][ty][tx] = __ldg(C.emu + id);
      E[2][ty][tx] = __ldg(C.eka + id);
    }
  }
  __syncthreads();
  int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
  if (I < mc && J < nc) {
    prolong32_apply(E[0], F.ephi, mc, I, J);
    prolong32_apply(E[1], F.emu, mc, I, J);
    prolong32_apply(E[2], F.eka, mc, I, J);
  }
}

// ---------------------------------------------------------------------------
// Coarsest grid, FP32: eliminate e_kappa and e_mu,
//   (I - c L diag(q) - c theta L^3) e_phi = r1 + c L (r2 + L r3),
// solve by Gaussian elimination with partial pivoting in one CTA, then
// e_kappa = r3 + theta L e_phi, e_mu = r2 + q e_phi + L e_kappa.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float nbsum32(const float* f, int m, int n, int t, int nyn) {
  int i = t % m, j = t / m;
  return (f[j * m + wrapm(i - 1, m)] + f[j * m + wrapm(i + 1, m)]) +
         (f[ywrap(j - 1, n, nyn) * m + i] + f[ywrap(j + 1, n, nyn) * m + i]);
}

// The whole block; smf holds G (G + 1) + 4 G floats.  C's planes may be in global or
// shared memory (plain loads).
__device__ void coarse32_block(const Lev32& C, const Coef32& k, const float* __restrict__ K3f, float* smf) {
  const int m = C.m, n = C.n, G = m * n, W = G + 1;
  float* A = smf;
  float* t1 = A + G * W;
  float* t2 = t1 + G;
  float* x = t2 + G;
  float* d = x + G;
  __shared__ int s_piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  // t1 = L r3 (with the 1/h^2 of L), t2 = r2 + t1
  for (int t = tid; t < G; t += nt) t1[t] = k.ih2 * (nbsum32(C.r3, m, n, t, C.nyn) - 4.f * C.r3[t]);
  __syncthreads();
  for (int t = tid; t < G; t += nt) t2[t] = C.r2[t] + t1[t];
  __syncthreads();
  for (int t = tid; t < G; t += nt) A[t * W + G] = C.r1[t] + k.cmu * (nbsum32(t2, m, n, t, C.nyn) - 4.f * t2[t]);
  const float* cLf = K3f + G * G;   // c L, after K3 in the coarse block
  auto entry = [&](int r, int col) { return K3f[r * G + col] - cLf[r * G + col] * C.q[col]; };
  if (G <= 31) {
    // one warp: a Jacobian column per lane in registers, Gauss-Jordan with implicit
    // pivoting (gauss_jordan_cols); the right-hand side in lane G
    __syncthreads();
    auto column = [&](auto& a) {
      constexpr int R = sizeof(a) / sizeof(a[0]);
#pragma unroll
      for (int r = 0; r < R; ++r)
        a[r] = (r < G) ? (tid < G ? entry(r, tid) : (tid == G ? A[r * W + G] : 0.f)) : 0.f;
      __syncwarp();
      gauss_jordan_cols<R>(a, G, x, t2, reinterpret_cast<int*>(d));
    };
    if (tid < 32) {
      if (G <= 16) {
        float a[16];
        column(a);
      } else {
        float a[32];
        column(a);
      }
    }
    __syncthreads();
  } else {
    for (int idx = tid; idx < G * G; idx += nt) A[(idx / G) * W + idx % G] = entry(idx / G, idx % G);
    __syncthreads();
    for (int col = 0; col < G; ++col) {
      if (tid == 0) {
        int piv = col;
        float best = fabsf(A[col * W + col]);
        for (int r = col + 1; r < G; ++r) {
          float v = fabsf(A[r * W + col]);
          if (v > best) { best = v; piv = r; }
        }
        s_piv = piv;
      }
      __syncthreads();
      int piv = s_piv;
      if (piv != col)
        for (int c2 = col + tid; c2 <= G; c2 += nt) {
          float t = A[col * W + c2];
          A[col * W + c2] = A[piv * W + c2];
          A[piv * W + c2] = t;
        }
      __syncthreads();
      for (int r = col + 1 + tid; r < G; r += nt) d[r] = A[r * W + col] / A[col * W + col];
      __syncthreads();
      int rows = G - col - 1, cols = G - col;
      for (int idx = tid; idx < rows * cols; idx += nt) {
        int r = col + 1 + idx / cols, c2 = col + 1 + idx % cols;
        A[r * W + c2] -= d[r] * A[col * W + c2];
      }
      __syncthreads();
    }
    if (tid == 0)
      for (int r = G - 1; r >= 0; --r) {
        float acc = A[r * W + G];
        for (int c2 = r + 1; c2 < G; ++c2) acc -= A[r * W + c2] * x[c2];
        x[r] = acc / A[r * W + r];
      }
    __syncthreads();
  }
  for (int t = tid; t < G; t += nt) t1[t] = C.r3[t] + k.th2 * (nbsum32(x, m, n, t, C.nyn) - 4.f * x[t]);   // e_kappa
  __syncthreads();
  for (int t = tid; t < G; t += nt) {
    C.emu[t] = C.r2[t] + C.q[t] * x[t] + k.ih2 * (nbsum32(t1, m, n, t, C.nyn) - 4.f * t1[t]);
    C.ephi[t] = x[t];
    C.eka[t] = t1[t];
  }
}

__global__ void k_coarse32(Lev32 C, Coef32 k, const float* __restrict__ K3f) {
  pdl_enter();
  extern __shared__ float smf[];
  coarse32_block(C, k, K3f, smf);
}

size_t coarse32_smem(const Lev32& C) {
  int G = C.m * C.n;
  return sizeof(float) * ((size_t)G * (G + 1) + 4 * (size_t)G);
}

// ---------------------------------------------------------------------------
// One full red-black sweep in one launch, out of place (e read from one copy, written
// to the other), over tiles of kSwX x ty cells staged in shared memory: e with a
// two-cell halo, q and r with a one-cell halo.  A tile updates the red cells of
// itself and of its one-cell ring (from the old black values), then its black cells
// (from the new red values), and writes itself to the destination copy.  Each plane's
// lines are read once per sweep instead of once per colour.  A ring cell's red update
// is computed by both tiles that hold it, from the same inputs with the same
// operations (smooth32_core), so the result is bit for bit that of the two half-sweep
// launches; reading and writing different copies lets the tiles run in any order.
// The kernel is persistent: each CTA walks its tiles with two shared-memory stages,
// the next tile's asynchronous copies (cp.async, wrapped periodic addresses) in flight
// while the current one is computed.
// ---------------------------------------------------------------------------
constexpr int kSwX = 64;                    // tile width in cells (rows are float4-aligned)
constexpr int kSwPad = 4;                   // columns staged left and right of the tile (>= 2)
constexpr int kSwW = kSwX + 2 * kSwPad;     // staged row length (floats)
constexpr int kSwThreads = 320;             // 10 warps

__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One stage: e (3 planes of ty + 4 staged rows) then q, r1, r2, r3 (ty + 2 rows), each plane's
// block starting on a 128-byte boundary (tensor copies write there).
__host__ __device__ __forceinline__ int sweep_plane_e(int ty) { return (kSwW * (ty + 4) + 31) / 32 * 32; }
__host__ __device__ __forceinline__ int sweep_plane_q(int ty) { return (kSwW * (ty + 2) + 31) / 32 * 32; }
__host__ __device__ __forceinline__ int sweep_stage_floats(int ty) { return 3 * sweep_plane_e(ty) + 4 * sweep_plane_q(ty); }
// dynamic shared memory of the kernel: two stages, two mbarriers, alignment slack
__host__ __device__ __forceinline__ size_t sweep_smem_bytes(int ty) {
  return 2 * sizeof(float) * (size_t)sweep_stage_floats(ty) + 16 + 128;
}

// Tensor maps of the planes a tile stages (interior tiles): the source copy of e and q, r.
struct SweepMaps {
  CUtensorMap e[3];
  CUtensorMap qr[4];
};

__device__ __forceinline__ void sw_bar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
}
__device__ __forceinline__ bool sw_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for a stage's tensor copies (about 1 s at the GPU's clock by default);
// false if they did not arrive.  The limit and the test hook's switch
// (mpfc_fp32_test_withhold_copy: the tensor copies of tile (1, 1), the second tile of
// the second tile row, are skipped) live in device variables.
constexpr long long kSwSpinLimit = 2000000000ll;
__device__ long long g_sw_spin_limit = kSwSpinLimit;
__device__ int g_sw_withhold = 0;
__device__ __forceinline__ bool sw_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64(), limit = g_sw_spin_limit;
  while (!sw_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void sw_tma_2d(float* dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ int sw_col(int x, int m) { x %= m; return x < 0 ? x + m : x; }
__device__ __forceinline__ int sw_row(int y, int n, int nyn) {
  if (nyn) return y < 0 ? 0 : (y >= n ? n - 1 : y);   // ghost rows read as the boundary row (A.7)
  y %= n;
  return y < 0 ? y + n : y;
}

struct SweepSrc {
  const float *ephi, *emu, *eka;   // source copy of e
  float *dphi, *dmu, *dka;         // destination copy
};

// Stages the tile (x0, y0) of TY rows: e rows y0-2 .. y0+TY+1 and q / r rows y0-1 ..
// y0+TY, columns x0-4 .. x0+67.  A tile that reaches no domain edge is staged by one
// thread with seven 2-D tensor copies (boxes of 72 columns, x0-4 a multiple of 4, so
// 16-byte aligned) completing on the stage's mbarrier; the others by 16-byte cp.async
// copies of every thread, wrapping the columns and rows (periodic) or clamping the rows
// (Neumann ghost rows, (A.7)).  Returns whether the tensor copies were used.
template <int TY>
__device__ __forceinline__ bool sweep_tile_load(const Lev32& L, const SweepSrc& S, const SweepMaps& M, bool use_tma,
                                                int x0, int y0, float* st, uint32_t bar, bool withhold = false) {
  constexpr int q4 = kSwW / 4, RE = TY + 4, RQ = TY + 2;
  const int PE = sweep_plane_e(TY), PQ = sweep_plane_q(TY);
  const int m = L.m, n = L.n;
  const bool inner = x0 >= kSwPad && x0 + kSwX + kSwPad <= m && y0 >= 2 && y0 + TY + 2 <= n;
  float* qb = st + 3 * PE;
  if (inner && use_tma) {
    if (threadIdx.x == 0 && !withhold) {
      // the stage was last read through the generic proxy (after the block barrier that
      // precedes this call); order those reads before the tensor copies' writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      constexpr uint32_t kBytes = (uint32_t)(sizeof(float) * kSwW * (3 * RE + 4 * RQ));
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBytes) : "memory");
      for (int p = 0; p < 3; ++p) sw_tma_2d(st + p * PE, &M.e[p], x0 - kSwPad, y0 - 2, bar);
      for (int p = 0; p < 4; ++p) sw_tma_2d(qb + p * PQ, &M.qr[p], x0 - kSwPad, y0 - 1, bar);
    }
    return true;
  }
  if (inner) {
    const size_t g0 = (size_t)(y0 - 2) * m + (x0 - kSwPad);
    for (int t = threadIdx.x; t < RE * q4; t += kSwThreads) {
      const int r = t / q4, c4 = t - r * q4;
      const size_t g = g0 + (size_t)r * m + 4 * c4;
      float* d = st + r * kSwW + 4 * c4;
      cp_async16(d, S.ephi + g);
      cp_async16(d + PE, S.emu + g);
      cp_async16(d + 2 * PE, S.eka + g);
    }
    for (int t = threadIdx.x; t < RQ * q4; t += kSwThreads) {
      const int r = t / q4, c4 = t - r * q4;
      const size_t g = g0 + (size_t)(r + 1) * m + 4 * c4;
      float* d = qb + r * kSwW + 4 * c4;
      cp_async16(d, L.q + g);
      cp_async16(d + PQ, L.r1 + g);
      cp_async16(d + 2 * PQ, L.r2 + g);
      cp_async16(d + 3 * PQ, L.r3 + g);
    }
    cp_async_commit();
    return false;
  }
  for (int t = threadIdx.x; t < RE * q4; t += kSwThreads) {
    const int r = t / q4, c4 = t - r * q4;
    const size_t g = (size_t)sw_row(y0 - 2 + r, n, L.nyn) * m + sw_col(x0 - kSwPad + 4 * c4, m);
    float* d = st + r * kSwW + 4 * c4;
    cp_async16(d, S.ephi + g);
    cp_async16(d + PE, S.emu + g);
    cp_async16(d + 2 * PE, S.eka + g);
  }
  for (int t = threadIdx.x; t < RQ * q4; t += kSwThreads) {
    const int r = t / q4, c4 = t - r * q4;
    const size_t g = (size_t)sw_row(y0 - 1 + r, n, L.nyn) * m + sw_col(x0 - kSwPad + 4 * c4, m);
    float* d = qb + r * kSwW + 4 * c4;
    cp_async16(d, L.q + g);
    cp_async16(d + PQ, L.r1 + g);
    cp_async16(d + 2 * PQ, L.r2 + g);
    cp_async16(d + 3 * PQ, L.r3 + g);
  }
  cp_async_commit();
  return false;
}

// The cell update of smooth32_cell on staged values: ce indexes the cell in the e
// arrays (row stride kSwW), cq in the q / r arrays; same sums, same core.
__device__ __forceinline__ void sweep_tile_cell(const Coef32& k, const Coef32& kb, bool bnd, float* E0, float* E1,
                                                float* E2, int ce, const float* Qs, int RQW, int cq) {
  const float smu = (E1[ce - 1] + E1[ce + 1]) + (E1[ce - kSwW] + E1[ce + kSwW]);
  const float ska = (E2[ce - 1] + E2[ce + 1]) + (E2[ce - kSwW] + E2[ce + kSwW]);
  const float sph = (E0[ce - 1] + E0[ce + 1]) + (E0[ce - kSwW] + E0[ce + kSwW]);
  float a = E0[ce], b = E1[ce], d = E2[ce];
  const float q = Qs[cq], r1 = Qs[RQW + cq], r2 = Qs[2 * RQW + cq], r3 = Qs[3 * RQW + cq];
  if (bnd)
    smooth32_core(kb, smu - b, ska - d, sph - a, q, r1, r2, r3, a, b, d);
  else
    smooth32_core(k, smu, ska, sph, q, r1, r2, r3, a, b, d);
  E0[ce] = a;
  E1[ce] = b;
  E2[ce] = d;
}

// Red cells ((x + y) even) of a staged tile of tw x th cells and of its one-cell ring,
// then (after a barrier) its black cells.
//
// A whole 64 x TY tile (FULL) maps each warp to 16 cells of one colour in each of two
// adjacent rows.  A colour's cells in one row sit at every other word, all of one
// parity, and the next row's at the other parity; with an even row stride (72 words)
// the two half-warps then read disjoint bank sets, and every access of the cell update
// (own cell, four neighbours, q and r) keeps that split, so none conflicts.  The red
// work is the 32 interior red cells of each of the TY + 2 ring rows, in row pairs and
// groups of 16, plus one item for the ring's 33rd red cell of each row (column x0-1 or
// x0+64); the black work is the 32 black cells of each of the TY rows.  An edge tile
// uses a plain loop over its ragged bounds.
template <int TY, bool FULL>
__device__ __forceinline__ void sweep_tile_compute(const Lev32& L, const Coef32& k, const Coef32& kb, float* E0, int x0,
                                                   int y0, int tw, int th, const SweepSrc& S) {
  constexpr int kWarps = kSwThreads / 32;
  const int PE = sweep_plane_e(TY), PQ = sweep_plane_q(TY);
  float* E1 = E0 + PE;
  float* E2 = E1 + PE;
  const float* Qs = E2 + PE;
  const int m = L.m, n = L.n;
  if (FULL) {
    constexpr int kRingItems = (TY + 2 + 31) / 32;   // the ring's 33rd red cells, 32 rows per item
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int item = warp; item < TY + 2 + kRingItems; item += kWarps) {
      int rr, cc;   // ring row (y = y0 - 1 + rr) and ring column (x = x0 - 1 + cc)
      if (item < TY + 2) {
        rr = 2 * (item >> 1) + (lane >> 4);
        cc = 1 + ((x0 + y0 - 1 + rr) & 1) + 2 * (16 * (item & 1) + (lane & 15));
      } else {
        rr = 32 * (item - (TY + 2)) + lane;
        if (rr >= TY + 2) continue;
        cc = ((x0 + y0 - 2 + rr) & 1) == 0 ? 0 : kSwX + 1;
      }
      const int y = y0 - 1 + rr;
      if (L.nyn && (y < 0 || y >= n)) continue;   // Neumann ghost rows hold no cells
      const bool bnd = L.nyn && (y == 0 || y == n - 1);
      sweep_tile_cell(k, kb, bnd, E0, E1, E2, (rr + 1) * kSwW + cc + kSwPad - 1, Qs, PQ,
                      rr * kSwW + cc + kSwPad - 1);
    }
    __syncthreads();
    // black cells; a warp then writes the 2 x 32 cells of its item (its black cells and
    // the red ones between them, final since the barrier) to the destination copy
    for (int item = warp; item < TY; item += kWarps) {
      const int r0 = 2 * (item >> 1), c0 = 32 * (item & 1);
      const int rr = r0 + (lane >> 4), y = y0 + rr;
      const int cc = ((x0 + y + 1) & 1) + 2 * (16 * (item & 1) + (lane & 15));
      const bool bnd = L.nyn && (y == 0 || y == n - 1);
      sweep_tile_cell(k, kb, bnd, E0, E1, E2, (rr + 2) * kSwW + cc + kSwPad, Qs, PQ,
                      (rr + 1) * kSwW + cc + kSwPad);
      __syncwarp();
      for (int v = lane; v < 48; v += 32) {   // 3 planes x 2 rows x 8 float4
        const int pl = v >> 4, row = (v >> 3) & 1, c4 = v & 7;
        const float* src = E0 + pl * PE + (r0 + row + 2) * kSwW + kSwPad + c0 + 4 * c4;
        float* dst = (pl == 0 ? S.dphi : pl == 1 ? S.dmu : S.dka) + (size_t)(y0 + r0 + row) * m + x0 + c0 + 4 * c4;
        *reinterpret_cast<float4*>(dst) = *reinterpret_cast<const float4*>(src);
      }
    }
    return;
  }
  {
    const int rw = tw + 2, per = (rw + 1) >> 1, rows = th + 2;
    for (int t = threadIdx.x; t < rows * per; t += kSwThreads) {
      const int rr = t / per, y = y0 - 1 + rr;
      const int cc = 2 * (t - rr * per) + ((x0 - 1 + y) & 1);
      if (cc >= rw) continue;
      if (L.nyn && (y < 0 || y >= n)) continue;   // Neumann ghost rows hold no cells
      const bool bnd = L.nyn && (y == 0 || y == n - 1);
      sweep_tile_cell(k, kb, bnd, E0, E1, E2, (rr + 1) * kSwW + cc + kSwPad - 1, Qs, PQ,
                      rr * kSwW + cc + kSwPad - 1);
    }
  }
  __syncthreads();
  {
    const int per = tw >> 1;
    for (int t = threadIdx.x; t < th * per; t += kSwThreads) {
      const int rr = t / per, y = y0 + rr;
      const int cc = 2 * (t - rr * per) + ((x0 + y + 1) & 1);
      const bool bnd = L.nyn && (y == 0 || y == n - 1);
      sweep_tile_cell(k, kb, bnd, E0, E1, E2, (rr + 2) * kSwW + cc + kSwPad, Qs, PQ,
                      (rr + 1) * kSwW + cc + kSwPad);
    }
  }
  __syncthreads();
  // the tile to the destination copy, float4 rows
  const int q4 = tw >> 2;
  for (int t = threadIdx.x; t < th * q4; t += kSwThreads) {
    const int rr = t / q4, c4 = t - rr * q4;
    const size_t g = (size_t)(y0 + rr) * m + x0 + 4 * c4;
    const int se = (rr + 2) * kSwW + kSwPad + 4 * c4;
    *reinterpret_cast<float4*>(S.dphi + g) = *reinterpret_cast<const float4*>(E0 + se);
    *reinterpret_cast<float4*>(S.dmu + g) = *reinterpret_cast<const float4*>(E1 + se);
    *reinterpret_cast<float4*>(S.dka + g) = *reinterpret_cast<const float4*>(E2 + se);
  }
}

template <int TY>
__global__ void __launch_bounds__(kSwThreads) k_sweep32_tiles(Lev32 L, SweepSrc S, Coef32 k, Coef32 kb,
                                                              const __grid_constant__ SweepMaps M, int use_tma) {
  extern __shared__ unsigned char sw_raw[];
  const int SF = sweep_stage_floats(TY);
  float* const base = reinterpret_cast<float*>(
      sw_raw + ((128u - ((uint32_t)__cvta_generic_to_shared(sw_raw) & 127u)) & 127u));   // stage s at base + s SF
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(base + 2 * SF);            // mbarrier of stage s: bar0 + 8 s
  if (threadIdx.x == 0) {
    sw_bar_init(bar0);
    sw_bar_init(bar0 + 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_enter();
  const int m = L.m, n = L.n;
  const int tiles_x = (m + kSwX - 1) / kSwX, ntiles = tiles_x * ((n + TY - 1) / TY);
  uint32_t parity = 0u;   // bit s: phase parity of stage s's next tensor-copy wait
  int tile = blockIdx.x;
  bool tma_cur = false;
  const int withheld = g_sw_withhold != 0 ? tiles_x + 1 : -1;   // test hook: tile (1, 1) gets no copies
  if (tile < ntiles)
    tma_cur = sweep_tile_load<TY>(L, S, M, use_tma != 0, (tile % tiles_x) * kSwX, (tile / tiles_x) * TY, base, bar0,
                                  tile == withheld);
  for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
    // this tile's copies have landed (every thread's, or the tensor copies on the
    // stage's mbarrier), and every warp is done with the previous tile, whose stage
    // the next tile's copies now reuse
    const int st = it & 1;
    bool ok = true;
    if (tma_cur) {
      ok = sw_wait(bar0 + 8u * st, (parity >> st) & 1u);
      parity ^= 1u << st;
    } else {
      cp_async_wait_all();
    }
    if (__syncthreads_or(!ok)) {
      // a tensor copy did not arrive: poison this CTA's tiles so that the defect the
      // solver computes from them is not finite and the step reports DIVERGED, give
      // the copy a last bounded wait, and stop
      const float nan = __int_as_float(0x7fffffff);
      for (int t2 = tile; t2 < ntiles; t2 += gridDim.x) {
        const int x0 = (t2 % tiles_x) * kSwX, y0 = (t2 / tiles_x) * TY;
        const int tw = min(kSwX, m - x0), th = min(TY, n - y0);
        for (int q = threadIdx.x; q < tw * th; q += kSwThreads) {
          const size_t g = (size_t)(y0 + q / tw) * m + x0 + q % tw;
          S.dphi[g] = nan;
          S.dmu[g] = nan;
          S.dka[g] = nan;
        }
      }
      if (threadIdx.x == 0) sw_wait(bar0 + 8u * st, (parity ^ (1u << st)) >> st & 1u);
      return;
    }
    const int next = tile + gridDim.x;
    bool tma_next = false;
    if (next < ntiles)
      tma_next = sweep_tile_load<TY>(L, S, M, use_tma != 0, (next % tiles_x) * kSwX, (next / tiles_x) * TY,
                                     base + (st ^ 1) * SF, bar0 + 8u * (st ^ 1), next == withheld);
    float* E0 = base + st * SF;
    const int x0 = (tile % tiles_x) * kSwX, y0 = (tile / tiles_x) * TY;
    const int tw = min(kSwX, m - x0), th = min(TY, n - y0);
    if (tw == kSwX && th == TY)
      sweep_tile_compute<TY, true>(L, k, kb, E0, x0, y0, tw, th, S);
    else
      sweep_tile_compute<TY, false>(L, k, kb, E0, x0, y0, tw, th, S);
    tma_cur = tma_next;
  }
}

// The instantiation for a tile height (4, 8, 16 or 32 rows).
using SweepKernel = void (*)(Lev32, SweepSrc, Coef32, Coef32, SweepMaps, int);
SweepKernel sweep_kernel(int ty) {
  switch (ty) {
    case 4: return k_sweep32_tiles<4>;
    case 8: return k_sweep32_tiles<8>;
    case 16: return k_sweep32_tiles<16>;
    default: return k_sweep32_tiles<32>;
  }
}

int sweep_tiles_per_sm(int ty);

// Whether level F takes the one-launch tiled sweep (its second copy of e exists and it
// is large enough for the handle's setting).
bool sweep_tiled(const mpfc_s* H, const Lev32& F) {
  return H->sweep_tile_rows > 0 && F.xphi && (long long)F.m * F.n >= H->sweep_tile_cells &&
         sweep_tiles_per_sm(H->sweep_tile_rows) > 0;
}

// Resident CTAs per SM of the tiled sweep with tiles of ty rows on the current device
// (raises that instantiation's dynamic shared-memory limit first), cached per device
// and tile height; 0 if the GPU cannot run it.
int sweep_tiles_per_sm(int ty) {
  constexpr int kDevs = 64;
  static std::atomic<int> cache[kDevs][6];   // tile heights 1 << idx; 0: not queried yet
  int dev = 0, idx = 0;
  while ((1 << idx) < ty && idx < 5) ++idx;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) dev = -1;
  if (dev >= 0)
    if (int c = cache[dev][idx].load()) return c;
  const size_t smem = sweep_smem_bytes(ty);
  int per_sm = 0;
  if (cudaFuncSetAttribute(sweep_kernel(ty), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel(ty), kSwThreads, smem) != cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    return 0;
  }
  if (dev >= 0) cache[dev][idx].store(per_sm);
  return per_sm;
}

// The driver's tensor-map encoder (cuTensorMapEncodeTiled), looked up once.
PFN_cuTensorMapEncodeTiled_v12000 sweep_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    (void)cudaGetLastError();
  });
  return fn;
}

// 2-D tensor map of one m x n FP32 plane with boxes of kSwW columns x rows rows (no
// swizzle; the plane and its row pitch m * 4 bytes are 16-byte aligned, m % 4 == 0).
bool sweep_plane_map(CUtensorMap* map, const float* plane, int m, int n, int rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = sweep_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(plane) & 15) || (m % 4)) return false;
  cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)m * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)kSwW, (cuuint32_t)rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(plane), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launches one tiled sweep reading e from (fp, fm, fk) and writing it to (tp, tm, tk).
void launch_sweep_tiles(const mpfc_s* H, const Lev32& F, const float* fp, const float* fm, const float* fk, float* tp,
                        float* tm, float* tk, const Coef32& kf, const Coef32& kb, cudaStream_t s) {
  const int ty = H->sweep_tile_rows;
  const size_t smem = sweep_smem_bytes(ty);
  const int per_sm = sweep_tiles_per_sm(ty);   // >= 1 (sweeps32 falls back when it is 0)
  const long long ntiles = (long long)((F.m + kSwX - 1) / kSwX) * ((F.n + ty - 1) / ty);
  const long long cap = (long long)per_sm * mpfc::sm_count();
  const int grid = (int)(ntiles < cap ? ntiles : cap);
  SweepSrc S = {fp, fm, fk, tp, tm, tk};
  SweepMaps M;
  memset(&M, 0, sizeof(M));
  const float* eplanes[3] = {fp, fm, fk};
  const float* qplanes[4] = {F.q, F.r1, F.r2, F.r3};
  bool tma = true;
  for (int p = 0; p < 3 && tma; ++p) tma = sweep_plane_map(&M.e[p], eplanes[p], F.m, F.n, ty + 4);
  for (int p = 0; p < 4 && tma; ++p) tma = sweep_plane_map(&M.qr[p], qplanes[p], F.m, F.n, ty + 2);
  mpfc_launch(H->shape, sweep_kernel(ty), dim3(grid), dim3(kSwThreads), smem, s, F, S, kf, kb, M, tma ? 1 : 0);
}

void sweeps32(const mpfc_s* H, const Lev32& F, const Coef32& kf, const Coef32& kb, int sweeps, cudaStream_t s) {
  const mpfc_launch_shape& sh = H->shape;
  int done = 0;
  if (sweep_tiled(H, F))   // pairs of one-launch sweeps, there and back: e ends in its own planes
    for (; done + 2 <= sweeps; done += 2) {
      launch_sweep_tiles(H, F, F.ephi, F.emu, F.eka, F.xphi, F.xmu, F.xka, kf, kb, s);
      launch_sweep_tiles(H, F, F.xphi, F.xmu, F.xka, F.ephi, F.emu, F.eka, kf, kb, s);
    }
  dim3 g = mpfc_grid_of(sh, F.m / 2, F.n), b = mpfc_blk_for(sh, F.m / 2, F.n);
  for (; done < sweeps; ++done) {
    mpfc_launch(sh, k_smooth32, g, b, 0, s, F, kf, kb, 0);
    mpfc_launch(sh, k_smooth32, g, b, 0, s, F, kf, kb, 1);
  }
}

int inner_cycles_of(const mpfc_s* H) { return H->p.inner_cycles > 0 ? H->p.inner_cycles : 2; }

// ---------------------------------------------------------------------------
// The coarse end of an inner V-cycle in one CTA with every level in shared memory:
// the sweeps, defect restrictions, coarsest solve and prolongations of the levels
// lt .. L-1, in the order of the per-level launches and with the same cell functions
// (so the same bits), separated by __syncthreads instead of kernel boundaries.  The
// FP32 work of a small level is far below a launch's cost.  Level lt's correction is
// read at the start and written back at the end; its defect source and every level's
// q are read from the global planes.
// ---------------------------------------------------------------------------
constexpr int kMaxTail32 = 8;
constexpr int kTail32Threads = 1024;
constexpr size_t kTail32MaxSmem = 200 * 1024;   // dynamic shared memory, below the 227 KB opt-in limit

struct Tail32Args {
  int nlev, nu1, nu2;
  const float* K3f;
  Lev32 g[kMaxTail32];    // the levels' global planes
  Coef32 k[kMaxTail32], kb[kMaxTail32];   // interior and Neumann-row cell systems
};

// e_f += P e_c at one fine cell, with the tile version's order of operations.
__device__ __forceinline__ void prolong32_fine(const float* ec, float* ef, int mc, int nc, int nyn, int fi, int fj) {
  const int I = fi >> 1, J = fj >> 1;
  const int Ix = wrapm(I + ((fi & 1) ? 1 : -1), mc), Jy = ywrap(J + ((fj & 1) ? 1 : -1), nc, nyn);
  const float e00 = ec[J * mc + I], ex = ec[J * mc + Ix], ey = ec[Jy * mc + I], exy = ec[Jy * mc + Ix];
  const float w9 = 9.f / 16.f, w3 = 3.f / 16.f, w1 = 1.f / 16.f;
  const int id = fj * (2 * mc) + fi;
  ef[id] += fmaf(w3, ex + ey, fmaf(w1, exy, w9 * e00));
}

size_t tail32_smem(const Lev32* levs, int nlev) {
  size_t cells = 0;
  for (int l = 0; l < nlev; ++l) cells += (size_t)levs[l].m * levs[l].n;
  const size_t gc = (size_t)levs[nlev - 1].m * levs[nlev - 1].n;
  return 7 * cells * sizeof(float) + coarse32_smem(levs[nlev - 1]) + 2 * gc * gc * sizeof(float);
}

__global__ void __launch_bounds__(kTail32Threads) k_tail32(const __grid_constant__ Tail32Args A) {
  extern __shared__ float ts[];
  __shared__ Lev32 sl[kMaxTail32];
  const int tid = threadIdx.x, nt = blockDim.x;
  // shared layout: the levels' planes, the coarse solve's scratch, then a copy of the
  // coarsest grid's K3 and c L blocks, loaded before the wait for the previous kernel
  // (they are written once, when the handle is created), out of the coarse solve's path
  float* scratch = ts;
  for (int l = 0; l < A.nlev; ++l) scratch += 7 * A.g[l].m * A.g[l].n;
  const Lev32& Cg = A.g[A.nlev - 1];
  const int gcc = Cg.m * Cg.n;
  float* k3s = scratch + gcc * (gcc + 1) + 4 * gcc;
  for (int t = tid; t < 2 * gcc * gcc; t += nt) k3s[t] = A.K3f[t];
  pdl_enter();
  if (tid == 0) {
    float* p = ts;
    for (int l = 0; l < A.nlev; ++l) {
      const int G = A.g[l].m * A.g[l].n;
      Lev32 v = A.g[l];
      v.ephi = p;
      v.emu = p + G;
      v.eka = p + 2 * G;
      v.r1 = p + 3 * G;
      v.r2 = p + 4 * G;
      v.r3 = p + 5 * G;
      v.q = p + 6 * G;
      sl[l] = v;
      p += 7 * G;
    }
  }
  __syncthreads();
  {
    const Lev32& T = sl[0];
    const Lev32& G0 = A.g[0];
    const int G = T.m * T.n;
    for (int t = tid; t < G; t += nt) {
      T.ephi[t] = G0.ephi[t];
      T.emu[t] = G0.emu[t];
      T.eka[t] = G0.eka[t];
      T.r1[t] = G0.r1[t];
      T.r2[t] = G0.r2[t];
      T.r3[t] = G0.r3[t];
    }
    for (int l = 0; l < A.nlev; ++l) {
      const int Gl = A.g[l].m * A.g[l].n;
      for (int t = tid; t < Gl; t += nt) sl[l].q[t] = A.g[l].q[t];
    }
  }
  __syncthreads();
  for (int l = 0; l < A.nlev - 1; ++l) {
    const Lev32& F = sl[l];
    const Lev32& C = sl[l + 1];
    const int half = F.m >> 1, hc = half * F.n;
    for (int sw = 0; sw < A.nu1; ++sw)
      for (int color = 0; color < 2; ++color) {
        for (int t = tid; t < hc; t += nt) {
          const int j = t / half, x = t - j * half;
          smooth32_cell<false>(F, A.k[l], A.kb[l], 2 * x + ((j + color) & 1), j);
        }
        __syncthreads();
      }
    const int cc = C.m * C.n;
    for (int t = tid; t < cc; t += nt) restrict_defect32_cell<false>(F, C, A.k[l], t % C.m, t / C.m);
    __syncthreads();
  }
  coarse32_block(sl[A.nlev - 1], A.k[A.nlev - 1], k3s, scratch);
  __syncthreads();
  for (int l = A.nlev - 2; l >= 0; --l) {
    const Lev32& F = sl[l];
    const Lev32& C = sl[l + 1];
    const int fc = F.m * F.n;
    for (int t = tid; t < fc; t += nt) {
      const int fi = t % F.m, fj = t / F.m;
      prolong32_fine(C.ephi, F.ephi, C.m, C.n, C.nyn, fi, fj);
      prolong32_fine(C.emu, F.emu, C.m, C.n, C.nyn, fi, fj);
      prolong32_fine(C.eka, F.eka, C.m, C.n, C.nyn, fi, fj);
    }
    __syncthreads();
    const int half = F.m >> 1, hc = half * F.n;
    for (int sw = 0; sw < A.nu2; ++sw)
      for (int color = 0; color < 2; ++color) {
        for (int t = tid; t < hc; t += nt) {
          const int j = t / half, x = t - j * half;
          smooth32_cell<false>(F, A.k[l], A.kb[l], 2 * x + ((j + color) & 1), j);
        }
        __syncthreads();
      }
  }
  {
    const Lev32& T = sl[0];
    const Lev32& G0 = A.g[0];
    const int G = T.m * T.n;
    for (int t = tid; t < G; t += nt) {
      G0.ephi[t] = T.ephi[t];
      G0.emu[t] = T.emu[t];
      G0.eka[t] = T.eka[t];
    }
  }
}

// First level of the shared-memory tail: the finest level of at most shape.tail_cells
// cells whose levels down to the coarsest fit in shared memory, leaving at least one
// level above the coarsest; nlev when no tail is used.
int tail32_first_level(const mpfc_s* H) {
  const int L = H->nlev;
  if (H->shape.tail_cells <= 0 || L < 2) return L;
  int lt = L - 1;
  while (lt > 0 && (long long)H->lev32[lt - 1].m * H->lev32[lt - 1].n <= H->shape.tail_cells &&
         L - (lt - 1) <= kMaxTail32 && tail32_smem(H->lev32 + lt - 1, L - lt + 1) <= kTail32MaxSmem)
    --lt;
  return lt > L - 2 ? L : lt;
}

void launch_tail32(mpfc_s* H, int scheme, int lt, cudaStream_t s) {
  Tail32Args A;
  A.nlev = H->nlev - lt;
  A.nu1 = H->p.nu1;
  A.nu2 = H->p.nu2;
  A.K3f = H->K3f[scheme - 1];
  for (int i = 0; i < A.nlev; ++i) {
    A.g[i] = H->lev32[lt + i];
    A.k[i] = coef32_of(H->coef[scheme - 1][lt + i]);
    A.kb[i] = coef32_of(H->coefb[scheme - 1][lt + i]);
  }
  mpfc_launch(H->shape, k_tail32, dim3(1), dim3(kTail32Threads), tail32_smem(H->lev32 + lt, A.nlev), s, A);
}

// One inner correction-scheme V-cycle.
void enqueue_inner_vcycle(mpfc_s* H, int scheme, cudaStream_t s) {
  const mpfc_params& p = H->p;
  const mpfc_launch_shape& sh = H->shape;
  const int L = H->nlev;
  const int lt = tail32_first_level(H);
  const int down = lt < L ? lt : L - 1;   // levels swept and restricted by per-level launches
  for (int l = 0; l < down; ++l) {
    const Lev32& F = H->lev32[l];
    const Lev32& C = H->lev32[l + 1];
    Coef32 kf = coef32_of(H->coef[scheme - 1][l]), kb = coef32_of(H->coefb[scheme - 1][l]);
    sweeps32(H, F, kf, kb, p.nu1, s);
    mpfc_launch(sh, k_restrict_defect32, mpfc_grid_of(sh, C.m, C.n), mpfc_blk_for(sh, C.m, C.n), 0, s, F, C, kf);
  }
  if (lt < L) {
    launch_tail32(H, scheme, lt, s);
  } else {
    const Lev32& Cc = H->lev32[L - 1];
    mpfc_launch(sh, k_coarse32, dim3(1), dim3(256), coarse32_smem(Cc), s, Cc, coef32_of(H->coef[scheme - 1][L - 1]),
                (const float*)H->K3f[scheme - 1]);
  }
  for (int l = down - 1; l >= 0; --l) {
    const Lev32& F = H->lev32[l];
    const Lev32& C = H->lev32[l + 1];
    Coef32 kf = coef32_of(H->coef[scheme - 1][l]), kb = coef32_of(H->coefb[scheme - 1][l]);
    mpfc_launch(sh, k_prolong32, grid_of(C.m, C.n), kBlk, 0, s, F, C);
    sweeps32(H, F, kf, kb, p.nu2, s);
  }
}

void enqueue_defect(mpfc_s* H, int scheme, int mode, cudaGraphConditionalHandle hnd, int set_cond, cudaStream_t s) {
  const Lev& L0 = H->lev[0];
  int blocks = mpfc_reduce_blocks((size_t)L0.m * L0.n);
  if (scheme == 1)
    mpfc_launch(H->shape, k_defect<1>, dim3(blocks), dim3(256), 0, s, L0, H->coef[0][0], H->lev32[0], H->ctl,
                H->partials, mode, hnd, set_cond);
  else
    mpfc_launch(H->shape, k_defect<2>, dim3(blocks), dim3(256), 0, s, L0, H->coef[1][0], H->lev32[0], H->ctl,
                H->partials, mode, hnd, set_cond);
}

// Body of one outer iteration: restrict q to the coarse grids, the inner V-cycles,
// u += e, and the FP64 defect with the loop test.
void outer_body(mpfc_s* H, int scheme, cudaStream_t s, cudaGraphConditionalHandle hnd, int set_cond) {
  for (int l = 1; l < H->nlev; ++l) {
    const Lev32& C = H->lev32[l];
    mpfc_launch(H->shape, k_restrict_q, grid_of(C.m, C.n), kBlk, 0, s, (const float*)H->lev32[l - 1].q, C.q, C.m,
                C.n);
  }
  for (int c = 0; c < inner_cycles_of(H); ++c) enqueue_inner_vcycle(H, scheme, s);
  const Lev& L0 = H->lev[0];
  mpfc_launch(H->shape, k_update, dim3(mpfc_reduce_blocks((size_t)L0.m * L0.n)), dim3(256), 0, s, L0, H->lev32[0]);
  enqueue_defect(H, scheme, 1, hnd, set_cond, s);
}

void graph_body(mpfc_s* H, int scheme, cudaStream_t s) { outer_body(H, scheme, s, H->cur_handle, 1); }

}  // namespace

size_t mpfc_fp32_carve(mpfc_s* H, const mpfc_params* p, size_t* off, char* base, int nlev) {
  if (p->precision != MPFC_FP32_INNER) return 0;
  size_t start = *off;
  auto take = [&](size_t count) -> float* {
    float* ptr = base ? reinterpret_cast<float*>(base + *off) : nullptr;
    *off = (*off + count * sizeof(float) + 255) & ~(size_t)255;
    return ptr;
  };
  int m = p->m, n = p->n;
  double h = p->h;
  for (int l = 0; l < nlev; ++l) {
    size_t G = (size_t)m * n;
    Lev32 v;
    v.m = m;
    v.n = n;
    v.nyn = p->bc == MPFC_BC_NEUMANN_Y;
    v.h = (float)h;
    v.ephi = take(G);
    v.emu = take(G);
    v.eka = take(G);
    v.r1 = take(G);
    v.r2 = take(G);
    v.r3 = take(G);
    v.q = take(G);
    // second copy of e for the one-launch sweeps (float4 rows need m a multiple of 4)
    v.xphi = v.xmu = v.xka = nullptr;
    if (m % 4 == 0) {
      v.xphi = take(G);
      v.xmu = take(G);
      v.xka = take(G);
    }
    if (H && base) H->lev32[l] = v;
    m /= 2;
    n /= 2;
    h *= 2.0;
  }
  return *off - start;
}

extern "C" int mpfc_fp32_test_withhold_copy(int withhold, long long spin_cycles) {
  if (withhold < 0 || withhold > 1 || spin_cycles < 0) return MPFC_ERR_INVALID;
  const int w = withhold;
  const long long lim = spin_cycles > 0 ? spin_cycles : kSwSpinLimit;
  cudaError_t e = cudaMemcpyToSymbol(g_sw_withhold, &w, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_sw_spin_limit, &lim, sizeof(long long));
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "fp32 sweep test hook", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  return MPFC_OK;
}

extern "C" int mpfc_set_fp32_sweep(mpfc_t* H, int tile_rows, int min_cells) {
  if (!H || H->p.precision != MPFC_FP32_INNER || min_cells < 0 ||
      (tile_rows != 0 && tile_rows != 4 && tile_rows != 8 && tile_rows != 16 && tile_rows != 32))
    return MPFC_ERR_INVALID;
  H->sweep_tile_rows = tile_rows;
  H->sweep_tile_cells = min_cells;
  mpfc_drop_graphs(H);
  return MPFC_OK;
}

extern "C" int mpfc_fp32_time_smooth(mpfc_t* H, int level, int sweeps, float* ms) {
  if (!H || H->p.precision != MPFC_FP32_INNER || level < 0 || level >= H->nlev || sweeps < 1 || !ms)
    return MPFC_ERR_INVALID;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "cudaEventCreate", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  if ((e = cudaEventRecord(e0, H->stream)) == cudaSuccess) {
    sweeps32(H, H->lev32[level], coef32_of(H->coef[0][level]), coef32_of(H->coefb[0][level]), sweeps, H->stream);
    if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaEventRecord(e1, H->stream)) == cudaSuccess &&
        (e = cudaEventSynchronize(e1)) == cudaSuccess)
      e = cudaEventElapsedTime(ms, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "mpfc_fp32_time_smooth", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  return MPFC_OK;
}

int mpfc_fp32_init(mpfc_s* H) {
  if (H->p.precision != MPFC_FP32_INNER) return MPFC_OK;
  H->K3f[0] = H->K3[0];
  H->K3f[1] = H->K3[1];
  cudaError_t e = cudaFuncSetAttribute(k_tail32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTail32MaxSmem);
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "shared memory of the FP32 tail kernel", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  return MPFC_OK;
}

void mpfc_fp32_destroy(mpfc_s* H) { (void)H; }

// Step graph of the mixed-precision form: prologue (FP64 source and guess), FP64
// defect (sets the loop condition), WHILE(cond){ outer body }, psi update.
int mpfc_fp32_enqueue_step(mpfc_s* H, int scheme, cudaStream_t cs, cudaGraphConditionalHandle hnd) {
  mpfc_enqueue_prologue(H, scheme, cs);
  enqueue_defect(H, scheme, 0, hnd, 1, cs);
  int rc = mpfc_capture_while(H, cs, hnd, &graph_body, scheme);
  if (rc != MPFC_OK) return rc;
  mpfc_enqueue_commit(H, scheme, cs);
  return MPFC_OK;
}

int mpfc_fp32_step_stream(mpfc_s* H, int scheme) {
  MpfcRange range("mpfc step (FP32 inner)");
  cudaStream_t s = H->stream;
  mpfc_enqueue_prologue(H, scheme, s);
  enqueue_defect(H, scheme, 0, 0, 0, s);
  for (;;) {
    Ctl c;
    cudaError_t e = cudaMemcpyAsync(&c, H->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      mpfc_set_cuda_error(e, "fp32 loop test", __FILE__, __LINE__);
      return MPFC_ERR_CUDA;
    }
    if (!mpfc_host_continue(&c)) break;
    MpfcRange orange("outer iteration");
    outer_body(H, scheme, s, 0, 0);
  }
  mpfc_enqueue_commit(H, scheme, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "fp32 step", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  return MPFC_OK;
}
