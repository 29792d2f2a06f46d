// Shared definitions of the libmpfc CUDA path (device structs, constants, helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpfc {

constexpr int kMaxLevels = 16;
constexpr int kMaxCoarseCells = 64;    // coarsest level solved by dense Newton in one CTA
constexpr int kMaxPartials = 1024;     // blocks of a deterministic two-pass reduction
constexpr int kMaxSums = 8;            // sums per reduction
constexpr int kInfoCap = 1024;         // per-step records per mpfc_step chunk

// One grid level: SoA planes, row-major [n][m].
struct Lev {
  int m, n;
  double h;
  double *phi, *mu, *ka;    // u = (phi, mu, kappa)
  double *S1, *S2, *S3;     // FAS source (tau-corrected below the finest level)
  double *b1, *b2, *b3;     // R u_f kept for the correction u_c_new - R u_f (levels >= 1)
  double* pk;               // phi^k on this level (scheme 2)
};

// Coefficients of the cell system of App. B on one level, for one scheme.
//   row 1: phi + a mu                 = S1 + cmu * sum_nb mu
//   row 2: -(gam + q) phi + mu + b ka = S2 + e + ih2 * sum_nb ka
//   row 3: b3 phi + ka                = S3 + th2 * sum_nb phi
struct Coef {
  double c, gam, theta, omega;
  double cmu;   // c / h^2
  double a;     // 4 c / h^2
  double ih2;   // 1 / h^2
  double b;     // 4 / h^2
  double b3;    // 4 theta / h^2
  double th2;   // theta / h^2
  double D0;    // 1 + a gam + a b b3    (determinant without the cubic)
  double Q0;    // gam + b b3            (Cramer numerator of mu without the cubic)
  double a3;    // 3 a                   (scheme 1: det = D0 + 3 a p^2)
  double omw;   // 1 - omega
  int relax;    // omega != 1
  int pad;
};

// Reciprocal by one Newton-Raphson step (r <- r + r (1 - x r), Newton's method for
// f(r) = 1/r - x) from the correctly rounded single-precision reciprocal of x.  The
// seed's relative error is below 2^-23 (including the rounding of x to single), and
// one step squares it: |r x - 1| < 2^-45 for x in the normal single range.  The
// smoother's cell solve needs no more: its error only perturbs an iterate, not the
// fixed point.
__device__ __forceinline__ double rcp_nr(double x) {
  double r = (double)__frcp_rn(__double2float_rn(x));
  return fma(r, fma(-x, r, 1.0), r);
}

// Device-side control block of the time stepper.
struct Ctl {
  double res0, res, tol;
  int cycles, max_cycles, fixed_cycles, status;   // status: 0 ok, 2 diverged
  int skip, halt, slot, pad0;
  unsigned int counter;                           // last-block-done counter of reductions
  unsigned int pad1;
  double sums[kMaxSums];                          // results of the last reduction
};

struct StepRecord {      // mirrors mpfc_step_info
  int cycles;
  int status;
  double res0;
  double res_final;
};

__device__ __forceinline__ int wrapm(int i, int m) { return i < 0 ? i + m : (i >= m ? i - m : i); }

// Nonlinear term of N^(2) and its derivative (App. B.1: phi^3; App. B.2:
// chi(phi, phik)(phi + phik)/2 with chi(a, b) = (a^2 + b^2)/2).
template <int SCH>
__device__ __forceinline__ double g_of(double p, double pk) {
  if (SCH == 1) return p * p * p;
  return 0.25 * (p * p + pk * pk) * (p + pk);
}
template <int SCH>
__device__ __forceinline__ double dg_of(double p, double pk) {
  if (SCH == 1) return 3.0 * p * p;
  return 0.25 * (3.0 * p * p + 2.0 * p * pk + pk * pk);
}

}  // namespace mpfc
