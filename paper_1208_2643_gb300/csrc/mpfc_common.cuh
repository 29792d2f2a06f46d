// Shared definitions of the libmpfc CUDA path (device structs, constants, helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpfc {

// Streaming multiprocessors of the current device (queried once per device), for the
// grids sized to the GPU: persistent kernels run one CTA (or a few) per SM.
int sm_count();

constexpr int kMaxLevels = 16;
constexpr int kMaxCoarseCells = 64;    // coarsest level solved by dense Newton in one CTA
constexpr int kMaxPartials = 1024;     // blocks of a deterministic two-pass reduction
constexpr int kMaxSums = 8;            // sums per reduction
constexpr int kInfoCap = 1024;         // per-step records per mpfc_step chunk

// One grid level: SoA planes, row-major [n][m].
struct Lev {
  int m, n;
  int nyn;                  // 1: homogeneous Neumann in y (ghost row = boundary row), 0: periodic
  double h;
  double *phi, *mu, *ka;    // u = (phi, mu, kappa)
  double *S1, *S2, *S3;     // FAS source (tau-corrected below the finest level)
  double *b1, *b2, *b3;     // R u_f kept for the correction u_c_new - R u_f (levels >= 1)
  double* pk;               // phi^k on this level (scheme 2)
  const double* W;          // pinning weight on this level (Sec. 4.6, scheme 2), nullptr: none
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
  // the determinant divided by omega, so that its reciprocal is omega / det at once:
  double D0w;   // D0 / omega
  double aw;    // a / omega
  double a3w;   // 3 a / omega
  int relax;    // omega != 1
  int pad;
};

// Conversions between binary64 and binary32 done with integer operations on the IEEE
// 754 bit fields (sign, biased exponent, significand), so that they run on the integer
// pipes instead of GB300's narrow FP64 pipe.  The bit arithmetic covers magnitudes in
// the normal binary32 range [2^-126, 2^128) and zero; every other input (binary32
// subnormals and underflow, overflow, infinities, NaN) takes the hardware conversion
// instead, so each function equals its IEEE counterpart for every input (the tests
// check them against the hardware conversions, special values included).  One
// unsigned range test on the exponent selects the rare branch.
//   f64_to_f32_trunc: rounded toward zero (relative error < 2^-23);
//   f64_to_f32_rn:    rounded to nearest, ties to even;
//   f32_to_f64:       exact.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  unsigned int hi = (unsigned int)(b >> 32);
  unsigned int eb = (hi >> 20) & 0x7FFu;                 // binary64 biased exponent
  if (eb - (1023u - 126u) >= 254u) {                     // outside [2^-126, 2^128)
    if ((b << 1) == 0ull) return __uint_as_float(hi & 0x80000000u);
    return __double2float_rz(x);
  }
  unsigned int e = eb - 1023u + 127u;
  unsigned int f = (hi & 0x80000000u) | (e << 23) | (unsigned int)((b >> 29) & 0x7FFFFFull);
  return __uint_as_float(f);
}
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
  unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  unsigned int eb = (unsigned int)(mag >> 52);
  if (eb - (1023u - 126u) >= 254u) {                     // outside [2^-126, 2^128)
    if (mag == 0ull) return __uint_as_float(sign);
    return __double2float_rn(x);
  }
  // binary32 magnitude bits with the exponent re-biased and the significand cut to 23
  // bits, then round to nearest even on the 29 dropped bits (a carry into the exponent
  // field is the correct result of rounding up a significand of all ones, up to
  // infinity past the largest finite binary32)
  unsigned long long keep = (mag >> 29) - ((unsigned long long)(1023 - 127) << 23);
  unsigned long long rest = mag & 0x1FFFFFFFull;
  unsigned long long half = 0x10000000ull;
  if (rest > half || (rest == half && (keep & 1ull))) keep += 1ull;
  return __uint_as_float(sign | (unsigned int)keep);
}
__device__ __forceinline__ double f32_to_f64(float f) {
  unsigned int u = __float_as_uint(f);
  unsigned int ef = (u >> 23) & 0xFFu;                   // binary32 biased exponent
  if (ef - 1u >= 254u) {                                 // zero, subnormal, infinity or NaN
    if ((u << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));
    return (double)f;
  }
  unsigned long long e = (unsigned long long)(ef - 127u + 1023u);
  unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) | (e << 52) |
                         ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}

// Reciprocal by one Newton-Raphson step (r <- r + r (1 - x r), Newton's method for
// f(r) = 1/r - x) from the correctly rounded single-precision reciprocal of x rounded
// down to single.  The seed's relative error is below 2^-22.4; one step squares it:
// |r x - 1| < 2^-44 for x in the normal single range.  The smoother's cell solve needs
// no more because it scales a correction with it (the correction d = A^-1 r of the
// cell's residual r), so its error shrinks with the residual and leaves the fixed point
// alone.
__device__ __forceinline__ double rcp_nr(double x) {
  double r = f32_to_f64(__frcp_rn(f64_to_f32_trunc(x)));
  return fma(r, fma(-x, r, 1.0), r);
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with programmatic
// stream serialization may be scheduled while its predecessor on the stream is still
// running.  griddepcontrol.wait blocks until that predecessor grid has completed and
// its memory operations are visible; launch_dependents then lets the launch of the
// next kernel begin while this one runs, so launch latency overlaps execution instead
// of adding to it.  For a kernel launched without the attribute both are no-ops.
// Every kernel of the time step calls this before its first memory access.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Loads of the per-cell stencil functions, by the kernel's memory situation:
//   kLdNC:    the read-only (non-coherent) path, for data no thread writes during the
//             kernel (the per-level kernels);
//   kLdL2:    L2 loads (ld.global.cg), for reading what other CTAs of a cluster wrote
//             before a release/acquire cluster barrier;
//   kLdPlain: plain loads, for a single CTA (its writes and reads meet in its own L1,
//             ordered by __syncthreads).
constexpr int kLdNC = 0, kLdL2 = 1, kLdPlain = 2;
template <int LD>
__device__ __forceinline__ double ldv(const double* p) {
  if (LD == kLdNC) return __ldg(p);
  if (LD == kLdL2) return __ldcg(p);
  return *p;
}
// A cell's own value, which the same thread may write later in the kernel.
template <int LD>
__device__ __forceinline__ double ldown(const double* p) {
  if (LD == kLdL2) return __ldcg(p);
  return *p;
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
// Stored row of row j in -1..n: periodic wrap, or with the Neumann rule of App. A
// ((A.7): phi_{i,0} = phi_{i,1}, phi_{i,n+1} = phi_{i,n}) the boundary row itself.
__device__ __forceinline__ int ywrap(int j, int n, int nyn) {
  return nyn ? (j < 0 ? 0 : (j >= n ? n - 1 : j)) : wrapm(j, n);
}

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
