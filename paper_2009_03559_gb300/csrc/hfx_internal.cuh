// Internal device-side definitions of the HFX library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hfx {

// ---------------------------------------------------------------------------
// Per-class recurrence description (generated tables, see gen_eri_tables.py)
// ---------------------------------------------------------------------------
struct EriClassInfo {
  int la, lb, lc, ld, E, F, Lt;
  int n_acc, work_base, scratch;       // group scratch (doubles): acc | VRR slots
  int n_bra_lv, n_ket_lv;
  int lv_off[8], lv_n[8];              // VRR levels: op offset (in uint4) and count
  int acc_off;                         // into kAccSrc: (acc index | slot << 16) entries
  int n_accl;                          // accumulators added after the levels (others are
                                       // accumulated by the op that makes them)
  int n_post;                          // post-contraction stages
  int post_type[8], post_off[8], post_n[8];  // 0 bra HRR, 1 ket HRR, 2 spherical
  int out_base;                        // final spherical block in group scratch
  int dims[4];                         // final block extents (a, b, c, d)
  int flops_prim, flops_quartet;       // flop model (VRR+acc per primitive quartet;
                                       // HRR+spherical+digest per contracted quartet)
  int flops_digest;                    // the digest part of flops_quartet (always FP64)
};

extern const EriClassInfo* class_info_host();

// ---------------------------------------------------------------------------
// Boys function table: rows at x_g = g h, column 0 = exp(-x_g), columns 1..16 =
// F_0..F_15 at x_g (F_m(x) = int_0^1 u^{2m} exp(-x u^2) du).
// ---------------------------------------------------------------------------
constexpr int kBoysCols = 17;
constexpr double kBoysInvStep = 32.0;
constexpr double kBoysStep = 1.0 / 32.0;
constexpr double kBoysXmax = 60.0;
constexpr int kBoysRows = 60 * 32 + 2;
constexpr int kMaxLt = 8;

// ---------------------------------------------------------------------------
// Primitive-pair record (one per surviving primitive pair of a shell pair).
// C = sqrt(2) pi^{5/4} w_a w_b exp(-ab/p |AB|^2) / p so that the primitive
// quartet prefactor 2 pi^{5/2} K_ab K_cd / (p q sqrt(p+q)) = C_ab C_cd / sqrt(p+q).
// ---------------------------------------------------------------------------
struct __align__(16) PrimPair {
  double p, inv2p;     // exponent sum and 1/(2p)
  double P[3];         // Gaussian product centre
  double PA[3];        // P - A (A = centre of the pair's first shell)
  double C;            // prefactor (see above)
  double pad;
  // FP32 copies for the FP32 recurrences (conversions would run on the FP64 pipe)
  float pf, inv2pf, PAf[3], pad_f[3];
};

// Device arrays describing shell pairs (indexed by candidate-pair id).
struct PairArrays {
  const int* sa;            // first shell (l_a >= l_b)
  const int* sb;            // second shell
  const int* prim_off;      // first PrimPair of the pair
  const int* prim_n;        // number of surviving primitive pairs
  const double* AB;         // 3 per pair: A - B
  const PrimPair* prim;     // primitive-pair records
};

struct ShellArrays {
  const int* bf_off;        // first function of each shell
  const int* atom;          // atom of each shell
};

// ---------------------------------------------------------------------------
// FP64 reciprocal and reciprocal square root: FP32 hardware seed (relative error below
// 2^-22) refined by one Newton-Raphson step, which squares the error: below 1e-13
// relative, far inside what the exchange matrix needs (FP64 instructions are the scarce
// resource on this part).  Arguments are positive and well inside FP32 range.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rcp_nr(double x) {
  const double r = (double)__frcp_rn((float)x);
  return fma(r, fma(-x, r, 1.0), r);
}

__device__ __forceinline__ double rsqrt_nr(double x) {
  const double y = (double)rsqrtf((float)x);
  return fma(0.5 * y, fma(-x * y, y, 1.0), y);  // y (1 + (1 - x y^2)/2)
}

// F_m(x) for m = 0..mmax (mmax <= kMaxLt).  Below kBoysXmax: seven-term Taylor
// expansion of F_mmax and exp(-x) about the nearest grid point (|x - x_g| <= h/2),
// then downward recursion F_{m-1} = (2x F_m + e^{-x}) / (2m-1); for mmax <= 1 every
// order is expanded directly.  Above: F_0 = sqrt(pi/x)/2 and F_{m+1} = (m+1/2) F_m / x
// (the neglected terms are below exp(-60) relative to F_m for m <= 8).
__device__ __forceinline__ void boys_eval(int mmax, double x, const double* __restrict__ tab,
                                          double* F) {
  if (x < kBoysXmax) {
    int g = __double2int_rn(x * kBoysInvStep);
    double md = fma(-kBoysStep, (double)g, x);  // x - x_g
    md = -md;
    const double* row = tab + g * kBoysCols;
    double d2 = md * 0.5, d3 = md * (1.0 / 3.0), d4 = md * 0.25, d5 = md * 0.2, d6 = md * (1.0 / 6.0);
    if (mmax <= 1) {
      for (int m = 0; m <= mmax; ++m) {
        const double* f = row + 1 + m;
        double r = f[6];
        r = fma(r, d6, f[5]);
        r = fma(r, d5, f[4]);
        r = fma(r, d4, f[3]);
        r = fma(r, d3, f[2]);
        r = fma(r, d2, f[1]);
        F[m] = fma(r, md, f[0]);
      }
      return;
    }
    const double* f = row + 1 + mmax;
    double r = f[6];
    r = fma(r, d6, f[5]);
    r = fma(r, d5, f[4]);
    r = fma(r, d4, f[3]);
    r = fma(r, d3, f[2]);
    r = fma(r, d2, f[1]);
    F[mmax] = fma(r, md, f[0]);
    double e = fma(d6, 1.0, 1.0);
    e = fma(e, d5, 1.0);
    e = fma(e, d4, 1.0);
    e = fma(e, d3, 1.0);
    e = fma(e, d2, 1.0);
    e = fma(e, md, 1.0);
    e *= row[0];
    double x2 = x + x;
#pragma unroll
    for (int m = kMaxLt; m >= 1; --m) {
      if (m <= mmax) F[m - 1] = fma(x2, F[m], e) * (1.0 / (2 * m - 1));
    }
  } else {
    double ix = rcp_nr(x);
    double f0 = 0.886226925452758014 * rsqrt_nr(x);  // sqrt(pi)/2 / sqrt(x)
    F[0] = f0;
#pragma unroll
    for (int m = 0; m < kMaxLt; ++m) {
      if (m < mmax) F[m + 1] = F[m] * ((m + 0.5) * ix);
    }
  }
}

// Arguments of one class launch (passed by value).
struct EriLaunch {
  EriClassInfo ci;
  PairArrays pa;
  ShellArrays sh;
  const int* sorted;          // sorted pair index -> candidate-pair id
  const long long* qoff;      // exclusive scan of quartets per row (global), + total
  int row_begin, row_end;     // rows of this class pair
  int bra_bin_start, ket_bin_start;
  long long q_begin, q_count; // quartet range of this class pair
  int schedule;               // 0 quartet split, 1 bra-pair split, 2 dynamic chunks
  unsigned long long* work;   // schedule 2: next unclaimed quartet (relative to q_begin)
  int chunk;                  // schedule 2: quartets per claim
  const double* boys;
  double omega2;
  const double* P;
  double* K;
  int ld;
  // Schwarz-diagonal mode: quartet (p|p) for candidate pairs [diag_begin, diag_end)
  const int* diag_list;
  int diag_n;
  double* diag_Q;
  unsigned long long* busy;     // optional per-SM globaltimer busy ns (indexed by %smid)
  unsigned long long* counters; // optional: [0] primitive quartets evaluated, [1] quartets, [2] skipped
  const double* pmax;           // optional: max |P| of each shell-pair block (ns x ns)
  int ns;
  int skip_zero;                // skip quartets whose four density blocks are all zero
  int fp32_ok;                  // mixed precision allowed for this class
  double fp32_tau;              // FP32 iff Q_IJ Q_KL Pmax < fp32_tau, Pmax = max|P_blocks| ...
  const double* pglob;          // ... or, when non-NULL, *pglob = max |P| over the matrix
  double dens_tau;              // > 0: drop quartets with Q_IJ Q_KL max|P_blocks| < dens_tau
  const double* Qs;             // Schwarz factor of each sorted pair
  // batched launch (n_sys > 0): quartets of all systems' lists for this class, concatenated;
  // seg[s] = first index of system s (seg[n_sys] = total = q_count); batch[s] = that
  // system's record for this class (device memory)
  int n_sys;
  const long long* seg;
  const EriLaunch* batch;
};


}  // namespace hfx
