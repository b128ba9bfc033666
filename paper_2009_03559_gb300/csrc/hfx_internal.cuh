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
// Boys function tables, one per order L = 0..kMaxLt, rows at x_g = g h (h = 1/32,
// g = 0..kBoysRows-1).  Row g of table L holds the coefficients of the Taylor expansions
// about x_g in powers of d = x - x_g:
//   [0] x_g,  [1 + k] (-1)^k F_{L+k}(x_g) / k!,  [8 + k] (-1)^k exp(-x_g) / k!  (k = 0..6),
//   [15] 0,
// with F_m(x) = int_0^1 u^{2m} exp(-x u^2) du.  Seven terms with |d| <= h/2 leave a
// relative error below 5e-17.
// ---------------------------------------------------------------------------
constexpr int kBoysRowLen = 16;
constexpr float kBoysInvStepF = 32.0f;
constexpr double kBoysStep = 1.0 / 32.0;
constexpr double kBoysXmax = 60.0;
constexpr int kBoysXmaxHi = 0x404E0000;   // high word of 60.0 (low word 0)
constexpr int kBoysRows = 60 * 32 + 2;
constexpr int kMaxLt = 8;
constexpr int kBoysTableLen = kBoysRows * kBoysRowLen;   // doubles per order

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
  double inv2p3;       // 3/(2p)
  // FP32 copies for the FP32 recurrences
  float pf, inv2pf, PAf[3], Pf[3];
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
// Conversions and reciprocals that keep the FP64 pipe free.  On this part the FP64 pipe
// executes one warp instruction every 16 SM cycles whatever the number of active lanes,
// while integer, FP32 and special-function units are some 64 times wider, so the FP32 seeds
// of reciprocals are made from the bit patterns of the doubles.
// ---------------------------------------------------------------------------
// FP32 value of a double x in [2^-126, 2^128) by truncation of the mantissa (0 below).
__device__ __forceinline__ float approx_f32(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int fb = (int)(((unsigned)(hi - (896 << 20)) << 3) | (lo >> 29));
  return __int_as_float(hi < (897 << 20) ? 0 : fb);
}
// Double with the value 2^e2 * f of a positive normal float f (e2 = 0 or -1): exact.
__device__ __forceinline__ double widen_f32(float f, int e2 = 0) {
  const int fb = __float_as_int(f);
  return __hiloint2double((fb >> 3) + ((896 + e2) << 20), fb << 29);
}
// 2^e x for a positive normal double x (exact; e small).
__device__ __forceinline__ double scale2(double x, int e) {
  return __hiloint2double(__double2hiint(x) + (e << 20), __double2loint(x));
}
// x >= 2^e... comparisons of non-negative doubles on the high word (integer units).
__device__ __forceinline__ bool ge_hi(double x, int hi) { return __double2hiint(x) >= hi; }

// FP32 value of any finite double by truncation of the mantissa (relative error below
// 2^-23): magnitudes below 2^-126 give 0, above 2^128 are not expected.
__device__ __forceinline__ float to_f32(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int mag = hi & 0x7fffffff;
  const unsigned fb = ((unsigned)(mag - (896 << 20)) << 3) | (lo >> 29);
  return __int_as_float((int)((mag < (897 << 20) ? 0u : fb) | ((unsigned)hi & 0x80000000u)));
}
// Exact double of a float (subnormal floats give 0).
__device__ __forceinline__ double to_f64(float f) {
  const int fb = __float_as_int(f);
  const int mag = fb & 0x7fffffff;
  if (mag < 0x00800000) return 0.0;
  return __hiloint2double(((mag >> 3) + (896 << 20)) | (fb & (int)0x80000000), mag << 29);
}

// 1/sqrt(x) for x > 0 in FP32 range: FP32 hardware seed (relative error below 2^-22),
// one Newton-Raphson step (the error squares: below 1e-13 relative).  3 FP64 instructions.
__device__ __forceinline__ double rsqrt_nr(double x) {
  const float yf = rsqrtf(approx_f32(x));
  const double y = widen_f32(yf);
  const double hy = widen_f32(yf, -1);            // y / 2
  const double r = fma(-x * y, y, 1.0);           // 1 - x y^2
  return fma(hy, r, y);
}

// F_L(x) and exp(-x) for 0 <= x < kBoysXmax from the table of order L (13 FP64
// instructions: the offset from the grid point and two Horner chains).
__device__ __forceinline__ void boys_top(double x, const double* __restrict__ tabL, double& F, double& e) {
  const int g = __float2int_rn(approx_f32(x) * kBoysInvStepF);
  const double2* row = reinterpret_cast<const double2*>(tabL + g * kBoysRowLen);
  const double2 r0 = __ldg(row), r1 = __ldg(row + 1), r2 = __ldg(row + 2), r3 = __ldg(row + 3);
  const double2 r4 = __ldg(row + 4), r5 = __ldg(row + 5), r6 = __ldg(row + 6), r7 = __ldg(row + 7);
  const double d = x - r0.x;
  F = fma(fma(fma(fma(fma(fma(r3.y, d, r3.x), d, r2.y), d, r2.x), d, r1.y), d, r1.x), d, r0.y);
  e = fma(fma(fma(fma(fma(fma(r7.x, d, r6.y), d, r6.x), d, r5.y), d, r5.x), d, r4.y), d, r4.x);
}

// F_L(x) for x >= kBoysXmax: (2L-1)!!/2^{L+1} sqrt(pi) x^{-L-1/2} (the neglected terms are
// below exp(-60) relative); exp(-x) is taken as 0.
__device__ __forceinline__ double boys_asym(int L, double x) {
  const double y = rsqrt_nr(x);
  const double y2 = y * y;
  double v = y;
  double c = 0.886226925452758014;  // sqrt(pi)/2
#pragma unroll
  for (int m = 0; m < kMaxLt; ++m) {
    if (m < L) {
      v *= y2;
      c *= (m + 0.5);
    }
  }
  return c * v;
}

// Schedule variant of a class for the warp kernel (generated; see gen_eri_tables.py).
struct SchedVariant {
  int k;       // primitive quartets run at a time (streams), 0 = variant absent
  int rsz;     // doubles (or floats) of group scratch per stream
  int zero;    // index of the zero slot in a stream's region
  int n_iter;  // iterations of 32 entries
  int off;     // first entry in kSched (uint4 units)
  int group;   // doubles of the stream regions together, at least the post-contraction scratch
};

// Lattice images (periodic builds): the library holds the home cell's shells repeated in a
// box of cells (the image shells, cell-major, the home cell first); every pair of the pair
// list has one shell in the home cell (list-IJ anchored in the home cell, Sec. 3.1).
struct PeriodicInfo {
  const int* shell_cell;            // image shell -> cell index (0 = home cell)
  const int* shell_bf;              // image shell -> first function in the home-cell numbering
  const int* cell_xyz;              // cell index -> integer cell coordinates (3 each)
  const unsigned char* home_first;  // candidate pair -> 1 if its first shell is the home-cell one
  const int* rmap;                  // density block index of cell R (-1: absent), R in [-rb, rb]^3
  int rb;
  const double* P;                  // density blocks P^R, n_R x nbf x nbf
  int nbf;
  const double* pmax;               // max |P^R| per (R, home shell, home shell): n_R x nsh x nsh
  int nsh;                          // shells of the home cell
};

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
  const double* boys;         // kMaxLt + 1 tables of kBoysTableLen doubles
  double omega, omega2;
  SchedVariant sv;             // warp kernel: the schedule variant of this class
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
  double dist_tau;              // > 0: drop quartets with Q_IJ Q_KL exp(-kappa rho R^2) < dist_tau
  const double* dist;           // per sorted pair: most diffuse primitive-pair centre (3), spread,
                                // smallest exponent sum (5 doubles)
  const double* Qs;             // Schwarz factor of each sorted pair
  // batched launch (n_sys > 0): quartets of all systems' lists for this class, concatenated;
  // seg[s] = first index of system s (seg[n_sys] = total = q_count); batch[s] = that
  // system's record for this class (device memory)
  int n_sys;
  const long long* seg;
  const EriLaunch* batch;
  // periodic launch: quartets (bra | ket + shift) of the pair list for the cell G; reverse = 0:
  // the bra pair carries the row function of K^G, 1: the ket pair does (the launch then
  // evaluates (q | p - G L) for the quartet (p | q + G L) of a lower bra class)
  PeriodicInfo per;
  double shift[3];
  int gcell[3];
  int reverse;
  double* KG;                 // K^G, nbf x nbf
};


}  // namespace hfx
