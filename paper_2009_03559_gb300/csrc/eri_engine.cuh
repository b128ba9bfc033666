// Table-driven engine for contracted shell quartets (ab|cd) with the erfc(omega r)/r
// kernel, fused with the exchange-matrix digest.  It runs in FP64; the recurrence and
// contraction steps are templated on the arithmetic type, so the mixed-precision kernel
// runs them in FP32 for the quartets that qualify (the Boys step stays FP64).
//
// One "group" of G lanes (G = 1 or G = 32) evaluates one contracted quartet:
//   1. for every surviving primitive quartet: the Boys step (G_m = F_m(T) -
//      kappa^{m+1/2} F_m(kappa T), times the prefactor), then the Obara-Saika vertical
//      recurrence level by level (ops of a level are independent and spread over the
//      lanes), then the contraction into the accumulator block (e0|f0);
//   2. the post-contraction stages: Head-Gordon-Pople horizontal recurrence on the bra,
//      Cartesian -> spherical on a and b, HRR on the ket, spherical on c and d;
//   3. the digest into the half exchange matrix A (K = A + A^T afterwards):
//      A_ac += sum_bd v P_bd, A_ad += sum_bc v P_bc, A_bc += sum_ad v P_ad,
//      A_bd += sum_ac v P_ac, with v = deg (ab|cd), deg = 1/2^[a=b] 1/2^[c=d] 1/2^[ab=cd].
// The per-class op lists come from gen_eri_tables.py (eri_tables.inc).
#pragma once
#include "hfx_internal.cuh"

namespace hfx {

#define HFX_TABLE_QUAL __device__ __align__(16) const
#include "eri_tables.inc"
#undef HFX_TABLE_QUAL

__device__ __constant__ double kSphCoef[6] = {0.0, 1.0, -0.28867513459481287, 0.57735026918962573,
                                              0.5, -0.5};
__device__ __constant__ float kSphCoefF[6] = {0.0f, 1.0f, -0.28867513459481287f, 0.57735026918962573f,
                                              0.5f, -0.5f};

// fused multiply-add in the precision of the arguments (an unqualified fma() on floats
// would promote to FP64, which runs on the FP64 pipe together with the conversions)
__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename R>
__device__ __forceinline__ R sph_coef(int i);
template <>
__device__ __forceinline__ float sph_coef<float>(int i) { return kSphCoefF[i]; }
template <>
__device__ __forceinline__ double sph_coef<double>(int i) { return kSphCoef[i]; }

// coefficient set of one primitive quartet (shared-memory layout for G > 1)
enum {
  CF_PA = 0, CF_WP = 3, CF_QC = 6, CF_WQ = 9,
  CF_CA = 12,   // [n] = n/(2p), n = 0..3
  CF_RP = 16,   // rho/p
  CF_CK = 17,   // [n] = n/(2q), n = 0..3
  CF_RQ = 21,   // rho/q
  CF_CB = 22,   // [n] = n/(2(p+q)), n = 0..4
  CF_G = 27,    // prefactor * G_m, m = 0..Lt
  CF_SKIP = 36, // nonzero: primitive quartet negligible (kappa T beyond the table)
  NCOEF = 37
};

// Coefficients held in registers (G = 1); selects avoid indexed register arrays.
struct CoefRg {
  double PA[3], WP[3], QC[3], WQ[3];
  double ca1, ca2, ca3, RP, ck1, ck2, ck3, RQ, cb1, cb2, cb3, cb4;
  __device__ __forceinline__ double pa(int i) const { return i == 0 ? PA[0] : (i == 1 ? PA[1] : PA[2]); }
  __device__ __forceinline__ double wp(int i) const { return i == 0 ? WP[0] : (i == 1 ? WP[1] : WP[2]); }
  __device__ __forceinline__ double qc(int i) const { return i == 0 ? QC[0] : (i == 1 ? QC[1] : QC[2]); }
  __device__ __forceinline__ double wq(int i) const { return i == 0 ? WQ[0] : (i == 1 ? WQ[1] : WQ[2]); }
  __device__ __forceinline__ double ca(int n) const { return n == 1 ? ca1 : (n == 2 ? ca2 : ca3); }
  __device__ __forceinline__ double ck(int n) const { return n == 1 ? ck1 : (n == 2 ? ck2 : ck3); }
  __device__ __forceinline__ double cb(int n) const {
    return n == 1 ? cb1 : (n == 2 ? cb2 : (n == 3 ? cb3 : cb4));
  }
  __device__ __forceinline__ double rp() const { return RP; }
  __device__ __forceinline__ double rq() const { return RQ; }
};

// Coefficients read from shared memory (G > 1), stored in the precision R of the
// recurrences (FP64, or FP32 for quartets selected for FP32).
template <typename R>
struct CoefSm {
  const R* c;
  __device__ __forceinline__ R pa(int i) const { return c[CF_PA + i]; }
  __device__ __forceinline__ R wp(int i) const { return c[CF_WP + i]; }
  __device__ __forceinline__ R qc(int i) const { return c[CF_QC + i]; }
  __device__ __forceinline__ R wq(int i) const { return c[CF_WQ + i]; }
  __device__ __forceinline__ R ca(int n) const { return c[CF_CA + n]; }
  __device__ __forceinline__ R ck(int n) const { return c[CF_CK + n]; }
  __device__ __forceinline__ R cb(int n) const { return c[CF_CB + n]; }
  __device__ __forceinline__ R rp() const { return c[CF_RP]; }
  __device__ __forceinline__ R rq() const { return c[CF_RQ]; }
};

// Primitive-quartet set-up.  Fills the register coefficient set and returns the
// prefactor-scaled attenuated Boys values in Gm[0..Lt]; returns false if the
// primitive quartet is negligible (kappa T >= table end: G_m <= exp(-kappa T)).
__device__ __forceinline__ bool prim_setup(const PrimPair& b, const PrimPair& k, int E, int F, int Lt,
                                           double omega2, const double* __restrict__ tab, CoefRg& c,
                                           double* Gm) {
  const double p = b.p, q = k.p;
  const double s = p + q;
  const double inv_s = rcp_nr(s);
  const double RP = q * inv_s;   // rho / p
  const double RQ = p * inv_s;   // rho / q
  const double rho = p * RP;
  const double PQ0 = b.P[0] - k.P[0], PQ1 = b.P[1] - k.P[1], PQ2 = b.P[2] - k.P[2];
  const double r2 = fma(PQ0, PQ0, fma(PQ1, PQ1, PQ2 * PQ2));
  const double T = rho * r2;
  double F1[kMaxLt + 1], F2[kMaxLt + 1];
  const double pref = b.C * k.C * rsqrt_nr(s);
  if (omega2 > 0.0) {
    const double kap = omega2 * rcp_nr(omega2 + rho);
    const double kT = kap * T;
    if (kT >= kBoysXmax) return false;
    boys_eval(Lt, T, tab, F1);
    boys_eval(Lt, kT, tab, F2);
    double a = pref * (kap * rsqrt_nr(kap));  // pref * kappa^{1/2}
#pragma unroll
    for (int m = 0; m <= kMaxLt; ++m) {
      if (m <= Lt) {
        Gm[m] = fma(-a, F2[m], pref * F1[m]);
        a *= kap;
      }
    }
  } else {
    boys_eval(Lt, T, tab, F1);
#pragma unroll
    for (int m = 0; m <= kMaxLt; ++m)
      if (m <= Lt) Gm[m] = pref * F1[m];
  }
  if (E > 0) {
    c.PA[0] = b.PA[0]; c.PA[1] = b.PA[1]; c.PA[2] = b.PA[2];
    c.WP[0] = -RP * PQ0; c.WP[1] = -RP * PQ1; c.WP[2] = -RP * PQ2;   // W - P
    c.ca1 = b.inv2p; c.ca2 = b.inv2p + b.inv2p; c.ca3 = 3.0 * b.inv2p;
    c.RP = RP;
  }
  if (F > 0) {
    c.QC[0] = k.PA[0]; c.QC[1] = k.PA[1]; c.QC[2] = k.PA[2];
    c.WQ[0] = RQ * PQ0; c.WQ[1] = RQ * PQ1; c.WQ[2] = RQ * PQ2;      // W - Q
    c.ck1 = k.inv2p; c.ck2 = k.inv2p + k.inv2p; c.ck3 = 3.0 * k.inv2p;
    c.RQ = RQ;
    const double h = 0.5 * inv_s;
    c.cb1 = h; c.cb2 = h + h; c.cb3 = 3.0 * h; c.cb4 = 4.0 * h;
  }
  return true;
}

// Set-up for the FP32 recurrences: the Boys step (rho, kappa, T, G_m, the prefactor) in FP64
// exactly as in prim_setup, the VRR coefficients in FP32 from the float copies of the pair
// data; only the G_m values are converted.  Writes the coefficient set cf (floats).
__device__ __forceinline__ void prim_setup_f32(const PrimPair& b, const PrimPair& k, int E, int F, int Lt,
                                               double omega2, const double* __restrict__ tab, float* cf) {
  const double p = b.p, q = k.p;
  const double s = p + q;
  const double inv_s = rcp_nr(s);
  const double rho = p * (q * inv_s);
  const double PQ0 = b.P[0] - k.P[0], PQ1 = b.P[1] - k.P[1], PQ2 = b.P[2] - k.P[2];
  const double T = rho * fma(PQ0, PQ0, fma(PQ1, PQ1, PQ2 * PQ2));
  double F1[kMaxLt + 1], F2[kMaxLt + 1];
  const double pref = b.C * k.C * rsqrt_nr(s);
  if (omega2 > 0.0) {
    const double kap = omega2 * rcp_nr(omega2 + rho);
    const double kT = kap * T;
    if (kT >= kBoysXmax) {
      cf[CF_SKIP] = 1.f;
      return;
    }
    boys_eval(Lt, T, tab, F1);
    boys_eval(Lt, kT, tab, F2);
    double a = pref * (kap * rsqrt_nr(kap));
    for (int m = 0; m <= Lt; ++m) {
      cf[CF_G + m] = (float)fma(-a, F2[m], pref * F1[m]);
      a *= kap;
    }
  } else {
    boys_eval(Lt, T, tab, F1);
    for (int m = 0; m <= Lt; ++m) cf[CF_G + m] = (float)(pref * F1[m]);
  }
  cf[CF_SKIP] = 0.f;
  const float pf = b.pf, qf = k.pf;
  const float inv_sf = __frcp_rn(pf + qf);
  const float RP = qf * inv_sf, RQ = pf * inv_sf;
  const float d0 = (float)PQ0, d1 = (float)PQ1, d2 = (float)PQ2;
  if (E > 0) {
    cf[CF_PA + 0] = b.PAf[0]; cf[CF_PA + 1] = b.PAf[1]; cf[CF_PA + 2] = b.PAf[2];
    cf[CF_WP + 0] = -RP * d0; cf[CF_WP + 1] = -RP * d1; cf[CF_WP + 2] = -RP * d2;
    cf[CF_CA + 1] = b.inv2pf; cf[CF_CA + 2] = 2.f * b.inv2pf; cf[CF_CA + 3] = 3.f * b.inv2pf;
    cf[CF_RP] = RP;
  }
  if (F > 0) {
    cf[CF_QC + 0] = k.PAf[0]; cf[CF_QC + 1] = k.PAf[1]; cf[CF_QC + 2] = k.PAf[2];
    cf[CF_WQ + 0] = RQ * d0; cf[CF_WQ + 1] = RQ * d1; cf[CF_WQ + 2] = RQ * d2;
    cf[CF_CK + 1] = k.inv2pf; cf[CF_CK + 2] = 2.f * k.inv2pf; cf[CF_CK + 3] = 3.f * k.inv2pf;
    cf[CF_RQ] = RQ;
    const float h = 0.5f * inv_sf;
    cf[CF_CB + 1] = h; cf[CF_CB + 2] = 2.f * h; cf[CF_CB + 3] = 3.f * h; cf[CF_CB + 4] = 4.f * h;
  }
}

template <typename R>
__device__ __forceinline__ void store_coef(const CoefRg& c, const double* Gm, int Lt, bool ok, R* cf) {
  cf[CF_SKIP] = ok ? R(0) : R(1);
  if (!ok) return;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cf[CF_PA + i] = c.PA[i];
    cf[CF_WP + i] = c.WP[i];
    cf[CF_QC + i] = c.QC[i];
    cf[CF_WQ + i] = c.WQ[i];
  }
  cf[CF_CA + 1] = c.ca1; cf[CF_CA + 2] = c.ca2; cf[CF_CA + 3] = c.ca3; cf[CF_RP] = c.RP;
  cf[CF_CK + 1] = c.ck1; cf[CF_CK + 2] = c.ck2; cf[CF_CK + 3] = c.ck3; cf[CF_RQ] = c.RQ;
  cf[CF_CB + 1] = c.cb1; cf[CF_CB + 2] = c.cb2; cf[CF_CB + 3] = c.cb3; cf[CF_CB + 4] = c.cb4;
#pragma unroll
  for (int m = 0; m <= kMaxLt; ++m)
    if (m <= Lt) cf[CF_G + m] = Gm[m];
}

__device__ __forceinline__ uint4 ld_op(const uint32_t* base, int idx) {
  return __ldg(reinterpret_cast<const uint4*>(base) + idx);
}

// VRR ops.  bra:  v = PA_i V[s1] + WP_i V[s2] (+ n/(2p) (V[s3] - rho/p V[s4]))
//           ket:  v = QC_i V[s1] + WQ_i V[s2] (+ n/(2q) (V[s3] - rho/q V[s4]))
//                                             (+ e_i/(2(p+q)) V[s5])
// The result is stored to V[dst]; ops flagged "acc" (targets no op reads) instead add it
// to the accumulator S[dst], starting their FMA chain from the accumulator value.
// FOLD = false compiles the plain form (no accumulator branch) for classes without folding.
template <bool FOLD, typename R, class Coef>
__device__ __forceinline__ void vrr_bra(uint4 op, R* V, R* S, int st, const Coef& c) {
  const int dst = op.x & 0xFFFF, s1 = op.x >> 16, s2 = op.y & 0xFFFF, s3 = op.y >> 16, s4 = op.z & 0xFFFF;
  const int i = op.w & 3, nA = (op.w >> 2) & 7;
  const bool acc = FOLD && ((op.w >> 8) & 1);
  R v = acc ? fmar(c.pa(i), V[s1 * st], S[dst * st]) : c.pa(i) * V[s1 * st];
  v = fmar(c.wp(i), V[s2 * st], v);
  if (nA) v = fmar(c.ca(nA), fmar(-c.rp(), V[s4 * st], V[s3 * st]), v);
  if (acc)
    S[dst * st] = v;
  else
    V[dst * st] = v;
}

template <bool FOLD, typename R, class Coef>
__device__ __forceinline__ void vrr_ket(uint4 op, R* V, R* S, int st, const Coef& c) {
  const int dst = op.x & 0xFFFF, s1 = op.x >> 16, s2 = op.y & 0xFFFF, s3 = op.y >> 16;
  const int s4 = op.z & 0xFFFF, s5 = op.z >> 16;
  const int i = op.w & 3, nA = (op.w >> 2) & 7, nB = (op.w >> 5) & 7;
  const bool acc = FOLD && ((op.w >> 8) & 1);
  R v = acc ? fmar(c.qc(i), V[s1 * st], S[dst * st]) : c.qc(i) * V[s1 * st];
  v = fmar(c.wq(i), V[s2 * st], v);
  if (nA) v = fmar(c.ck(nA), fmar(-c.rq(), V[s4 * st], V[s3 * st]), v);
  if (nB) v = fmar(c.cb(nB), V[s5 * st], v);
  if (acc)
    S[dst * st] = v;
  else
    V[dst * st] = v;
}

// Post-contraction op on the group scratch S.
template <typename R>
__device__ __forceinline__ void post_op(uint4 op, int type, R* S, int st, const R* AB, const R* CD) {
  const int dst = op.x & 0xFFFF, s1 = op.x >> 16, s2 = op.y & 0xFFFF, s3 = op.y >> 16;
  R v;
  if (type == 2) {
    const int c0 = op.z & 15, c1 = (op.z >> 4) & 15, c2 = (op.z >> 8) & 15;
    v = sph_coef<R>(c0) * S[s1 * st];
    if (c1) v = fmar(sph_coef<R>(c1), S[s2 * st], v);
    if (c2) v = fmar(sph_coef<R>(c2), S[s3 * st], v);
  } else {
    const int i = (op.z >> 12) & 3;
    const R d = (type == 0) ? AB[i] : CD[i];
    v = fmar(d, S[s2 * st], S[s1 * st]);
  }
  S[dst * st] = v;
}

// Digest of the final spherical block v (stride st) into the half matrix A.
// Outputs o in [o0, nout) step ostep (lanes of the group).
template <typename R>
__device__ __forceinline__ void digest(const EriClassInfo& ci, const R* v, int st, int A, int B,
                                       int C, int D, double deg, const double* __restrict__ P,
                                       double* K, int ld, int o0, int ostep) {
  const int na = ci.dims[0], nb = ci.dims[1], nc = ci.dims[2], nd = ci.dims[3];
  const int nAC = na * nc, nAD = na * nd, nBC = nb * nc, nBD = nb * nd;
  const int nout = nAC + nAD + nBC + nBD;
  for (int o = o0; o < nout; o += ostep) {
    double acc = 0.0;
    int row, col;
    if (o < nAC) {
      const int a = o / nc, c = o - a * nc;
      for (int b = 0; b < nb; ++b)
        for (int d = 0; d < nd; ++d)
          acc = fma((double)v[(((a * nb + b) * nc + c) * nd + d) * st], __ldg(P + (size_t)(B + b) * ld + D + d), acc);
      row = A + a; col = C + c;
    } else if (o < nAC + nAD) {
      const int t = o - nAC, a = t / nd, d = t - a * nd;
      for (int b = 0; b < nb; ++b)
        for (int c = 0; c < nc; ++c)
          acc = fma((double)v[(((a * nb + b) * nc + c) * nd + d) * st], __ldg(P + (size_t)(B + b) * ld + C + c), acc);
      row = A + a; col = D + d;
    } else if (o < nAC + nAD + nBC) {
      const int t = o - nAC - nAD, b = t / nc, c = t - b * nc;
      for (int a = 0; a < na; ++a)
        for (int d = 0; d < nd; ++d)
          acc = fma((double)v[(((a * nb + b) * nc + c) * nd + d) * st], __ldg(P + (size_t)(A + a) * ld + D + d), acc);
      row = B + b; col = C + c;
    } else {
      const int t = o - nAC - nAD - nBC, b = t / nd, d = t - b * nd;
      for (int a = 0; a < na; ++a)
        for (int c = 0; c < nc; ++c)
          acc = fma((double)v[(((a * nb + b) * nc + c) * nd + d) * st], __ldg(P + (size_t)(A + a) * ld + C + c), acc);
      row = B + b; col = D + d;
    }
    atomicAdd(K + (size_t)row * ld + col, deg * acc);
  }
}

// Diagonal (Schwarz) epilogue: max_{a,b} |(ab|ab)|.
__device__ __forceinline__ double diag_max(const EriClassInfo& ci, const double* v, int st) {
  const int na = ci.dims[0], nb = ci.dims[1];
  double mx = 0.0;
  for (int a = 0; a < na; ++a)
    for (int b = 0; b < nb; ++b) mx = fmax(mx, fabs(v[(((a * nb + b) * na + a) * nb + b) * st]));
  return mx;
}

// Locate the row of quartet q (global index) in [rlo, rhi): qoff[r] <= q < qoff[r+1].
__device__ __forceinline__ int find_row(const long long* qoff, int rlo, int rhi, long long q) {
  int lo = rlo, hi = rhi - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(qoff + mid) <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// The quartet range [q0, q1) handled by group gid of ngroups.
__device__ __forceinline__ void group_range(const EriLaunch& L, long long gid, long long ngroups,
                                            long long& q0, long long& q1) {
  if (L.schedule == 1) {
    // parallel-pair split (paper Algorithm 2): an even share of the bra pairs, whatever
    // the number of quartets they carry
    const long long nr = L.row_end - L.row_begin;
    const int r0 = L.row_begin + (int)(nr * gid / ngroups);
    const int r1 = L.row_begin + (int)(nr * (gid + 1) / ngroups);
    q0 = __ldg(L.qoff + r0);
    q1 = __ldg(L.qoff + r1);
  } else {
    // parallel-quartet split (paper Algorithm 3 without the replicated screening): an
    // even share of the screened quartet list
    q0 = L.q_begin + L.q_count * gid / ngroups;
    q1 = L.q_begin + L.q_count * (gid + 1) / ngroups;
  }
}

}  // namespace hfx
