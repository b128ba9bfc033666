// Table-driven engine for contracted shell quartets (ab|cd) with the erfc(omega r)/r
// kernel, fused with the exchange-matrix digest.  It runs in FP64; the recurrence and
// contraction steps are templated on the arithmetic type, and an FP32 primitive set-up
// (prim_core_f32) feeds them, so the mixed-precision kernel runs set-up, recurrences and
// contraction in FP32 for the quartets that qualify (HRR, spherical step and digest in FP64).
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
#include <type_traits>
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
__device__ __forceinline__ float2 fmar(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float4 fmar(float4 a, float4 b, float4 c) {
  const float2 lo = __ffma2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y), make_float2(c.x, c.y));
  const float2 hi = __ffma2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w), make_float2(c.z, c.w));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}
// index of the all-zero coefficient set of a packed layout (32 sets of one primitive quartet,
// 16 of two, 8 of four)
template <typename R>
__host__ __device__ constexpr int zero_set() {
  return std::is_same<R, float4>::value ? 8 : (std::is_same<R, float2>::value ? 16 : 32);
}
template <typename R>
__device__ __forceinline__ R sph_coef(int i);
template <>
__device__ __forceinline__ float sph_coef<float>(int i) { return kSphCoefF[i]; }
template <>
__device__ __forceinline__ double sph_coef<double>(int i) { return kSphCoef[i]; }

// Coefficients held in registers (one quartet per thread); selects avoid indexed
// register arrays.
template <typename R>
struct CoefRgT {
  R PA[3], WP[3], QC[3], WQ[3];
  R ca1, ca2, ca3, RP, ck1, ck2, ck3, RQ, cb1, cb2, cb3, cb4;
  __device__ __forceinline__ R pa(int i) const { return i == 0 ? PA[0] : (i == 1 ? PA[1] : PA[2]); }
  __device__ __forceinline__ R wp(int i) const { return i == 0 ? WP[0] : (i == 1 ? WP[1] : WP[2]); }
  __device__ __forceinline__ R qc(int i) const { return i == 0 ? QC[0] : (i == 1 ? QC[1] : QC[2]); }
  __device__ __forceinline__ R wq(int i) const { return i == 0 ? WQ[0] : (i == 1 ? WQ[1] : WQ[2]); }
  __device__ __forceinline__ R ca(int n) const { return n == 1 ? ca1 : (n == 2 ? ca2 : ca3); }
  __device__ __forceinline__ R ck(int n) const { return n == 1 ? ck1 : (n == 2 ? ck2 : ck3); }
  __device__ __forceinline__ R cb(int n) const { return n == 1 ? cb1 : (n == 2 ? cb2 : (n == 3 ? cb3 : cb4)); }
  __device__ __forceinline__ R rp() const { return RP; }
  __device__ __forceinline__ R rq() const { return RQ; }
};
using CoefRg = CoefRgT<double>;

// FP32 copy of a coefficient set (conversions on the integer units, see to_f32)
__device__ __forceinline__ CoefRgT<float> coef_f32(const CoefRg& c, int E, int F) {
  CoefRgT<float> f;
  if (E > 0) {
    for (int i = 0; i < 3; ++i) {
      f.PA[i] = to_f32(c.PA[i]);
      f.WP[i] = to_f32(c.WP[i]);
    }
    f.ca1 = to_f32(c.ca1); f.ca2 = to_f32(c.ca2); f.ca3 = to_f32(c.ca3); f.RP = to_f32(c.RP);
  }
  if (F > 0) {
    for (int i = 0; i < 3; ++i) {
      f.QC[i] = to_f32(c.QC[i]);
      f.WQ[i] = to_f32(c.WQ[i]);
    }
    f.ck1 = to_f32(c.ck1); f.ck2 = to_f32(c.ck2); f.ck3 = to_f32(c.ck3); f.RQ = to_f32(c.RQ);
    f.cb1 = to_f32(c.cb1); f.cb2 = to_f32(c.cb2); f.cb3 = to_f32(c.cb3); f.cb4 = to_f32(c.cb4);
  }
  return f;
}

// Scalars of one primitive quartet besides its Boys values.
struct PrimScalars {
  double RP, RQ, inv_s, PQ[3];
};

// Primitive-quartet set-up: the prefactor-scaled attenuated Boys values
//   G_m = C_ab C_cd / sqrt(p+q) * (F_m(T) - kappa^{m+1/2} F_m(kappa T)),  m = 0..Lt,
// kappa = omega^2 / (omega^2 + rho), T = rho |PQ|^2 (omega = 0: the Coulomb F_m(T)).  Both
// Boys functions are taken at the top order only; the lower orders come from one downward
// recursion on G itself: with A_m = pref F_m(T) and B_m = pref kappa^{m+1/2} F_m(kappa T),
// F_{m-1}(x) = (2x F_m(x) + e^{-x}) / (2m-1) gives
//   G_{m-1} = (2T G_m + pref e^{-T} - pref kappa^{m-1/2} e^{-kappa T}) / (2m-1).
// Returns false if the quartet is negligible (kappa T beyond the tables: G_m < e^{-60}).
__device__ __forceinline__ bool prim_core(const PrimPair& b, const PrimPair& k, int Lt, double omega, double omega2,
                                          const double* __restrict__ tabs, double* G, PrimScalars& ps) {
  const double p = b.p, q = k.p;
  const double s = p + q;
  const double y = rsqrt_nr(s);   // 1/sqrt(p+q)
  const double inv_s = y * y;
  ps.inv_s = inv_s;
  ps.RP = q * inv_s;              // rho / p
  ps.RQ = p * inv_s;              // rho / q
  const double rho = p * ps.RP;
  ps.PQ[0] = b.P[0] - k.P[0];
  ps.PQ[1] = b.P[1] - k.P[1];
  ps.PQ[2] = b.P[2] - k.P[2];
  const double T = rho * fma(ps.PQ[0], ps.PQ[0], fma(ps.PQ[1], ps.PQ[1], ps.PQ[2] * ps.PQ[2]));
  const double pref = (b.C * k.C) * y;
  const double* tabL = tabs + Lt * kBoysTableLen;
  double F1, e1 = 0.0;
  if (!ge_hi(T, kBoysXmaxHi))
    boys_top(T, tabL, F1, e1);
  else
    F1 = boys_asym(Lt, T);
  const double T2 = T + T;
  if (omega2 > 0.0) {
    const double sk = omega * rsqrt_nr(omega2 + rho);   // sqrt(kappa)
    const double kap = sk * sk;
    const double kT = kap * T;
    if (ge_hi(kT, kBoysXmaxHi)) return false;
    double F2, e2;
    boys_top(kT, tabL, F2, e2);
    // c[m] = pref kappa^{m-1/2}, m = 1..Lt+1
    double c[kMaxLt + 2];
    c[1] = pref * sk;
#pragma unroll
    for (int m = 1; m <= kMaxLt; ++m)
      if (m <= Lt) c[m + 1] = c[m] * kap;
    const double pe1 = pref * e1;
    double g = 0.0;
#pragma unroll
    for (int m = 0; m <= kMaxLt; ++m)
      if (m == Lt) g = fma(-c[m + 1], F2, pref * F1);
    G[Lt] = g;
#pragma unroll
    for (int m = kMaxLt; m >= 1; --m) {
      if (m <= Lt) {
        g = fma(T2, g, fma(-c[m], e2, pe1)) * (1.0 / (2 * m - 1));
        G[m - 1] = g;
      }
    }
  } else {
    const double pe1 = pref * e1;
    double g = pref * F1;
    G[Lt] = g;
#pragma unroll
    for (int m = kMaxLt; m >= 1; --m) {
      if (m <= Lt) {
        g = fma(T2, g, pe1) * (1.0 / (2 * m - 1));
        G[m - 1] = g;
      }
    }
  }
  return true;
}

// Set-up into registers (one quartet per thread).
__device__ __forceinline__ bool prim_setup(const PrimPair& b, const PrimPair& k, int E, int F, int Lt, double omega,
                                           double omega2, const double* __restrict__ tabs, CoefRg& c, double* Gm) {
  PrimScalars ps;
  if (!prim_core(b, k, Lt, omega, omega2, tabs, Gm, ps)) return false;
  if (E > 0) {
    c.PA[0] = b.PA[0]; c.PA[1] = b.PA[1]; c.PA[2] = b.PA[2];
    c.WP[0] = -ps.RP * ps.PQ[0]; c.WP[1] = -ps.RP * ps.PQ[1]; c.WP[2] = -ps.RP * ps.PQ[2];   // W - P
    c.ca1 = b.inv2p; c.ca2 = scale2(b.inv2p, 1); c.ca3 = b.inv2p3;
    c.RP = ps.RP;
  }
  if (F > 0) {
    c.QC[0] = k.PA[0]; c.QC[1] = k.PA[1]; c.QC[2] = k.PA[2];
    c.WQ[0] = ps.RQ * ps.PQ[0]; c.WQ[1] = ps.RQ * ps.PQ[1]; c.WQ[2] = ps.RQ * ps.PQ[2];      // W - Q
    c.ck1 = k.inv2p; c.ck2 = scale2(k.inv2p, 1); c.ck3 = k.inv2p3;
    c.RQ = ps.RQ;
    c.cb1 = scale2(ps.inv_s, -1); c.cb2 = ps.inv_s; c.cb3 = 1.5 * ps.inv_s; c.cb4 = scale2(ps.inv_s, 1);
  }
  return true;
}

// ---------------------------------------------------------------------------
// FP32 set-up (FP32 passes of the mixed-precision build).  With a = m + 1/2,
//   F_m(T) - kappa^a F_m(kappa T) = 1/2 T^{-a} (Gamma(a, kappa T) - Gamma(a, T)),
// because F_m(x) = 1/2 x^{-a} gamma(a, x) and gamma(a, x) = Gamma(a) - Gamma(a, x).  So with
// A_m = 1/2 T^{-a} Gamma(a, kappa T) and B_m = 1/2 T^{-a} Gamma(a, T), from Gamma(1/2, x) =
// sqrt(pi) erfc(sqrt x) and Gamma(a + 1, x) = a Gamma(a, x) + x^a e^{-x}:
//   A_0 = 1/2 sqrt(pi/T) erfc(sqrt(kappa T)),  A_{m+1} = ((m + 1/2) A_m + 1/2 kappa^{m+1/2} e^{-kappa T}) / T,
//   B_0 = 1/2 sqrt(pi/T) erfc(sqrt(T)),        B_{m+1} = ((m + 1/2) B_m + 1/2 e^{-T}) / T.
// Every term is positive, so this upward recursion keeps FP32's relative accuracy at any T; the
// one subtraction, G_m = pref (A_m - B_m), loses at most a factor 1 / (1 - B_m / A_m).  Where
// B_m > A_m / 64 for some m (T (1 - kappa) small: close or diffuse pairs) the primitive quartet
// takes the FP64 set-up instead.  P - Q is formed in FP64 (3 instructions), so that T keeps
// FP32's relative accuracy for centres far from the origin; nothing else runs on the FP64 pipe.
// ---------------------------------------------------------------------------
struct PrimScalarsF {
  float RP, RQ, inv_s, PQ[3];
};

enum { F32_SKIP = 0, F32_OK = 1, F32_FP64 = 2 };

__device__ __forceinline__ int prim_core_f32(const PrimPair& b, const PrimPair& k, int Lt, float omega_f, float* G,
                                             PrimScalarsF& ps) {
  const float p = b.pf, q = k.pf;
  const float y = rsqrtf(p + q);  // 1/sqrt(p+q)
  const float inv_s = y * y;
  ps.inv_s = inv_s;
  ps.RP = q * inv_s;
  ps.RQ = p * inv_s;
  const float rho = p * ps.RP;
  ps.PQ[0] = to_f32(b.P[0] - k.P[0]);
  ps.PQ[1] = to_f32(b.P[1] - k.P[1]);
  ps.PQ[2] = to_f32(b.P[2] - k.P[2]);
  const float T = rho * fmaf(ps.PQ[0], ps.PQ[0], fmaf(ps.PQ[1], ps.PQ[1], ps.PQ[2] * ps.PQ[2]));
  const float sk = omega_f * rsqrtf(fmaf(omega_f, omega_f, rho));  // sqrt(kappa)
  const float kap = sk * sk;
  const float kT = kap * T;
  if (kT >= 60.0f) return F32_SKIP;  // as the FP64 set-up: G_m < e^{-60}
  const float pref = to_f32(b.C) * to_f32(k.C) * y;
  const float yT = rsqrtf(T);
  const float invT = yT * yT;
  const float c0 = 0.886226925f * yT;  // sqrt(pi) / 2 / sqrt(T)
  float A = c0 * erfcf(sqrtf(kT));
  float B = c0 * erfcf(sqrtf(T));
  const float hk = 0.5f * expf(-kT), h1 = 0.5f * expf(-T);
  // accepted only with B_m <= A_m / 64 and A_m finite at every order (on this path A_m stays far
  // below 1: T (1 - kappa) is not small); T near 0 overflows the recursion and is declined
  bool ok = (B <= A * (1.0f / 64.0f)) && (A <= 1e30f);
  G[0] = pref * (A - B);
  float kp = sk;  // kappa^{m+1/2}
#pragma unroll
  for (int m = 0; m < kMaxLt; ++m) {
    if (m < Lt) {
      const float a = (float)m + 0.5f;
      A = fmaf(a, A, kp * hk) * invT;
      B = fmaf(a, B, h1) * invT;
      kp *= kap;
      ok = ok && (B <= A * (1.0f / 64.0f)) && (A <= 1e30f);
      G[m + 1] = pref * (A - B);
    }
  }
  return ok ? F32_OK : F32_FP64;
}

// Register coefficients from the FP32 set-up (one quartet per thread).
__device__ __forceinline__ int prim_setup_f32(const PrimPair& b, const PrimPair& k, int E, int F, int Lt,
                                              float omega_f, CoefRgT<float>& c, float* G) {
  PrimScalarsF ps;
  const int st = prim_core_f32(b, k, Lt, omega_f, G, ps);
  if (st != F32_OK) return st;
  if (E > 0) {
    c.PA[0] = b.PAf[0]; c.PA[1] = b.PAf[1]; c.PA[2] = b.PAf[2];
    c.WP[0] = -ps.RP * ps.PQ[0]; c.WP[1] = -ps.RP * ps.PQ[1]; c.WP[2] = -ps.RP * ps.PQ[2];
    c.ca1 = b.inv2pf; c.ca2 = 2.0f * b.inv2pf; c.ca3 = 3.0f * b.inv2pf;
    c.RP = ps.RP;
  }
  if (F > 0) {
    c.QC[0] = k.PAf[0]; c.QC[1] = k.PAf[1]; c.QC[2] = k.PAf[2];
    c.WQ[0] = ps.RQ * ps.PQ[0]; c.WQ[1] = ps.RQ * ps.PQ[1]; c.WQ[2] = ps.RQ * ps.PQ[2];
    c.ck1 = k.inv2pf; c.ck2 = 2.0f * k.inv2pf; c.ck3 = 3.0f * k.inv2pf;
    c.RQ = ps.RQ;
    c.cb1 = 0.5f * ps.inv_s; c.cb2 = ps.inv_s; c.cb3 = 1.5f * ps.inv_s; c.cb4 = 2.0f * ps.inv_s;
  }
  return F32_OK;
}

// A coefficient set (layout of write_set) from the FP32 set-up values.
template <int CS = 1>
__device__ __forceinline__ void write_set_f32(const PrimPair& b, const PrimPair& k, int E, int F, int Lt,
                                              const float* G, const PrimScalarsF& ps, float* cf) {
#pragma unroll
  for (int m = 0; m <= kMaxLt; ++m)
    if (m <= Lt) cf[(HFX_CF_G + m) * CS] = G[m];
  cf[(HFX_CF_ONE) * CS] = 1.0f;
  cf[(HFX_CF_ZERO) * CS] = 0.0f;
  cf[(HFX_CF_CA) * CS] = 0.0f;
  cf[(HFX_CF_CK) * CS] = 0.0f;
  cf[(HFX_CF_CB) * CS] = 0.0f;
  if (E > 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      cf[(HFX_CF_PA + i) * CS] = b.PAf[i];
      cf[(HFX_CF_WP + i) * CS] = -ps.RP * ps.PQ[i];
    }
    cf[(HFX_CF_CA + 1) * CS] = b.inv2pf;
    cf[(HFX_CF_CA + 2) * CS] = 2.0f * b.inv2pf;
    cf[(HFX_CF_CA + 3) * CS] = 3.0f * b.inv2pf;
    cf[HFX_CF_RP * CS] = -ps.RP;
  }
  if (F > 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      cf[(HFX_CF_QC + i) * CS] = k.PAf[i];
      cf[(HFX_CF_WQ + i) * CS] = ps.RQ * ps.PQ[i];
    }
    cf[(HFX_CF_CK + 1) * CS] = k.inv2pf;
    cf[(HFX_CF_CK + 2) * CS] = 2.0f * k.inv2pf;
    cf[(HFX_CF_CK + 3) * CS] = 3.0f * k.inv2pf;
    cf[HFX_CF_RQ * CS] = -ps.RQ;
    cf[(HFX_CF_CB + 1) * CS] = 0.5f * ps.inv_s;
    cf[(HFX_CF_CB + 2) * CS] = ps.inv_s;
    cf[(HFX_CF_CB + 3) * CS] = 1.5f * ps.inv_s;
    cf[(HFX_CF_CB + 4) * CS] = 2.0f * ps.inv_s;
  }
}

// A coefficient set in group scratch (warp kernel) from the set-up values, in the precision
// R of the recurrences: every set-up step runs in FP64; an FP32 set is the rounded FP64 one.
template <typename R>
__device__ __forceinline__ R to_R(double x) {
  if constexpr (sizeof(R) == 4)
    return to_f32(x);
  else
    return x;
}

// CS = 1: a set of R values; CS = 2 (R = float): one half of a set of float pairs (the
// packed FP32 engine runs two primitive quartets per slot).
template <typename R, int CS = 1>
__device__ __forceinline__ void write_set(const PrimPair& b, const PrimPair& k, int E, int F, int Lt,
                                          const double* G, const PrimScalars& ps, R* cf) {
#pragma unroll
  for (int m = 0; m <= kMaxLt; ++m)
    if (m <= Lt) cf[(HFX_CF_G + m) * CS] = to_R<R>(G[m]);
  cf[(HFX_CF_ONE) * CS] = to_R<R>(1);
  cf[(HFX_CF_ZERO) * CS] = to_R<R>(0);
  cf[(HFX_CF_CA) * CS] = to_R<R>(0);
  cf[(HFX_CF_CK) * CS] = to_R<R>(0);
  cf[(HFX_CF_CB) * CS] = to_R<R>(0);
  if (E > 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      cf[(HFX_CF_PA + i) * CS] = to_R<R>(b.PA[i]);
      cf[(HFX_CF_WP + i) * CS] = to_R<R>(-ps.RP * ps.PQ[i]);
    }
    cf[(HFX_CF_CA + 1) * CS] = to_R<R>(b.inv2p);
    cf[(HFX_CF_CA + 2) * CS] = to_R<R>(scale2(b.inv2p, 1));
    cf[(HFX_CF_CA + 3) * CS] = to_R<R>(b.inv2p3);
    cf[HFX_CF_RP * CS] = to_R<R>(-ps.RP);  // stored negated: the VRR term is V3 - rho/p V4
  }
  if (F > 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      cf[(HFX_CF_QC + i) * CS] = to_R<R>(k.PA[i]);
      cf[(HFX_CF_WQ + i) * CS] = to_R<R>(ps.RQ * ps.PQ[i]);
    }
    cf[(HFX_CF_CK + 1) * CS] = to_R<R>(k.inv2p);
    cf[(HFX_CF_CK + 2) * CS] = to_R<R>(scale2(k.inv2p, 1));
    cf[(HFX_CF_CK + 3) * CS] = to_R<R>(k.inv2p3);
    cf[HFX_CF_RQ * CS] = to_R<R>(-ps.RQ);
    cf[(HFX_CF_CB + 1) * CS] = to_R<R>(scale2(ps.inv_s, -1));
    cf[(HFX_CF_CB + 2) * CS] = to_R<R>(ps.inv_s);
    cf[(HFX_CF_CB + 3) * CS] = to_R<R>(1.5 * ps.inv_s);
    cf[(HFX_CF_CB + 4) * CS] = to_R<R>(scale2(ps.inv_s, 1));
  }
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

// One entry of a warp schedule (gen_eri_tables.py): this lane's op in the current iteration,
// on the region X of its stream, with the coefficient set of the primitive quartet that
// stream runs (sets j + u of the chunk; set 32, all zeros, once the chunk is used up).
// The shape bits (11, 12) are the same on every valid lane of an iteration, so the optional
// terms are warp-uniform branches; ops of a simpler shape in such an iteration read the
// zero coefficient n = 0 and the zero slot.
template <typename R>
__device__ __forceinline__ void sched_op(uint4 e, R* S, int rsz, int zero, const R* CF, int j, int nv) {
  const uint32_t w = e.w;
  if (!(w & (1u << 10))) return;
  const int u = (w >> 13) & 7;
  const int p = j + u;
  // past the last set: the all-zero set
  const R* cf = CF + (p < nv ? p : zero_set<R>()) * HFX_NCOEF;
  R* X = S + u * rsz;
  const int base = (w & (1u << 7)) ? HFX_CF_KET_BASE : 0;
  const int dir = w & 3;
  const bool add = (w >> 9) & 1;
  const int i1 = add ? HFX_CF_ONE : base + HFX_CF_PA + dir;
  const int i2 = add ? HFX_CF_ZERO : base + HFX_CF_WP + dir;
  const int dst = e.x & 0xFFFF;
  const int s0 = ((w >> 8) & 1) ? dst : zero;
  R v = fmar(cf[i1], X[e.x >> 16], X[s0]);
  v = fmar(cf[i2], X[e.y & 0xFFFF], v);
  if (w & (1u << 11))
    v = fmar(cf[base + HFX_CF_CA + ((w >> 2) & 3)], fmar(cf[base + HFX_CF_RP], X[e.z & 0xFFFF], X[e.y >> 16]), v);
  if (w & (1u << 12)) v = fmar(cf[HFX_CF_CB + ((w >> 4) & 7)], X[e.z >> 16], v);
  X[dst] = v;
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
