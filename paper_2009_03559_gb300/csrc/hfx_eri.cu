// ERI kernels: one class launch evaluates every screened quartet of one class pair
// (bra pair bin >= ket pair bin) -- of one system, or of all systems of a batch -- and
// digests it into the half exchange matrix, or, in diagonal mode, evaluates (p|p) for
// candidate pairs and stores the Schwarz factor.
#include <algorithm>
#include <cstdio>
#include <type_traits>
#include "eri_engine.cuh"
#include "hfx_eri.h"

namespace hfx {

const EriClassInfo* class_info_host() { return kClassInfo; }

// ---------------------------------------------------------------------------
// Contracted quartet, G = 1: the thread owns the quartet.  Group scratch slots are
// interleaved over the block's threads (slot k of thread t at smem[k*st + t]).
// ---------------------------------------------------------------------------
// ci is the launch's class record (kernel parameter space); L supplies the system's data.
// R = float runs the recurrences and the contraction on FP32 slots, slot k in the first half
// of the thread's own FP64 slot k (so no other lane's slots are ever touched); the
// accumulated block is then widened in place into the FP64 slots Sd, where the horizontal
// recurrences and the spherical step run.  R = double: the FP64 slots themselves.
template <typename R, bool PER = false>
__device__ __forceinline__ int contract_g1(const EriClassInfo& ci, const EriLaunch& L, int bra, int ket, double* Sd,
                                           int st) {
  R* S = reinterpret_cast<R*>(Sd);
  const int sts = st * (int)(sizeof(double) / sizeof(R));  // slot stride in units of R
  const PairArrays pa = L.pa;
  const double omega = L.omega, omega2 = L.omega2;
  const double* boys = L.boys;
  R* V = S + ci.work_base * sts;
  const int nb = __ldg(pa.prim_n + bra), nk = __ldg(pa.prim_n + ket);
  const PrimPair* pb = pa.prim + __ldg(pa.prim_off + bra);
  const PrimPair* pk = pa.prim + __ldg(pa.prim_off + ket);
  for (int a = 0; a < ci.n_acc; ++a) S[a * sts] = R(0);
  int any = 0;
  // one flat loop over the primitive quartets: lanes whose quartets have the same count
  // (the queue groups them so) run the same number of iterations
  const int npq = nb * nk;
  if constexpr (sizeof(R) == 4) {
    static_assert(!PER, "the periodic build runs in FP64");
    // vertical recurrences and contraction on FP32 slots for one primitive quartet
    auto vrr = [&](const CoefRgT<float>& cf, const float* Gf) {
      for (int m = 0; m <= ci.Lt; ++m) V[m * sts] = Gf[m];
      for (int lv = 0; lv < ci.n_bra_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = 0; o < n; ++o) vrr_bra<true>(ld_op(kVrrOps, off + o), V, S, sts, cf);
      }
      for (int lv = ci.n_bra_lv; lv < ci.n_bra_lv + ci.n_ket_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = 0; o < n; ++o) vrr_ket<true>(ld_op(kVrrOps, off + o), V, S, sts, cf);
      }
      for (int a = 0; a < ci.n_accl; ++a) {
        const uint32_t w = __ldg(kAccSrc + ci.acc_off + a);
        S[(w & 0xFFFF) * sts] += V[(w >> 16) * sts];
      }
    };
    // the FP64 set-up of one primitive quartet, rounded to FP32 (false: negligible)
    auto setup64 = [&](int t, CoefRgT<float>& cf, float* Gf) {
      const int ib = t / nk, ik = t - ib * nk;
      CoefRg c;
      double Gm[kMaxLt + 1];
      if (!prim_setup(pb[ib], pk[ik], ci.E, ci.F, ci.Lt, omega, omega2, boys, c, Gm)) return false;
      cf = coef_f32(c, ci.E, ci.F);
      for (int m = 0; m <= ci.Lt; ++m) Gf[m] = to_f32(Gm[m]);
      return true;
    };
    // FP32 set-up first; the primitive quartets it declines (bit t - c0 of pend) take the FP64
    // set-up at the end of their chunk of 96, so that a lane's FP64 set-ups run together with
    // the other lanes' instead of once per iteration in which any lane needs one
    const float omega_f = to_f32(omega);
    for (int c0 = 0; c0 < npq; c0 += 96) {
      const int c1 = min(npq, c0 + 96);
      unsigned pend0 = 0, pend1 = 0, pend2 = 0;
      for (int t = c0; t < c1; ++t) {
        const int ib = t / nk, ik = t - ib * nk;
        CoefRgT<float> cf;
        float Gf[kMaxLt + 1];
        const int stt = prim_setup_f32(pb[ib], pk[ik], ci.E, ci.F, ci.Lt, omega_f, cf, Gf);
        if (stt == F32_SKIP) continue;
        if (stt == F32_FP64) {
          const int u = t - c0;
          if (u < 32) pend0 |= 1u << u;
          else if (u < 64) pend1 |= 1u << (u - 32);
          else pend2 |= 1u << (u - 64);
          continue;
        }
        ++any;
        vrr(cf, Gf);
      }
      while (pend0 | pend1 | pend2) {
        int t;
        if (pend0) {
          t = c0 + __ffs(pend0) - 1;
          pend0 &= pend0 - 1;
        } else if (pend1) {
          t = c0 + 32 + __ffs(pend1) - 1;
          pend1 &= pend1 - 1;
        } else {
          t = c0 + 64 + __ffs(pend2) - 1;
          pend2 &= pend2 - 1;
        }
        CoefRgT<float> cf;
        float Gf[kMaxLt + 1];
        if (!setup64(t, cf, Gf)) continue;
        ++any;
        vrr(cf, Gf);
      }
    }
  } else {
    auto vrr = [&](const CoefRg& c, const double* Gm) {
      for (int m = 0; m <= ci.Lt; ++m) V[m * sts] = Gm[m];
      for (int lv = 0; lv < ci.n_bra_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = 0; o < n; ++o) vrr_bra<true>(ld_op(kVrrOps, off + o), V, S, sts, c);
      }
      for (int lv = ci.n_bra_lv; lv < ci.n_bra_lv + ci.n_ket_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = 0; o < n; ++o) vrr_ket<true>(ld_op(kVrrOps, off + o), V, S, sts, c);
      }
      for (int a = 0; a < ci.n_accl; ++a) {
        const uint32_t w = __ldg(kAccSrc + ci.acc_off + a);
        S[(w & 0xFFFF) * sts] += V[(w >> 16) * sts];
      }
    };
    auto ket_of = [&](int ik) {
      PrimPair k = pk[ik];
      if constexpr (PER) {  // the ket pair's image in cell G (its centre moves, P - C does not)
        k.P[0] += L.shift[0];
        k.P[1] += L.shift[1];
        k.P[2] += L.shift[2];
      }
      return k;
    };
    for (int t = 0; t < npq; ++t) {
      const int ib = t / nk, ik = t - ib * nk;
      CoefRg c;
      double Gm[kMaxLt + 1];
      if (!prim_setup(pb[ib], ket_of(ik), ci.E, ci.F, ci.Lt, omega, omega2, boys, c, Gm)) continue;
      ++any;
      vrr(c, Gm);
    }
  }
  if (!any) return 0;
  if constexpr (sizeof(R) == 4) {
    for (int a = 0; a < ci.n_acc; ++a) Sd[a * st] = to_f64(S[a * sts]);  // in place: read, then write
  }
  double AB[3], CD[3];
  for (int i = 0; i < 3; ++i) {
    AB[i] = __ldg(pa.AB + 3 * bra + i);
    CD[i] = __ldg(pa.AB + 3 * ket + i);
  }
  for (int s = 0; s < ci.n_post; ++s) {
    const int off = ci.post_off[s], n = ci.post_n[s], type = ci.post_type[s];
    for (int o = 0; o < n; ++o) post_op(ld_op(kPostOps, off + o), type, Sd, st, AB, CD);
  }
  return any;
}

// ---------------------------------------------------------------------------
// Contracted quartet, one warp: lanes set up 32 primitive quartets at a time (coefficient
// sets in group scratch, compacted so that negligible ones take no place), then the warp
// runs the class's schedule over k of them at a time (k streams, each with its own region
// of accumulators and VRR slots), and finally sums the streams' accumulators.
// ---------------------------------------------------------------------------
// HRR and Cartesian -> spherical stages on the group scratch S (lanes share each stage)
template <typename R>
__device__ __forceinline__ void post_stages(const EriClassInfo& ci, const PairArrays& pa, int bra, int ket, R* S,
                                            int lane) {
  R AB[3], CD[3];
  for (int i = 0; i < 3; ++i) {
    AB[i] = R(__ldg(pa.AB + 3 * bra + i));
    CD[i] = R(__ldg(pa.AB + 3 * ket + i));
  }
  for (int s = 0; s < ci.n_post; ++s) {
    const int off = ci.post_off[s], n = ci.post_n[s], type = ci.post_type[s];
    for (int o = lane; o < n; o += 32) post_op<R>(ld_op(kPostOps, off + o), type, S, 1, AB, CD);
    __syncwarp();
  }
}

// primitive quartets per slot of the packed FP32 pass (2: float2, 4: float4)
#ifndef HFX_FP32_PACK
#define HFX_FP32_PACK 4
#endif

// Group scratch of one warp (in doubles): k stream regions, 33 coefficient sets (the last
// one all zeros), one spare double.
__host__ __device__ __forceinline__ int g32_stride(const SchedVariant& sv, int prec = 0) {
  // the packed FP32 pass holds two primitive quartets per set (16 sets and the zero set), or
  // four (stream regions of twice the size, 8 sets and the zero set, in doubles twice 9 x NCOEF)
  if (prec != 2) return sv.group + 33 * HFX_NCOEF + 1;
  // float4 slots need 16-byte alignment: an even stride keeps every warp's region aligned
  return HFX_FP32_PACK == 4 ? 2 * sv.group + 9 * HFX_NCOEF * 2 + 2 : sv.group + 17 * HFX_NCOEF + 1;
}

template <bool PER = false>
__device__ __forceinline__ int contract_g32(const EriClassInfo& ci, const SchedVariant& sv, const EriLaunch& L,
                                            int bra, int ket, double* S, double* CF, int lane) {
  const PairArrays pa = L.pa;
  const double omega = L.omega, omega2 = L.omega2;
  const double* boys = L.boys;
  const int nb = __ldg(pa.prim_n + bra), nk = __ldg(pa.prim_n + ket);
  const PrimPair* pb = pa.prim + __ldg(pa.prim_off + bra);
  const PrimPair* pk = pa.prim + __ldg(pa.prim_off + ket);
  const int k = sv.k, rsz = sv.rsz, nacc = ci.n_acc, nbase = ci.Lt + 1;
  for (int i = lane; i < k * nacc; i += 32) {
    const int u = i / nacc;
    S[u * rsz + (i - u * nacc)] = 0.0;
  }
  if (lane < k) S[lane * rsz + sv.zero] = 0.0;
  // coefficient set 32: all zeros, for streams past the chunk's last primitive quartet
  for (int i = lane; i < HFX_NCOEF; i += 32) CF[32 * HFX_NCOEF + i] = 0.0;
  const uint4* sched = reinterpret_cast<const uint4*>(kSched) + sv.off;
  const int npq = nb * nk;
  int any = 0;
  for (int base = 0; base < npq; base += 32) {
    const int t = base + lane;
    double G[kMaxLt + 1];
    PrimScalars ps;
    int ib = 0, ik = 0;
    bool ok = false;
    if (t < npq) {
      ib = t / nk;
      ik = t - ib * nk;
      PrimPair k = pk[ik];
      if constexpr (PER) {  // the ket pair's image in cell G
        k.P[0] += L.shift[0];
        k.P[1] += L.shift[1];
        k.P[2] += L.shift[2];
      }
      ok = prim_core(pb[ib], k, ci.Lt, omega, omega2, boys, G, ps);
    }
    const unsigned okm = __ballot_sync(0xffffffffu, ok);
    if (ok)
      write_set<double>(pb[ib], pk[ik], ci.E, ci.F, ci.Lt, G, ps, CF + __popc(okm & ((1u << lane) - 1u)) * HFX_NCOEF);
    const int nv = __popc(okm);
    any += nv;
    __syncwarp();
    for (int j = 0; j < nv; j += k) {
      for (int i = lane; i < k * nbase; i += 32) {
        const int u = i / nbase, m = i - u * nbase;
        S[u * rsz + nacc + m] = (j + u < nv) ? CF[(j + u) * HFX_NCOEF + HFX_CF_G + m] : 0.0;
      }
      __syncwarp();
      uint4 e = __ldg(sched + lane);
      for (int it = 1; it <= sv.n_iter; ++it) {
        // the next entry is fetched before this one runs (the last fetch reads one
        // iteration past the variant's table: the tables end with a padding iteration)
        const uint4 en = __ldg(sched + it * 32 + lane);
        sched_op<double>(e, S, rsz, sv.zero, CF, j, nv);
        __syncwarp();
        e = en;
      }
    }
  }
  if (!any) return 0;
  if (k > 1) {
    for (int a = lane; a < nacc; a += 32) {
      double sum = S[a];
      for (int u = 1; u < k; ++u) sum += S[u * rsz + a];
      S[a] = sum;
    }
    __syncwarp();
  }
  post_stages<double>(ci, pa, bra, ket, S, lane);
  return any;
}

// Position of set bit number n (0-based, from the least significant) of m; -1 if m has fewer.
__device__ __forceinline__ int nth_bit(unsigned m, int n) {
  for (int i = 0; i < n; ++i) m &= m - 1u;
  return __ffs(m) - 1;
}

// Packed FP32 (mixed precision): every slot and coefficient holds W primitive quartets'
// values (a float2 for W = 2, a float4 for W = 4), so one op of the schedule advances W
// primitive quartets with one W-wide load per operand and W/2 FFMA2.  The stream regions hold
// W floats per slot; the coefficient area holds 32/W sets and the zero set.  The contracted
// block is widened to FP64 (the W components summed in FP64) for the horizontal recurrences,
// the spherical step and the digest, which run on the FP64 view of the same memory.
template <int W>
struct PackV;
template <>
struct PackV<2> {
  using T = float2;
};
template <>
struct PackV<4> {
  using T = float4;
};

template <int W>
__device__ __forceinline__ int contract_g32_xw(const EriClassInfo& ci, const SchedVariant& sv, const EriLaunch& L,
                                               int bra, int ket, double* Sd, double* CFd, int lane) {
  using V = typename PackV<W>::T;
  constexpr int kZeroSet = 32 / W;
  V* S = reinterpret_cast<V*>(Sd);
  V* CF = reinterpret_cast<V*>(CFd);
  V zv;
  float* zf = reinterpret_cast<float*>(&zv);
#pragma unroll
  for (int c = 0; c < W; ++c) zf[c] = 0.f;
  const PairArrays pa = L.pa;
  const double omega = L.omega, omega2 = L.omega2;
  const double* boys = L.boys;
  const int nb = __ldg(pa.prim_n + bra), nk = __ldg(pa.prim_n + ket);
  const PrimPair* pb = pa.prim + __ldg(pa.prim_off + bra);
  const PrimPair* pk = pa.prim + __ldg(pa.prim_off + ket);
  const int k = sv.k, rsz = sv.rsz, nacc = ci.n_acc, nbase = ci.Lt + 1;
  for (int i = lane; i < k * nacc; i += 32) {
    const int u = i / nacc;
    S[u * rsz + (i - u * nacc)] = zv;
  }
  if (lane < k) S[lane * rsz + sv.zero] = zv;
  for (int i = lane; i < HFX_NCOEF; i += 32) CF[kZeroSet * HFX_NCOEF + i] = zv;
  const uint4* sched = reinterpret_cast<const uint4*>(kSched) + sv.off;
  const int npq = nb * nk;
  int any = 0;
  // component pos of the packed sets (pos < 32)
  auto slot_of = [&](int pos) { return reinterpret_cast<float*>(CF + (pos / W) * HFX_NCOEF) + (pos % W); };
  // the sets of the lanes in okm (at most 32) are in CF: run the schedule over them
  auto run_sets = [&](unsigned okm) {
    const int nv = __popc(okm);
    any += nv;
    const int r = nv % W;
    if (r)  // the unused components of the last packed set: all-zero primitive quartets
      for (int i = lane; i < HFX_NCOEF * (W - r); i += 32) {
        const int c = i / (W - r);
        reinterpret_cast<float*>(CF + (nv / W) * HFX_NCOEF + c)[r + (i - c * (W - r))] = 0.f;
      }
    __syncwarp();
    const int np = (nv + W - 1) / W;
    for (int j = 0; j < np; j += k) {
      for (int i = lane; i < k * nbase; i += 32) {
        const int u = i / nbase, m = i - u * nbase;
        S[u * rsz + nacc + m] = (j + u < np) ? CF[(j + u) * HFX_NCOEF + HFX_CF_G + m] : zv;
      }
      __syncwarp();
      uint4 e = __ldg(sched + lane);
      for (int it = 1; it <= sv.n_iter; ++it) {
        const uint4 en = __ldg(sched + it * 32 + lane);
        sched_op<V>(e, S, rsz, sv.zero, CF, j, np);
        __syncwarp();
        e = en;
      }
    }
  };
  // the primitive quartets c0 + (bits of m0, m1 << 32, m2 << 64) set up in FP64, 32 at a time
  auto fp64_sets = [&](unsigned m0, unsigned m1, unsigned m2, int c0) {
    const int n0 = __popc(m0), n1 = __popc(m1), nf = n0 + n1 + __popc(m2);
    for (int base = 0; base < nf; base += 32) {
      const int idx = base + lane;
      bool ok = false;
      int ib = 0, ik = 0;
      double G[kMaxLt + 1];
      PrimScalars ps;
      if (idx < nf) {
        const int u = idx < n0 ? nth_bit(m0, idx) : (idx < n0 + n1 ? 32 + nth_bit(m1, idx - n0) : 64 + nth_bit(m2, idx - n0 - n1));
        const int t = c0 + u;
        if (u >= 0 && t < npq) {
          ib = t / nk;
          ik = t - ib * nk;
          ok = prim_core(pb[ib], pk[ik], ci.Lt, omega, omega2, boys, G, ps);
        }
      }
      const unsigned okm = __ballot_sync(0xffffffffu, ok);
      const int pos = __popc(okm & ((1u << lane) - 1u));
      if (ok) write_set<float, W>(pb[ib], pk[ik], ci.E, ci.F, ci.Lt, G, ps, slot_of(pos));
      run_sets(okm);
    }
  };
  // FP32 set-up first (prim_core_f32); the primitive quartets it declines are set up in FP64 at
  // the end of their chunk of 96 (three rounds), 32 at a time, so that the FP64 set-up runs
  // once per 32 of them rather than in every round in which one lane needs it
  const float omega_f = to_f32(omega);
  for (int c0 = 0; c0 < npq; c0 += 96) {
    unsigned fm[3] = {0u, 0u, 0u};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int base = c0 + 32 * r;
      if (base >= npq) break;
      const int t = base + lane;
      float G[kMaxLt + 1];
      PrimScalarsF ps;
      int ib = 0, ik = 0, stt = F32_SKIP;
      if (t < npq) {
        ib = t / nk;
        ik = t - ib * nk;
        stt = prim_core_f32(pb[ib], pk[ik], ci.Lt, omega_f, G, ps);
      }
      fm[r] = __ballot_sync(0xffffffffu, stt == F32_FP64);
      const bool ok = stt == F32_OK;
      const unsigned okm = __ballot_sync(0xffffffffu, ok);
      const int pos = __popc(okm & ((1u << lane) - 1u));
      if (ok) write_set_f32<W>(pb[ib], pk[ik], ci.E, ci.F, ci.Lt, G, ps, slot_of(pos));
      run_sets(okm);
    }
    if (fm[0] | fm[1] | fm[2]) fp64_sets(fm[0], fm[1], fm[2], c0);
  }
  if (!any) return 0;
  // the streams' sums, widened to FP64 in place: accumulator a's double overlaps the packed
  // slot a / (W / 2), which the same or an earlier 32-wide slice reads, so each slice reads all
  // its slots before any lane writes (the other streams' regions lie above the block)
  for (int a0 = 0; a0 < nacc; a0 += 32) {
    const int a = a0 + lane;
    double w = 0.0;
    if (a < nacc) {
      V sum = S[a];
      float* sf = reinterpret_cast<float*>(&sum);
      for (int u = 1; u < k; ++u) {
        const V v = S[u * rsz + a];
        const float* vf = reinterpret_cast<const float*>(&v);
#pragma unroll
        for (int c = 0; c < W; ++c) sf[c] += vf[c];
      }
      w = to_f64(sf[0]);
#pragma unroll
      for (int c = 1; c < W; ++c) w += to_f64(sf[c]);
    }
    __syncwarp();
    if (a < nacc) Sd[a] = w;
  }
  __syncwarp();
  post_stages<double>(ci, pa, bra, ket, Sd, lane);
  return any;
}

// Register caps (blocks of 64 threads per SM).  Thread-per-quartet FP64: 6 (at most 170
// registers), measured fastest; warp kernel: 8 (128 registers: the schedule keeps few values
// live); the batched thread kernel carries the batch bookkeeping too and the FP32 passes
// both recurrence precisions' set-up, so they get 4-6 to stay free of spills.
#ifndef HFX_G1_MINB
#define HFX_G1_MINB 6
#endif
#ifndef HFX_G32_MINB
#define HFX_G32_MINB 8
#endif
#ifndef HFX_G1B_MINB
#define HFX_G1B_MINB 6
#endif
#ifndef HFX_G1F_MINB
#define HFX_G1F_MINB 4
#endif
#ifndef HFX_G32B_MINB
#define HFX_G32B_MINB 8
#endif
#ifndef HFX_G32F_MINB  // packed FP32 pass: 10 or 12 blocks spill (64-atom mixed build 3354 / 3309 ms vs 3021)
#define HFX_G32F_MINB 8
#endif

// Precision passes of a class launch: 0 every quartet in FP64; 1 (mixed precision, first
// pass) the quartets that must stay FP64; 2 (second pass) those whose recurrences run in FP32.
// PREC_PERIODIC: the FP64 periodic instance (quartets of the lattice sums, see per_quartet).
enum { PREC_FP64 = 0, PREC_MIXED64 = 1, PREC_MIXED32 = 2, PREC_PERIODIC = 3 };

// The digest reads P_bd, P_bc, P_ad, P_ac.  max of their max|P| (or 1 without the table):
// 0 means the quartet contributes exactly nothing; the mixed-precision and the
// density-weighted screening tests use it too.
__device__ __forceinline__ double pmax4(const EriLaunch& L, int sa, int sb, int sc, int sd) {
  if (!L.pmax) return 1.0;
  const double* pm = L.pmax;
  const size_t ns = L.ns;
  return fmax(fmax(__ldg(pm + sb * ns + sd), __ldg(pm + sb * ns + sc)),
              fmax(__ldg(pm + sa * ns + sd), __ldg(pm + sa * ns + sc)));
}

// Distance-aware test: Q_IJ Q_KL exp(-kappa rho R^2) >= dist_tau (see hfx_options.dist_tau).
__device__ __forceinline__ bool dist_keeps(const EriLaunch& Ls, int bra_s, int ket_s) {
  if (!(Ls.dist_tau > 0.0)) return true;
  const double* a = Ls.dist + 5 * (size_t)bra_s;
  const double* b = Ls.dist + 5 * (size_t)ket_s;
  const double dx = __ldg(a) - __ldg(b), dy = __ldg(a + 1) - __ldg(b + 1), dz = __ldg(a + 2) - __ldg(b + 2);
  double r = sqrt(dx * dx + dy * dy + dz * dz) - __ldg(a + 3) - __ldg(b + 3);
  if (r < 0.0) r = 0.0;
  const double p = __ldg(a + 4), q = __ldg(b + 4);
  const double rho = p * q / (p + q);
  const double lam = Ls.omega2 * rho / (Ls.omega2 + rho);
  return __ldg(Ls.Qs + bra_s) * __ldg(Ls.Qs + ket_s) * exp(-lam * r * r) >= Ls.dist_tau;
}

// Mixed precision: FP32 recurrences for the quartet when the class allows it and its
// Schwarz bound times the largest density element it touches (or the largest of all of P)
// is below fp32_tau.
__device__ __forceinline__ bool fp32_eligible(const EriLaunch& Ls, int bra_s, int ket_s, double pm) {
  if (!Ls.fp32_ok) return false;
  const double pf = Ls.pglob ? __ldg(Ls.pglob) : pm;
  return __ldg(Ls.Qs + bra_s) * __ldg(Ls.Qs + ket_s) * pf < Ls.fp32_tau;
}

// whether pass PREC takes the quartet
template <int PREC>
__device__ __forceinline__ bool pass_takes(const EriLaunch& Ls, int bra_s, int ket_s, double pm) {
  if constexpr (PREC == PREC_FP64) return true;
  const bool f32 = fp32_eligible(Ls, bra_s, ket_s, pm);
  return PREC == PREC_MIXED32 ? f32 : !f32;
}

__device__ __forceinline__ void record_busy(const EriLaunch& L, unsigned long long t0) {
  if (L.busy && threadIdx.x == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    atomicAdd(L.busy + smid, globaltimer_ns() - t0);
  }
}

// ---------------------------------------------------------------------------
// Periodic quartets (Eq. vx with lattice images): the launch for cell G evaluates
// (X | Y + shift) for bra pair X and ket pair Y of the home-anchored pair list and adds
//   K^G_{ab} += sum_{c,d} (a c | b d) P^{R}_{cd},   R = cell(d) - cell(c),
// where a is the home-cell shell of the pair holding the row function (X for a forward
// launch, Y for a reverse one), c its partner, b the home-cell shell of the other pair
// (in cell G) and d its partner.  Every ordered pair of pairs is one quartet (no
// permutational symmetry is used across cells), so the degeneracy factor is 1.
// ---------------------------------------------------------------------------
struct PerQuartet {
  int pa, pb, pc, pd;        // positions of shells a, b, c, d in the quartet block (x1 x2 y1 y2)
  int bfa, bfb, bfc, bfd;    // their first functions (home-cell numbering)
  const double* PR;          // density block P^R
};

__device__ __forceinline__ bool per_quartet(const EriLaunch& L, int bra, int ket, PerQuartet& q) {
  const PeriodicInfo& pi = L.per;
  const int sax = __ldg(L.pa.sa + bra), sbx = __ldg(L.pa.sb + bra);
  const int say = __ldg(L.pa.sa + ket), sby = __ldg(L.pa.sb + ket);
  const bool hx = __ldg(pi.home_first + bra), hy = __ldg(pi.home_first + ket);
  const int hxs = hx ? sax : sbx, oxs = hx ? sbx : sax;
  const int hys = hy ? say : sby, oys = hy ? sby : say;
  const int* cx = pi.cell_xyz + 3 * __ldg(pi.shell_cell + oxs);
  const int* cy = pi.cell_xyz + 3 * __ldg(pi.shell_cell + oys);
  const int w = 2 * pi.rb + 1;
  int idx = 0;
  for (int i = 0; i < 3; ++i) {
    const int d = __ldg(cy + i) - __ldg(cx + i);
    const int R = L.gcell[i] + (L.reverse ? -d : d);
    if (R < -pi.rb || R > pi.rb) return false;
    idx = idx * w + (R + pi.rb);
  }
  const int blk = __ldg(pi.rmap + idx);
  if (blk < 0) return false;
  // an exactly zero density block P^R_{cd} makes the quartet's contribution exactly zero
  {
    const int c = L.reverse ? oys : oxs, d = L.reverse ? oxs : oys;
    if (__ldg(pi.pmax + ((size_t)blk * pi.nsh + c % pi.nsh) * pi.nsh + d % pi.nsh) == 0.0) return false;
  }
  q.PR = pi.P + (size_t)blk * pi.nbf * pi.nbf;
  const int phx = hx ? 0 : 1, pox = 1 - phx, phy = hy ? 2 : 3, poy = 5 - phy;
  if (!L.reverse) {
    q.pa = phx; q.pc = pox; q.pb = phy; q.pd = poy;
    q.bfa = __ldg(pi.shell_bf + hxs); q.bfc = __ldg(pi.shell_bf + oxs);
    q.bfb = __ldg(pi.shell_bf + hys); q.bfd = __ldg(pi.shell_bf + oys);
  } else {
    q.pa = phy; q.pc = poy; q.pb = phx; q.pd = pox;
    q.bfa = __ldg(pi.shell_bf + hys); q.bfc = __ldg(pi.shell_bf + oys);
    q.bfb = __ldg(pi.shell_bf + hxs); q.bfd = __ldg(pi.shell_bf + oxs);
  }
  return true;
}

// K^G_{ab} += sum_{cd} v P^R_{cd} for the final block v (stride st); outputs o0, o0 + ostep, ...
__device__ __forceinline__ void digest_per(const EriClassInfo& ci, const double* v, int st, const PerQuartet& q,
                                           double* KG, int nbf, int o0, int ostep) {
  int str[4];
  str[3] = 1;
  str[2] = ci.dims[3];
  str[1] = ci.dims[2] * str[2];
  str[0] = ci.dims[1] * str[1];
  const int na = ci.dims[q.pa], nb = ci.dims[q.pb], nc = ci.dims[q.pc], nd = ci.dims[q.pd];
  const int sa = str[q.pa], sb = str[q.pb], sc = str[q.pc], sd = str[q.pd];
  for (int o = o0; o < na * nb; o += ostep) {
    const int ia = o / nb, ib = o - ia * nb;
    double acc = 0.0;
    for (int ic = 0; ic < nc; ++ic)
      for (int id = 0; id < nd; ++id)
        acc = fma(v[(ia * sa + ib * sb + ic * sc + id * sd) * st], __ldg(q.PR + (size_t)(q.bfc + ic) * nbf + q.bfd + id),
                  acc);
    atomicAdd(KG + (size_t)(q.bfa + ia) * nbf + q.bfb + ib, acc);
  }
}

// Per-thread tallies of one kernel, added to the launch's counters once at the end.
struct Tally {
  unsigned long long prim = 0, quart = 0, skip = 0, q32 = 0, p32 = 0;
};

// One quartet evaluated and digested by one lane (one quartet per thread), recurrences in
// precision R; Sd: the thread's FP64 slots.
template <typename R, bool PER = false>
__device__ __forceinline__ void g1_quartet(const EriClassInfo& ci, const EriLaunch& Ls, int bra_s, int ket_s,
                                           double* Sd, int st, Tally& t) {
  const int bra = __ldg(Ls.sorted + bra_s), ket = __ldg(Ls.sorted + ket_s);
  if constexpr (PER) {
    PerQuartet pq;
    if (!per_quartet(Ls, bra, ket, pq)) return;
    const int npq = __ldg(Ls.pa.prim_n + bra) * __ldg(Ls.pa.prim_n + ket);
    const int ne = contract_g1<double, true>(ci, Ls, bra, ket, Sd, st);
    t.prim += ne;
    t.skip += npq - ne;
    if (!ne) return;
    ++t.quart;
    digest_per(ci, Sd + ci.out_base * st, st, pq, Ls.KG, Ls.per.nbf, 0, 1);
    return;
  }
  const int sa = __ldg(Ls.pa.sa + bra), sb = __ldg(Ls.pa.sb + bra);
  const int sc = __ldg(Ls.pa.sa + ket), sd = __ldg(Ls.pa.sb + ket);
  const int npq = __ldg(Ls.pa.prim_n + bra) * __ldg(Ls.pa.prim_n + ket);
  const int ne = contract_g1<R>(ci, Ls, bra, ket, Sd, st);
  t.prim += ne;
  t.skip += npq - ne;
  if (!ne) return;
  ++t.quart;
  if (sizeof(R) == 4) {
    ++t.q32;
    t.p32 += ne;
  }
  double deg = 1.0;
  if (sa == sb) deg *= 0.5;
  if (sc == sd) deg *= 0.5;
  if (bra_s == ket_s) deg *= 0.5;
  digest(ci, Sd + ci.out_base * st, st, __ldg(Ls.sh.bf_off + sa), __ldg(Ls.sh.bf_off + sb), __ldg(Ls.sh.bf_off + sc),
         __ldg(Ls.sh.bf_off + sd), deg, Ls.P, Ls.K, Ls.ld, 0, 1);
}

// Per-warp queue of the quartets that pass the density tests (64 entries: system, bra
// position, ket position, primitive quartets).  Lanes evaluate quartets 32 at a time, the
// 32 with the most primitive quartets first, so that few lanes idle while the others
// finish their primitive loops (the FP64 pipe charges a warp instruction in full whatever
// the number of active lanes).
struct G1Queue {
  int4* q;
  int n;
};

// Descending bitonic sort of 64 keys, two per lane (element i = lane + 32 h).
__device__ __forceinline__ void sort64_desc(int& k0, int& k1, int lane) {
#pragma unroll
  for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      int o0, o1;
      if (stride == 32) {
        o0 = k1;
        o1 = k0;
      } else {
        o0 = __shfl_xor_sync(0xffffffffu, k0, stride);
        o1 = __shfl_xor_sync(0xffffffffu, k1, stride);
      }
      const int i0 = lane, i1 = lane + 32;
      const int j0 = i0 ^ stride, j1 = i1 ^ stride;
      const bool d0 = ((min(i0, j0) & size) == 0), d1 = ((min(i1, j1) & size) == 0);
      const bool m0 = (i0 < j0) == d0, m1 = (i1 < j1) == d1;
      k0 = m0 ? max(k0, o0) : min(k0, o0);
      k1 = m1 ? max(k1, o1) : min(k1, o1);
    }
  }
}

template <bool BATCH, typename R, bool PER = false>
__device__ __forceinline__ void g1_drain(const EriLaunch& L, const EriClassInfo& ci, G1Queue& Q, int lane,
                                         double* Sd, int st, Tally& t, bool all) {
  while (Q.n >= 32 || (all && Q.n > 0)) {
    int4 e;
    int take;
    if (Q.n >= 32) {
      // the 32 entries with the most primitive quartets; the rest move to the front
      int k0 = lane < Q.n ? ((Q.q[lane].w << 6) | lane) : -1;
      int k1 = lane + 32 < Q.n ? ((Q.q[lane + 32].w << 6) | (lane + 32)) : -1;
      sort64_desc(k0, k1, lane);
      e = Q.q[k0 & 63];
      int4 rest = make_int4(0, 0, 0, 0);
      if (k1 >= 0) rest = Q.q[k1 & 63];
      __syncwarp();
      if (k1 >= 0) Q.q[lane] = rest;
      take = 32;
    } else {
      e = Q.q[lane];
      take = Q.n;
    }
    __syncwarp();
    Q.n -= take;
    if (lane < take) g1_quartet<R, PER>(ci, BATCH ? L.batch[e.x] : L, e.y, e.z, Sd, st, t);
  }
}

// Quartets [q0, q1) of the launch record Ls (system sys), one quartet per thread: the warp
// tests 32 consecutive quartets at a time and queues the survivors.
template <bool BATCH, int PREC, typename R, bool PER = false>
__device__ __forceinline__ void g1_range(const EriLaunch& L, const EriClassInfo& ci, const EriLaunch& Ls, int sys,
                                         long long q0, long long q1, double* Sd, int st, int lane, G1Queue& Q,
                                         Tally& t) {
  const long long* qoff = Ls.qoff;
  const int row_begin = Ls.row_begin, bra0 = Ls.bra_bin_start, ket0 = Ls.ket_bin_start;
  const bool skip = Ls.skip_zero;
  const double dens = Ls.dens_tau;
  int r = -1;
  for (long long base = q0; base < q1; base += 32) {
    const long long q = base + lane;
    bool keep = false;
    int bra_s = 0, ket_s = 0, npq = 0;
    if (q < q1) {
      if (r < 0) r = find_row(qoff, row_begin, Ls.row_end, q);
      while (__ldg(qoff + r + 1) <= q) ++r;
      bra_s = bra0 + (r - row_begin);
      ket_s = ket0 + (int)(q - __ldg(qoff + r));
      const int bra = __ldg(Ls.sorted + bra_s), ket = __ldg(Ls.sorted + ket_s);
      if constexpr (PER) {
        PerQuartet pq;
        keep = per_quartet(Ls, bra, ket, pq);  // a density block exists for its cell offset
      } else {
        const double pm = pmax4(Ls, __ldg(Ls.pa.sa + bra), __ldg(Ls.pa.sb + bra), __ldg(Ls.pa.sa + ket),
                                __ldg(Ls.pa.sb + ket));
        keep = !(skip && pm == 0.0) && !(dens > 0.0 && __ldg(Ls.Qs + bra_s) * __ldg(Ls.Qs + ket_s) * pm < dens) &&
               dist_keeps(Ls, bra_s, ket_s) && pass_takes<PREC>(Ls, bra_s, ket_s, pm);
      }
      npq = __ldg(Ls.pa.prim_n + bra) * __ldg(Ls.pa.prim_n + ket);
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) Q.q[Q.n + __popc(m & ((1u << lane) - 1u))] = make_int4(sys, bra_s, ket_s, npq);
    Q.n += __popc(m);
    __syncwarp();
    g1_drain<BATCH, R, PER>(L, ci, Q, lane, Sd, st, t, false);
  }
}

// Quartets [q0, q1) of the launch record Ls, one warp: the warp takes them one by one.
// ci and sv: the launch's class record and schedule variant.
template <int PREC>
__device__ __forceinline__ void g32_range(const EriClassInfo& ci, const SchedVariant& sv, const EriLaunch& Ls,
                                          long long q0, long long q1, double* S, double* CF, int lane, Tally& t) {
  if (q0 >= q1) return;
  int r = find_row(Ls.qoff, Ls.row_begin, Ls.row_end, q0);
  for (long long q = q0; q < q1; ++q) {
    while (__ldg(Ls.qoff + r + 1) <= q) ++r;
    const int bra_s = Ls.bra_bin_start + (r - Ls.row_begin);
    const int ket_s = Ls.ket_bin_start + (int)(q - __ldg(Ls.qoff + r));
    const int bra = __ldg(Ls.sorted + bra_s), ket = __ldg(Ls.sorted + ket_s);
    const int sa = __ldg(Ls.pa.sa + bra), sb = __ldg(Ls.pa.sb + bra);
    const int sc = __ldg(Ls.pa.sa + ket), sd = __ldg(Ls.pa.sb + ket);
    const double pm = pmax4(Ls, sa, sb, sc, sd);
    if (Ls.skip_zero && pm == 0.0) continue;
    // density-weighted screening (off when dens_tau = 0)
    if (Ls.dens_tau > 0.0 && __ldg(Ls.Qs + bra_s) * __ldg(Ls.Qs + ket_s) * pm < Ls.dens_tau) continue;
    // distance-aware screening (off when dist_tau = 0)
    if (!dist_keeps(Ls, bra_s, ket_s)) continue;
    // mixed precision: this pass's share of the quartets (warp-uniform decision)
    if (!pass_takes<PREC>(Ls, bra_s, ket_s, pm)) continue;
    const int npq = __ldg(Ls.pa.prim_n + bra) * __ldg(Ls.pa.prim_n + ket);
    const bool f32 = PREC == PREC_MIXED32;
    int ne;
    if (f32)
      ne = contract_g32_xw<HFX_FP32_PACK>(ci, sv, Ls, bra, ket, S, S + (HFX_FP32_PACK / 2) * sv.group, lane);
    else
      ne = contract_g32<false>(ci, sv, Ls, bra, ket, S, CF, lane);
    t.prim += ne;
    t.skip += npq - ne;
    if (!ne) continue;
    ++t.quart;
    if (f32) {
      ++t.q32;
      t.p32 += ne;
    }
    double deg = 1.0;
    if (sa == sb) deg *= 0.5;
    if (sc == sd) deg *= 0.5;
    if (bra_s == ket_s) deg *= 0.5;
    const int A = __ldg(Ls.sh.bf_off + sa), B = __ldg(Ls.sh.bf_off + sb);
    const int C = __ldg(Ls.sh.bf_off + sc), D = __ldg(Ls.sh.bf_off + sd);
    // an FP32 quartet leaves its final block in FP64 too (see contract_g32)
    digest(ci, S + ci.out_base, 1, A, B, C, D, deg, Ls.P, Ls.K, Ls.ld, lane, 32);
    __syncwarp();
  }
}

// Periodic quartets [q0, q1) of the launch (FP64), one warp per quartet.
__device__ __forceinline__ void g32_range_per(const EriClassInfo& ci, const SchedVariant& sv, const EriLaunch& Ls,
                                              long long q0, long long q1, double* S, double* CF, int lane, Tally& t) {
  if (q0 >= q1) return;
  int r = find_row(Ls.qoff, Ls.row_begin, Ls.row_end, q0);
  for (long long q = q0; q < q1; ++q) {
    while (__ldg(Ls.qoff + r + 1) <= q) ++r;
    const int bra_s = Ls.bra_bin_start + (r - Ls.row_begin);
    const int ket_s = Ls.ket_bin_start + (int)(q - __ldg(Ls.qoff + r));
    const int bra = __ldg(Ls.sorted + bra_s), ket = __ldg(Ls.sorted + ket_s);
    PerQuartet pq;
    if (!per_quartet(Ls, bra, ket, pq)) continue;
    const int npq = __ldg(Ls.pa.prim_n + bra) * __ldg(Ls.pa.prim_n + ket);
    const int ne = contract_g32<true>(ci, sv, Ls, bra, ket, S, CF, lane);
    t.prim += ne;
    t.skip += npq - ne;
    if (!ne) continue;
    ++t.quart;
    digest_per(ci, S + ci.out_base, 1, pq, Ls.KG, Ls.per.nbf, lane, 32);
    __syncwarp();
  }
}

// The quartet ranges a warp works on.  Static schedules: one range (group_range).
// Dynamic: chunks claimed from the launch's device counter.  Batched (L.n_sys > 0): chunks
// of the systems' concatenated quartet lists; a chunk is split at system boundaries
// (L.seg[s] = first index of system s) and each part runs with that system's record.
template <bool BATCH, int GS, class F>
__device__ __forceinline__ void for_each_range(const EriLaunch& L, long long wid, long long nw, int lane, unsigned gm,
                                               F&& f) {
  if (!BATCH && L.schedule != 2) {
    long long q0, q1;
    group_range(L, wid, nw, q0, q1);
    f(L, 0, q0, q1);
    return;
  }
  const long long total = L.q_count;
  while (true) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(L.work, (unsigned long long)L.chunk);
    c = __shfl_sync(gm, c, 0, GS);
    long long c0 = (long long)c;
    if (c0 >= total) break;
    const long long c1 = min(c0 + L.chunk, total);
    if constexpr (!BATCH) {
      f(L, 0, L.q_begin + c0, L.q_begin + c1);
    } else {
      while (c0 < c1) {
        int lo = 0, hi = L.n_sys - 1;  // last s with seg[s] <= c0
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (__ldg(L.seg + mid) <= c0) lo = mid; else hi = mid - 1;
        }
        const long long e = min(c1, __ldg(L.seg + lo + 1));
        const EriLaunch& Ls = L.batch[lo];
        f(Ls, lo, Ls.q_begin + (c0 - __ldg(L.seg + lo)), Ls.q_begin + (e - __ldg(L.seg + lo)));
        c0 = e;
      }
    }
  }
}

__device__ __forceinline__ void flush_tally(const EriLaunch& L, const Tally& t) {
  if (!L.counters) return;
  atomicAdd(L.counters + 0, t.prim);
  atomicAdd(L.counters + 1, t.quart);
  atomicAdd(L.counters + 2, t.skip);
  atomicAdd(L.counters + 3, t.q32);
  atomicAdd(L.counters + 4, t.p32);
}

template <int MODE, int PREC, bool BATCH, bool PER = false>
__global__ void __launch_bounds__(64, PREC == PREC_MIXED32 ? HFX_G1F_MINB : (BATCH ? HFX_G1B_MINB : HFX_G1_MINB))
    eri_g1_kernel(const EriLaunch L) {
  extern __shared__ double smem[];
  const int st = blockDim.x;
  double* Sd = smem + threadIdx.x;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ng = (long long)gridDim.x * blockDim.x;
  unsigned long long t0 = 0;
  if (L.busy && threadIdx.x == 0) t0 = globaltimer_ns();
  if (MODE == 0) {
    using R = typename std::conditional<PREC == PREC_MIXED32, float, double>::type;
    const int lane = threadIdx.x & 31;
    Tally t;
    G1Queue Q{reinterpret_cast<int4*>(smem + (size_t)L.ci.scratch * blockDim.x) + (threadIdx.x >> 5) * 64, 0};
    for_each_range<BATCH, 32>(L, gid >> 5, ng >> 5, lane, 0xffffffffu,
                              [&](const EriLaunch& Ls, int sys, long long q0, long long q1) {
                                g1_range<BATCH, PREC, R, PER>(L, L.ci, Ls, sys, q0, q1, Sd, st, lane, Q, t);
                              });
    g1_drain<BATCH, R, PER>(L, L.ci, Q, lane, Sd, st, t, true);
    flush_tally(L, t);
  } else {
    for (long long t = gid; t < L.diag_n; t += ng) {
      const int p = __ldg(L.diag_list + t);
      double mx = 0.0;
      if (contract_g1<double>(L.ci, L, p, p, Sd, st)) mx = diag_max(L.ci, Sd + L.ci.out_base * st, st);
      L.diag_Q[p] = sqrt(mx);
    }
  }
  record_busy(L, t0);
}

template <int MODE, int PREC, bool BATCH, bool PER = false>
__global__ void __launch_bounds__(64, BATCH ? HFX_G32B_MINB : (PREC == PREC_MIXED32 ? HFX_G32F_MINB : HFX_G32_MINB))
    eri_g32_kernel(const EriLaunch L) {
  extern __shared__ __align__(16) double smem[];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int gpb = blockDim.x >> 5;
  double* S = smem + grp * g32_stride(L.sv, PREC);
  double* CF = S + L.sv.group;
  const long long gid = (long long)blockIdx.x * gpb + grp;
  const long long ng = (long long)gridDim.x * gpb;
  unsigned long long t0 = 0;
  if (L.busy && threadIdx.x == 0) t0 = globaltimer_ns();
  if (MODE == 0) {
    Tally t;
    for_each_range<BATCH, 32>(L, gid, ng, lane, 0xffffffffu,
                              [&](const EriLaunch& Ls, int, long long q0, long long q1) {
                                if constexpr (PER)
                                  g32_range_per(L.ci, L.sv, Ls, q0, q1, S, CF, lane, t);
                                else
                                  g32_range<PREC>(L.ci, L.sv, Ls, q0, q1, S, CF, lane, t);
                              });
    if (lane == 0) flush_tally(L, t);
  } else {
    for (long long t = gid; t < L.diag_n; t += ng) {
      const int p = __ldg(L.diag_list + t);
      double mx = 0.0;
      if (contract_g32<false>(L.ci, L.sv, L, p, p, S, CF, lane)) mx = diag_max(L.ci, S + L.ci.out_base, 1);
      if (lane == 0) L.diag_Q[p] = sqrt(mx);
      __syncwarp();
    }
  }
  record_busy(L, t0);
}

// ---------------------------------------------------------------------------
// Host-side launch helpers
// ---------------------------------------------------------------------------
static const int kBlock = 64;

int eri_group_size(int cls) {
  // thread-per-quartet for classes whose scratch fits comfortably; warp otherwise
  return kClassInfo[cls].scratch <= HFX_G1_MAX_SCRATCH ? 1 : 32;
}

// Groups of 8 or 16 lanes (several quartets per warp) were measured on the 64-atom diamond:
// 1.1x to 10x slower than whole warps in every warp-group class and slower than one thread
// per quartet in the others, because each group needs its own scratch and coefficient
// sets, so shared memory caps the resident warps.  The kernel keeps the group size as a
// template parameter; only 32 is built.
bool eri_group_size_valid(int gs) { return gs == 1 || gs == 32; }

// Streams of the warp kernel per class (primitive quartets run at a time).  Defaults from a
// sweep of k = 1, 2, 4 over every warp class of the 64-atom diamond build (plain FP64): more
// streams fill the iterations with fewer FP64 warp instructions per primitive quartet, but
// their larger group scratch lowers the resident warps, which the largest classes feel most.
static const int kDefaultStreams[HFX_N_CLASSES] = {
    4, 4, 4, 4, 4, 4,   // ss|ss ps|ss ps|ps pp|ss pp|ps pp|pp
    4, 4, 4, 4,         // ds|ss ds|ps ds|pp ds|ds
    4, 4, 2, 4, 2,      // dp|ss dp|ps dp|pp dp|ds dp|dp
    4, 4, 2, 2, 1, 1};  // dd|ss dd|ps dd|pp dd|ds dd|dp dd|dd

static int variant_index(int cls, int streams) {
  const SchedVariant* v = kSchedInfo[cls];
  if (streams > 0) {
    for (int i = 0; i < 3; ++i)
      if (v[i].k == streams) return i;
    return -1;
  }
  int best = 0;  // the largest variant carried up to the default
  for (int i = 1; i < 3; ++i)
    if (v[i].k && v[i].k <= kDefaultStreams[cls]) best = i;
  return best;
}

bool eri_streams_valid(int cls, int streams) {
  return cls >= 0 && cls < HFX_N_CLASSES && (streams == 0 || variant_index(cls, streams) >= 0);
}

int eri_streams(int cls, int streams) {
  const int i = variant_index(cls, streams);
  return i < 0 ? 0 : kSchedInfo[cls][i].k;
}

// The kernel instance for a class launch.  gs: lanes per quartet (1 = a thread, 32 = a warp);
// mode 1 = Schwarz diagonal; prec: precision pass; batch = quartets of several systems.
template <int PREC>
static const void* kernel_ptr_p(int gs, bool batch) {
  if (gs == 1) return batch ? (const void*)eri_g1_kernel<0, PREC, true> : (const void*)eri_g1_kernel<0, PREC, false>;
  return batch ? (const void*)eri_g32_kernel<0, PREC, true> : (const void*)eri_g32_kernel<0, PREC, false>;
}

static const void* kernel_ptr(int mode, int gs, int prec, bool batch) {
  if (mode == 1) return gs == 1 ? (const void*)eri_g1_kernel<1, 0, false> : (const void*)eri_g32_kernel<1, 0, false>;
  if (prec == PREC_PERIODIC)
    return gs == 1 ? (const void*)eri_g1_kernel<0, 0, false, true> : (const void*)eri_g32_kernel<0, 0, false, true>;
  if (prec == PREC_MIXED64) return kernel_ptr_p<PREC_MIXED64>(gs, batch);
  if (prec == PREC_MIXED32) return kernel_ptr_p<PREC_MIXED32>(gs, batch);
  return kernel_ptr_p<PREC_FP64>(gs, batch);
}

static int effective_gs(int gs) { return gs == 1 ? 1 : 32; }

size_t eri_smem_bytes(int cls, int gs, int streams, int prec) {
  // one quartet per thread: interleaved scratch, then a 64-entry quartet queue per warp
  if (gs == 1) return sizeof(double) * (size_t)kClassInfo[cls].scratch * kBlock + sizeof(int4) * 64 * (kBlock / 32);
  const int i = variant_index(cls, streams);
  if (i < 0) return (size_t)1 << 30;
  return sizeof(double) * (size_t)g32_stride(kSchedInfo[cls][i], prec) * (kBlock / 32);
}

int eri_block_size() { return kBlock; }

cudaError_t eri_prepare() {
  // allow the largest dynamic shared memory any class needs, for every instance
  size_t mx = 0;
  for (int c = 0; c < HFX_N_CLASSES; ++c) {
    mx = std::max(mx, eri_smem_bytes(c, 1, 0));
    for (int i = 0; i < 3; ++i)
      if (kSchedInfo[c][i].k) mx = std::max(mx, eri_smem_bytes(c, 32, kSchedInfo[c][i].k));
  }
  if (mx > 227 * 1024) mx = 227 * 1024;
  for (int gs : {1, 32}) {
    cudaError_t e = cudaFuncSetAttribute(kernel_ptr(1, gs, 0, false), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mx);
    if (e != cudaSuccess) return e;
    for (int prec = 0; prec < 4; ++prec)
      for (int batch = 0; batch < (prec == PREC_PERIODIC ? 1 : 2); ++batch) {
        e = cudaFuncSetAttribute(kernel_ptr(0, gs, prec, batch), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
        if (e != cudaSuccess) return e;
      }
  }
  return cudaSuccess;
}

int eri_blocks_per_sm(int cls, int mode, int gs, int prec, bool batch, int streams) {
  int n = 0;
  const int g = effective_gs(gs);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_ptr(mode, g, prec, batch), kBlock,
                                                    eri_smem_bytes(cls, g, streams, prec)) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

int eri_groups_per_block(int gs) { return kBlock / effective_gs(gs); }

cudaError_t eri_launch(const EriLaunch& L0, int cls, int mode, int grid, cudaStream_t stream, int gs, int prec,
                       bool batch, int streams) {
  const int g = effective_gs(gs);
  const size_t smem = eri_smem_bytes(cls, g, streams, prec);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  const void* k = kernel_ptr(mode, g, prec, batch);
  EriLaunch L = L0;
  if (g == 32) L.sv = kSchedInfo[cls][variant_index(cls, streams)];
  void* args[] = {(void*)&L};
  return cudaLaunchKernel(k, dim3(grid), dim3(kBlock), args, smem, stream);
}

}  // namespace hfx
