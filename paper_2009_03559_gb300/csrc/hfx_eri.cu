// ERI kernels: one class launch evaluates every screened quartet of one class pair
// (bra pair bin >= ket pair bin) -- of one system, or of all systems of a batch -- and
// digests it into the half exchange matrix, or, in diagonal mode, evaluates (p|p) for
// candidate pairs and stores the Schwarz factor.
#include <algorithm>
#include <cstdio>
#include "eri_engine.cuh"
#include "hfx_eri.h"

namespace hfx {

const EriClassInfo* class_info_host() { return kClassInfo; }

// ---------------------------------------------------------------------------
// Contracted quartet, G = 1: the thread owns the quartet.  Group scratch slots are
// interleaved over the block's threads (slot k of thread t at smem[k*st + t]).
// ---------------------------------------------------------------------------
// ci is the launch's class record (kernel parameter space); L supplies the system's data.
// In batched launches L lives in global memory: the fields the primitive loop needs are
// read into registers once per quartet.
__device__ __forceinline__ int contract_g1(const EriClassInfo& ci, const EriLaunch& L, int bra, int ket, double* S,
                                           int st) {
  const PairArrays pa = L.pa;
  const double omega2 = L.omega2;
  const double* boys = L.boys;
  double* V = S + ci.work_base * st;
  const int nb = __ldg(pa.prim_n + bra), nk = __ldg(pa.prim_n + ket);
  const PrimPair* pb = pa.prim + __ldg(pa.prim_off + bra);
  const PrimPair* pk = pa.prim + __ldg(pa.prim_off + ket);
  for (int a = 0; a < ci.n_acc; ++a) S[a * st] = 0.0;
  int any = 0;
  for (int ib = 0; ib < nb; ++ib) {
    const PrimPair b = pb[ib];
    for (int ik = 0; ik < nk; ++ik) {
      const PrimPair k = pk[ik];
      CoefRg c;
      double Gm[kMaxLt + 1];
      if (!prim_setup(b, k, ci.E, ci.F, ci.Lt, omega2, boys, c, Gm)) continue;
      ++any;
      for (int m = 0; m <= ci.Lt; ++m) V[m * st] = Gm[m];
      for (int lv = 0; lv < ci.n_bra_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = 0; o < n; ++o) vrr_bra<true>(ld_op(kVrrOps, off + o), V, S, st, c);
      }
      for (int lv = ci.n_bra_lv; lv < ci.n_bra_lv + ci.n_ket_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = 0; o < n; ++o) vrr_ket<true>(ld_op(kVrrOps, off + o), V, S, st, c);
      }
      for (int a = 0; a < ci.n_accl; ++a) {
        const uint32_t w = __ldg(kAccSrc + ci.acc_off + a);
        S[(w & 0xFFFF) * st] += V[(w >> 16) * st];
      }
    }
  }
  if (!any) return 0;
  double AB[3], CD[3];
  for (int i = 0; i < 3; ++i) {
    AB[i] = __ldg(pa.AB + 3 * bra + i);
    CD[i] = __ldg(pa.AB + 3 * ket + i);
  }
  for (int s = 0; s < ci.n_post; ++s) {
    const int off = ci.post_off[s], n = ci.post_n[s], type = ci.post_type[s];
    for (int o = 0; o < n; ++o) post_op(ld_op(kPostOps, off + o), type, S, st, AB, CD);
  }
  return any;
}

// ---------------------------------------------------------------------------
// Contracted quartet, G = GS (8, 16 or 32 lanes of one warp, gm = their lane mask): the
// group owns the quartet.  Lanes set up GS primitive quartets at a time (coefficient sets
// in shared memory), then share the ops of each recurrence level.  Smaller groups keep
// more lanes busy in classes whose recurrence levels have few ops.
// ---------------------------------------------------------------------------
// HRR and Cartesian -> spherical stages on the group scratch S (lanes share each stage)
template <typename R, int GS>
__device__ __forceinline__ void post_stages(const EriClassInfo& ci, const PairArrays& pa, int bra, int ket, R* S,
                                            int lane, unsigned gm) {
  R AB[3], CD[3];
  for (int i = 0; i < 3; ++i) {
    AB[i] = R(__ldg(pa.AB + 3 * bra + i));
    CD[i] = R(__ldg(pa.AB + 3 * ket + i));
  }
  for (int s = 0; s < ci.n_post; ++s) {
    const int off = ci.post_off[s], n = ci.post_n[s], type = ci.post_type[s];
    for (int o = lane; o < n; o += GS) post_op<R>(ld_op(kPostOps, off + o), type, S, 1, AB, CD);
    __syncwarp(gm);
  }
}

template <typename R, bool FOLD, int GS>
__device__ __forceinline__ int contract_g32(const EriClassInfo& ci, const EriLaunch& L, int bra, int ket, R* S, R* CF,
                                            int lane, unsigned gm) {
  const PairArrays pa = L.pa;
  const double omega2 = L.omega2;
  const double* boys = L.boys;
  R* V = S + ci.work_base;
  const int nb = __ldg(pa.prim_n + bra), nk = __ldg(pa.prim_n + ket);
  const PrimPair* pb = pa.prim + __ldg(pa.prim_off + bra);
  const PrimPair* pk = pa.prim + __ldg(pa.prim_off + ket);
  for (int a = lane; a < ci.n_acc; a += GS) S[a] = R(0);
  const int npq = nb * nk;
  int any = 0;
  for (int base = 0; base < npq; base += GS) {
    const int t = base + lane;
    if (t < npq) {
      const int ib = t / nk, ik = t - ib * nk;
      // the Boys step and the quantities feeding it stay in FP64 in either precision
      if constexpr (sizeof(R) == 4) {
        prim_setup_f32(pb[ib], pk[ik], ci.E, ci.F, ci.Lt, omega2, boys, reinterpret_cast<float*>(CF + lane * NCOEF));
      } else {
        CoefRg c;
        double Gm[kMaxLt + 1];
        const bool ok = prim_setup(pb[ib], pk[ik], ci.E, ci.F, ci.Lt, omega2, boys, c, Gm);
        store_coef<R>(c, Gm, ci.Lt, ok, CF + lane * NCOEF);
      }
    }
    __syncwarp(gm);
    const int nchunk = min(GS, npq - base);
    for (int u = 0; u < nchunk; ++u) {
      const R* cf = CF + u * NCOEF;
      if (cf[CF_SKIP] != R(0)) continue;
      ++any;
      const CoefSm<R> c{cf};
      for (int m = lane; m <= ci.Lt; m += GS) V[m] = cf[CF_G + m];
      __syncwarp(gm);
      for (int lv = 0; lv < ci.n_bra_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = lane; o < n; o += GS) vrr_bra<FOLD>(ld_op(kVrrOps, off + o), V, S, 1, c);
        __syncwarp(gm);
      }
      for (int lv = ci.n_bra_lv; lv < ci.n_bra_lv + ci.n_ket_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = lane; o < n; o += GS) vrr_ket<FOLD>(ld_op(kVrrOps, off + o), V, S, 1, c);
        __syncwarp(gm);
      }
      for (int a = lane; a < ci.n_accl; a += GS) {
        const uint32_t w = __ldg(kAccSrc + ci.acc_off + a);
        S[w & 0xFFFF] += V[w >> 16];
      }
      __syncwarp(gm);
    }
    __syncwarp(gm);  // every lane is done with this chunk's coefficient sets
  }
  if (!any) return 0;
  if constexpr (sizeof(R) == 4) {
    // FP32 recurrences end at the contracted block: widen it to FP64 (through the free
    // coefficient area) so the horizontal recurrences and the spherical step, which cancel
    // across distant pairs, run in FP64 on the group's FP64 scratch
    double* Sd = reinterpret_cast<double*>(S);
    double* tmp = reinterpret_cast<double*>(CF);
    for (int a = lane; a < ci.n_acc; a += GS) tmp[a] = (double)S[a];
    __syncwarp(gm);
    for (int a = lane; a < ci.n_acc; a += GS) Sd[a] = tmp[a];
    __syncwarp(gm);
    post_stages<double, GS>(ci, pa, bra, ket, Sd, lane, gm);
  } else {
    post_stages<R, GS>(ci, pa, bra, ket, S, lane, gm);
  }
  return any;
}

// Register caps: 6 blocks of 64 threads per SM (at most 170 registers) measured fastest
// for both kernels; the FP64 set-up phase otherwise takes registers the hot VRR loop
// does not need and costs occupancy.
#ifndef HFX_G1_MINB
#define HFX_G1_MINB 6
#endif
#ifndef HFX_G32_MINB
#define HFX_G32_MINB 6
#endif
// the batched thread-per-quartet kernel carries the batch bookkeeping too: 4 blocks per SM
// keep it free of spills
#ifndef HFX_G1B_MINB
#define HFX_G1B_MINB 4
#endif
// the mixed-precision warp kernel carries both recurrence paths: 4 blocks per SM keep it
// free of spills
#ifndef HFX_G32M_MINB
#define HFX_G32M_MINB 4
#endif

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

__device__ __forceinline__ void record_busy(const EriLaunch& L, unsigned long long t0) {
  if (L.busy && threadIdx.x == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    atomicAdd(L.busy + smid, globaltimer_ns() - t0);
  }
}

// Per-thread tallies of one kernel, added to the launch's counters once at the end.
struct Tally {
  unsigned long long prim = 0, quart = 0, skip = 0, q32 = 0, p32 = 0;
};

// Quartets [q0, q1) of the launch record Ls, G = 1: lane `lane` of the warp takes
// q0 + lane, q0 + lane + 32, ... (neighbouring lanes on neighbouring quartets).  ci: the
// launch's class record; the system fields used per quartet are copied to registers once
// per range (Ls may live in global memory, where the K updates could alias it).
__device__ __forceinline__ void g1_range(const EriClassInfo& ci, const EriLaunch& Ls, long long q0, long long q1,
                                         double* S, int st, int lane, Tally& t) {
  if (q0 + lane >= q1) return;
  const long long* qoff = Ls.qoff;
  const int* sorted = Ls.sorted;
  const int* psa = Ls.pa.sa;
  const int* psb = Ls.pa.sb;
  const int* pn = Ls.pa.prim_n;
  const int* bf_off = Ls.sh.bf_off;
  const int row_begin = Ls.row_begin, bra0 = Ls.bra_bin_start, ket0 = Ls.ket_bin_start;
  const bool skip = Ls.skip_zero;
  const double dens = Ls.dens_tau;
  const double* Qs = Ls.Qs;
  const double* P = Ls.P;
  double* K = Ls.K;
  const int ld = Ls.ld;
  int r = find_row(qoff, row_begin, Ls.row_end, q0 + lane);
  for (long long q = q0 + lane; q < q1; q += 32) {
    while (__ldg(qoff + r + 1) <= q) ++r;
    const int bra_s = bra0 + (r - row_begin);
    const int ket_s = ket0 + (int)(q - __ldg(qoff + r));
    const int bra = __ldg(sorted + bra_s), ket = __ldg(sorted + ket_s);
    const int sa = __ldg(psa + bra), sb = __ldg(psb + bra);
    const int sc = __ldg(psa + ket), sd = __ldg(psb + ket);
    const double pm = pmax4(Ls, sa, sb, sc, sd);
    if (skip && pm == 0.0) continue;
    if (dens > 0.0 && __ldg(Qs + bra_s) * __ldg(Qs + ket_s) * pm < dens) continue;
    const int npq = __ldg(pn + bra) * __ldg(pn + ket);
    const int ne = contract_g1(ci, Ls, bra, ket, S, st);
    t.prim += ne;
    t.skip += npq - ne;
    if (!ne) continue;
    ++t.quart;
    double deg = 1.0;
    if (sa == sb) deg *= 0.5;
    if (sc == sd) deg *= 0.5;
    if (bra_s == ket_s) deg *= 0.5;
    digest(ci, S + ci.out_base * st, st, __ldg(bf_off + sa), __ldg(bf_off + sb), __ldg(bf_off + sc),
           __ldg(bf_off + sd), deg, P, K, ld, 0, 1);
  }
}

// Quartets [q0, q1) of the launch record Ls, G = 32: the warp takes them one by one.
template <bool FOLD, bool MIXED, int GS>
__device__ __forceinline__ void g32_range(const EriClassInfo& ci, const EriLaunch& Ls, long long q0, long long q1,
                                          double* S, double* CF, int lane, unsigned gm, Tally& t) {
  float* Sf = reinterpret_cast<float*>(S);  // the FP32 engine reuses the group's memory
  float* CFf = reinterpret_cast<float*>(CF);
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
    // mixed precision: FP32 recurrences when the Schwarz bound times the largest density
    // element the quartet touches (or the largest of all of P) is below fp32_tau
    // (warp-uniform decision)
    bool f32 = false;
    if (MIXED && Ls.fp32_ok) {
      const double pf = Ls.pglob ? __ldg(Ls.pglob) : pm;
      f32 = __ldg(Ls.Qs + bra_s) * __ldg(Ls.Qs + ket_s) * pf < Ls.fp32_tau;
    }
    const int npq = __ldg(Ls.pa.prim_n + bra) * __ldg(Ls.pa.prim_n + ket);
    int ne;
    if (MIXED && f32)
      ne = contract_g32<float, FOLD, GS>(ci, Ls, bra, ket, Sf, CFf, lane, gm);
    else
      ne = contract_g32<double, FOLD, GS>(ci, Ls, bra, ket, S, CF, lane, gm);
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
    digest(ci, S + ci.out_base, 1, A, B, C, D, deg, Ls.P, Ls.K, Ls.ld, lane, GS);
    __syncwarp(gm);
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
    f(L, q0, q1);
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
      f(L, L.q_begin + c0, L.q_begin + c1);
    } else {
      while (c0 < c1) {
        int lo = 0, hi = L.n_sys - 1;  // last s with seg[s] <= c0
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (__ldg(L.seg + mid) <= c0) lo = mid; else hi = mid - 1;
        }
        const long long e = min(c1, __ldg(L.seg + lo + 1));
        const EriLaunch& Ls = L.batch[lo];
        f(Ls, Ls.q_begin + (c0 - __ldg(L.seg + lo)), Ls.q_begin + (e - __ldg(L.seg + lo)));
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

template <int MODE, bool BATCH>
__global__ void __launch_bounds__(64, BATCH ? HFX_G1B_MINB : HFX_G1_MINB) eri_g1_kernel(const EriLaunch L) {
  extern __shared__ double smem[];
  const int st = blockDim.x;
  double* S = smem + threadIdx.x;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ng = (long long)gridDim.x * blockDim.x;
  unsigned long long t0 = 0;
  if (L.busy && threadIdx.x == 0) t0 = globaltimer_ns();
  if (MODE == 0) {
    const int lane = threadIdx.x & 31;
    Tally t;
    for_each_range<BATCH, 32>(L, gid >> 5, ng >> 5, lane, 0xffffffffu,
                          [&](const EriLaunch& Ls, long long q0, long long q1) {
                            g1_range(L.ci, Ls, q0, q1, S, st, lane, t);
                          });
    flush_tally(L, t);
  } else {
    for (long long t = gid; t < L.diag_n; t += ng) {
      const int p = __ldg(L.diag_list + t);
      double mx = 0.0;
      if (contract_g1(L.ci, L, p, p, S, st)) mx = diag_max(L.ci, S + L.ci.out_base * st, st);
      L.diag_Q[p] = sqrt(mx);
    }
  }
  record_busy(L, t0);
}

template <int MODE, bool FOLD, bool MIXED, bool BATCH, int GS>
__global__ void __launch_bounds__(64, MIXED ? HFX_G32M_MINB : HFX_G32_MINB) eri_g32_kernel(const EriLaunch L,
                                                                                            int group_stride) {
  static_assert(GS == 8 || GS == 16 || GS == 32, "group size");
  static_assert(!MIXED || GS == 32, "the FP32 engine widens its block through 32 coefficient sets");
  extern __shared__ double smem[];
  const int lane = threadIdx.x & (GS - 1), grp = threadIdx.x / GS;
  const unsigned gm = GS == 32 ? 0xffffffffu : (((1u << GS) - 1u) << ((threadIdx.x & 31) & ~(GS - 1)));
  const int gpb = blockDim.x / GS;
  double* S = smem + grp * group_stride;
  double* CF = S + L.ci.scratch + (L.ci.scratch & 1);
  const long long gid = (long long)blockIdx.x * gpb + grp;
  const long long ng = (long long)gridDim.x * gpb;
  unsigned long long t0 = 0;
  if (L.busy && threadIdx.x == 0) t0 = globaltimer_ns();
  if (MODE == 0) {
    Tally t;
    for_each_range<BATCH, GS>(L, gid, ng, lane, gm, [&](const EriLaunch& Ls, long long q0, long long q1) {
      g32_range<FOLD, MIXED, GS>(L.ci, Ls, q0, q1, S, CF, lane, gm, t);
    });
    if (lane == 0) flush_tally(L, t);
  } else {
    for (long long t = gid; t < L.diag_n; t += ng) {
      const int p = __ldg(L.diag_list + t);
      double mx = 0.0;
      if (contract_g32<double, FOLD, GS>(L.ci, L, p, p, S, CF, lane, gm)) mx = diag_max(L.ci, S + L.ci.out_base, 1);
      if (lane == 0) L.diag_Q[p] = sqrt(mx);
      __syncwarp(gm);
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

static int group_stride(int cls, int gs) {
  const int s = kClassInfo[cls].scratch;
  return s + (s & 1) + gs * NCOEF + 1;  // +1: stagger the groups' banks
}

// classes whose tables fold the accumulation (the thread-per-quartet ones)
static bool class_folds(int cls) { return kClassInfo[cls].scratch <= HFX_G1_MAX_SCRATCH; }

template <int MODE, bool MIXED, bool BATCH, int GS>
static const void* group_kernel(bool fold) {
  return fold ? (const void*)eri_g32_kernel<MODE, true, MIXED, BATCH, GS>
              : (const void*)eri_g32_kernel<MODE, false, MIXED, BATCH, GS>;
}

// The kernel instance for a class launch.  gs: lanes per quartet (1 = a thread, 32 = a warp);
// mode 1 = Schwarz diagonal; batch = quartets of several systems in one launch.
static const void* kernel_ptr(int cls, int mode, int gs, bool mixed, bool batch) {
  const bool fold = class_folds(cls);
  if (gs == 1) {
    if (mode == 1) return (const void*)eri_g1_kernel<1, false>;
    return batch ? (const void*)eri_g1_kernel<0, true> : (const void*)eri_g1_kernel<0, false>;
  }
  if (mode == 1) return group_kernel<1, false, false, 32>(fold);
  if (mixed) return batch ? group_kernel<0, true, true, 32>(fold) : group_kernel<0, true, false, 32>(fold);
  return batch ? group_kernel<0, false, true, 32>(fold) : group_kernel<0, false, false, 32>(fold);
}

// the group size a launch actually runs with
static int effective_gs(int mode, int gs, bool mixed) {
  if (gs == 1) return 1;
  return (mode == 1 || mixed || !eri_group_size_valid(gs)) ? 32 : gs;
}

size_t eri_smem_bytes(int cls, int gs) {
  if (gs == 1) return sizeof(double) * (size_t)kClassInfo[cls].scratch * kBlock;
  return sizeof(double) * (size_t)group_stride(cls, gs) * (kBlock / gs);
}

int eri_block_size() { return kBlock; }

cudaError_t eri_prepare() {
  // allow the largest dynamic shared memory any class needs, for every instance
  size_t mx = 0;
  for (int c = 0; c < HFX_N_CLASSES; ++c)
    for (int gs : {1, 32}) mx = std::max(mx, eri_smem_bytes(c, gs));
  if (mx > 227 * 1024) mx = 227 * 1024;
  for (int cls : {0, HFX_N_CLASSES - 1})
    for (int mode = 0; mode < 2; ++mode)
      for (int gs : {1, 32})
        for (int mixed = 0; mixed < 2; ++mixed)
          for (int batch = 0; batch < 2; ++batch) {
            cudaError_t e = cudaFuncSetAttribute(kernel_ptr(cls, mode, gs, mixed, batch),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
            if (e != cudaSuccess) return e;
          }
  return cudaSuccess;
}

int eri_blocks_per_sm(int cls, int mode, int gs, bool mixed, bool batch) {
  int n = 0;
  const int g = effective_gs(mode, gs, mixed);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_ptr(cls, mode, g, mixed, batch), kBlock,
                                                    eri_smem_bytes(cls, g)) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

int eri_groups_per_block(int mode, int gs, bool mixed) { return kBlock / effective_gs(mode, gs, mixed); }

cudaError_t eri_launch(const EriLaunch& L, int cls, int mode, int grid, cudaStream_t stream, int gs, bool mixed,
                       bool batch) {
  const int g = effective_gs(mode, gs, mixed);
  const size_t smem = eri_smem_bytes(cls, g);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  const void* k = kernel_ptr(cls, mode, g, mixed, batch);
  int stride = group_stride(cls, g);
  void* args_g1[] = {(void*)&L};
  void* args_grp[] = {(void*)&L, (void*)&stride};
  return cudaLaunchKernel(k, dim3(grid), dim3(kBlock), g == 1 ? args_g1 : args_grp, smem, stream);
}

}  // namespace hfx
