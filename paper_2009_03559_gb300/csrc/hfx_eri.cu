// ERI kernels: one class launch evaluates every screened quartet of one class pair
// (bra pair bin >= ket pair bin) and digests it into the half exchange matrix, or, in
// diagonal mode, evaluates (p|p) for candidate pairs and stores the Schwarz factor.
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
__device__ __forceinline__ int contract_g1(const EriLaunch& L, int bra, int ket, double* S, int st) {
  const EriClassInfo& ci = L.ci;
  const PairArrays& pa = L.pa;
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
      if (!prim_setup(b, k, ci.E, ci.F, ci.Lt, L.omega2, L.boys, c, Gm)) continue;
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
// Contracted quartet, G = 32: a warp owns the quartet.  Lanes set up 32 primitive
// quartets at a time (coefficient sets in shared memory), then share the ops of each
// recurrence level.
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

template <typename R, bool FOLD>
__device__ __forceinline__ int contract_g32(const EriLaunch& L, int bra, int ket, R* S, R* CF, int lane) {
  const EriClassInfo& ci = L.ci;
  const PairArrays& pa = L.pa;
  R* V = S + ci.work_base;
  const int nb = __ldg(pa.prim_n + bra), nk = __ldg(pa.prim_n + ket);
  const PrimPair* pb = pa.prim + __ldg(pa.prim_off + bra);
  const PrimPair* pk = pa.prim + __ldg(pa.prim_off + ket);
  for (int a = lane; a < ci.n_acc; a += 32) S[a] = R(0);
  const int npq = nb * nk;
  int any = 0;
  for (int base = 0; base < npq; base += 32) {
    const int t = base + lane;
    if (t < npq) {
      const int ib = t / nk, ik = t - ib * nk;
      // the Boys step and the quantities feeding it stay in FP64 in either precision
      if constexpr (sizeof(R) == 4) {
        prim_setup_f32(pb[ib], pk[ik], ci.E, ci.F, ci.Lt, L.omega2, L.boys, reinterpret_cast<float*>(CF + lane * NCOEF));
      } else {
        CoefRg c;
        double Gm[kMaxLt + 1];
        const bool ok = prim_setup(pb[ib], pk[ik], ci.E, ci.F, ci.Lt, L.omega2, L.boys, c, Gm);
        store_coef<R>(c, Gm, ci.Lt, ok, CF + lane * NCOEF);
      }
    }
    __syncwarp();
    const int nchunk = min(32, npq - base);
    for (int u = 0; u < nchunk; ++u) {
      const R* cf = CF + u * NCOEF;
      if (cf[CF_SKIP] != R(0)) continue;
      ++any;
      const CoefSm<R> c{cf};
      for (int m = lane; m <= ci.Lt; m += 32) V[m] = cf[CF_G + m];
      __syncwarp();
      for (int lv = 0; lv < ci.n_bra_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = lane; o < n; o += 32) vrr_bra<FOLD>(ld_op(kVrrOps, off + o), V, S, 1, c);
        __syncwarp();
      }
      for (int lv = ci.n_bra_lv; lv < ci.n_bra_lv + ci.n_ket_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = lane; o < n; o += 32) vrr_ket<FOLD>(ld_op(kVrrOps, off + o), V, S, 1, c);
        __syncwarp();
      }
      for (int a = lane; a < ci.n_accl; a += 32) {
        const uint32_t w = __ldg(kAccSrc + ci.acc_off + a);
        S[w & 0xFFFF] += V[w >> 16];
      }
      __syncwarp();
    }
    __syncwarp();  // every lane is done with this chunk's coefficient sets
  }
  if (!any) return 0;
  if constexpr (sizeof(R) == 4) {
    // FP32 recurrences end at the contracted block: widen it to FP64 (through the free
    // coefficient area) so the horizontal recurrences and the spherical step, which cancel
    // across distant pairs, run in FP64 on the group's FP64 scratch
    double* Sd = reinterpret_cast<double*>(S);
    double* tmp = reinterpret_cast<double*>(CF);
    for (int a = lane; a < ci.n_acc; a += 32) tmp[a] = (double)S[a];
    __syncwarp();
    for (int a = lane; a < ci.n_acc; a += 32) Sd[a] = tmp[a];
    __syncwarp();
    post_stages<double>(ci, pa, bra, ket, Sd, lane);
  } else {
    post_stages<R>(ci, pa, bra, ket, S, lane);
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
// the mixed-precision warp kernel carries both recurrence paths: 4 blocks per SM keep it
// free of spills
#ifndef HFX_G32M_MINB
#define HFX_G32M_MINB 4
#endif

// The digest reads P_bd, P_bc, P_ad, P_ac.  max of their max|P| (or 1 without the table):
// 0 means the quartet contributes exactly nothing; the mixed-precision test uses it too.
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

template <int MODE>
__global__ void __launch_bounds__(64, HFX_G1_MINB) eri_g1_kernel(const EriLaunch L) {
  extern __shared__ double smem[];
  const int st = blockDim.x;
  double* S = smem + threadIdx.x;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ng = (long long)gridDim.x * blockDim.x;
  unsigned long long t0 = 0, n_prim = 0, n_skip = 0, n_quart = 0;
  if (L.busy && threadIdx.x == 0) t0 = globaltimer_ns();
  if (MODE == 0) {
    // a warp works on a range of the quartet list (an even share, or chunks claimed from
    // the device counter); its lanes take interleaved quartets of the range, so
    // neighbouring lanes work on neighbouring quartets
    const int lane = threadIdx.x & 31;
    long long q0, q1;
    bool more = true;
    if (L.schedule != 2) group_range(L, gid >> 5, ng >> 5, q0, q1);
    while (more) {
      if (L.schedule == 2) {
        unsigned long long c0 = 0;
        if (lane == 0) c0 = atomicAdd(L.work, (unsigned long long)L.chunk);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if ((long long)c0 >= L.q_count) break;
        q0 = L.q_begin + (long long)c0;
        q1 = min(q0 + L.chunk, L.q_begin + L.q_count);
      } else {
        more = false;
      }
      if (q0 + lane >= q1) continue;
      int r = find_row(L.qoff, L.row_begin, L.row_end, q0 + lane);
      for (long long q = q0 + lane; q < q1; q += 32) {
        while (__ldg(L.qoff + r + 1) <= q) ++r;
        const int bra_s = L.bra_bin_start + (r - L.row_begin);
        const int ket_s = L.ket_bin_start + (int)(q - __ldg(L.qoff + r));
        const int bra = __ldg(L.sorted + bra_s), ket = __ldg(L.sorted + ket_s);
        const int sa = __ldg(L.pa.sa + bra), sb = __ldg(L.pa.sb + bra);
        const int sc = __ldg(L.pa.sa + ket), sd = __ldg(L.pa.sb + ket);
        if (L.skip_zero && pmax4(L, sa, sb, sc, sd) == 0.0) continue;
        const int npq = __ldg(L.pa.prim_n + bra) * __ldg(L.pa.prim_n + ket);
        const int ne = contract_g1(L, bra, ket, S, st);
        n_prim += ne;
        n_skip += npq - ne;
        if (!ne) continue;
        ++n_quart;
        double deg = 1.0;
        if (sa == sb) deg *= 0.5;
        if (sc == sd) deg *= 0.5;
        if (bra_s == ket_s) deg *= 0.5;
        digest(L.ci, S + L.ci.out_base * st, st, __ldg(L.sh.bf_off + sa), __ldg(L.sh.bf_off + sb),
               __ldg(L.sh.bf_off + sc), __ldg(L.sh.bf_off + sd), deg, L.P, L.K, L.ld, 0, 1);
      }
    }
  } else {
    for (long long t = gid; t < L.diag_n; t += ng) {
      const int p = __ldg(L.diag_list + t);
      double mx = 0.0;
      if (contract_g1(L, p, p, S, st)) mx = diag_max(L.ci, S + L.ci.out_base * st, st);
      L.diag_Q[p] = sqrt(mx);
    }
  }
  record_busy(L, t0);
  if (L.counters && MODE == 0) {
    atomicAdd(L.counters + 0, n_prim);
    atomicAdd(L.counters + 1, n_quart);
    atomicAdd(L.counters + 2, n_skip);
  }
}

template <int MODE, bool FOLD, bool MIXED>
__global__ void __launch_bounds__(64, MIXED ? HFX_G32M_MINB : HFX_G32_MINB) eri_g32_kernel(const EriLaunch L,
                                                                                            int group_stride) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gpb = blockDim.x >> 5;
  double* S = smem + warp * group_stride;
  double* CF = S + L.ci.scratch + (L.ci.scratch & 1);
  float* Sf = reinterpret_cast<float*>(S);    // the FP32 engine reuses the group's memory
  float* CFf = reinterpret_cast<float*>(CF);
  unsigned long long n32q = 0, n32p = 0;
  const long long gid = (long long)blockIdx.x * gpb + warp;
  const long long ng = (long long)gridDim.x * gpb;
  unsigned long long t0 = 0, n_prim = 0, n_skip = 0, n_quart = 0;
  if (L.busy && threadIdx.x == 0) t0 = globaltimer_ns();
  if (MODE == 0) {
    long long q0, q1;
    bool more = true;
    if (L.schedule != 2) group_range(L, gid, ng, q0, q1);
    while (more) {
      if (L.schedule == 2) {
        unsigned long long c0 = 0;
        if (lane == 0) c0 = atomicAdd(L.work, (unsigned long long)L.chunk);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if ((long long)c0 >= L.q_count) break;
        q0 = L.q_begin + (long long)c0;
        q1 = min(q0 + L.chunk, L.q_begin + L.q_count);
      } else {
        more = false;
      }
      if (q0 >= q1) continue;
      int r = find_row(L.qoff, L.row_begin, L.row_end, q0);
      for (long long q = q0; q < q1; ++q) {
        while (__ldg(L.qoff + r + 1) <= q) ++r;
        const int bra_s = L.bra_bin_start + (r - L.row_begin);
        const int ket_s = L.ket_bin_start + (int)(q - __ldg(L.qoff + r));
        const int bra = __ldg(L.sorted + bra_s), ket = __ldg(L.sorted + ket_s);
        const int sa = __ldg(L.pa.sa + bra), sb = __ldg(L.pa.sb + bra);
        const int sc = __ldg(L.pa.sa + ket), sd = __ldg(L.pa.sb + ket);
        const double pm = pmax4(L, sa, sb, sc, sd);
        if (L.skip_zero && pm == 0.0) continue;
        // mixed precision: FP32 recurrences when the Schwarz bound times the largest density
        // element the quartet touches is below fp32_tau (warp-uniform decision)
        const bool f32 = MIXED && L.fp32_ok && __ldg(L.Qs + bra_s) * __ldg(L.Qs + ket_s) * pm < L.fp32_tau;
        const int npq = __ldg(L.pa.prim_n + bra) * __ldg(L.pa.prim_n + ket);
        int ne;
        if (MIXED && f32)
          ne = contract_g32<float, FOLD>(L, bra, ket, Sf, CFf, lane);
        else
          ne = contract_g32<double, FOLD>(L, bra, ket, S, CF, lane);
        n_prim += ne;
        n_skip += npq - ne;
        if (!ne) continue;
        ++n_quart;
        if (f32) {
          ++n32q;
          n32p += ne;
        }
        double deg = 1.0;
        if (sa == sb) deg *= 0.5;
        if (sc == sd) deg *= 0.5;
        if (bra_s == ket_s) deg *= 0.5;
        const int A = __ldg(L.sh.bf_off + sa), B = __ldg(L.sh.bf_off + sb);
        const int C = __ldg(L.sh.bf_off + sc), D = __ldg(L.sh.bf_off + sd);
        // an FP32 quartet leaves its final block in FP64 too (see contract_g32)
        digest(L.ci, S + L.ci.out_base, 1, A, B, C, D, deg, L.P, L.K, L.ld, lane, 32);
        __syncwarp();
      }
    }
  } else {
    for (long long t = gid; t < L.diag_n; t += ng) {
      const int p = __ldg(L.diag_list + t);
      double mx = 0.0;
      if (contract_g32<double, FOLD>(L, p, p, S, CF, lane)) mx = diag_max(L.ci, S + L.ci.out_base, 1);
      if (lane == 0) L.diag_Q[p] = sqrt(mx);
      __syncwarp();
    }
  }
  record_busy(L, t0);
  if (L.counters && MODE == 0 && lane == 0) {
    atomicAdd(L.counters + 0, n_prim);
    atomicAdd(L.counters + 1, n_quart);
    atomicAdd(L.counters + 2, n_skip);
    atomicAdd(L.counters + 3, n32q);
    atomicAdd(L.counters + 4, n32p);
  }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers
// ---------------------------------------------------------------------------
static const int kBlock = 64;

int eri_group_size(int cls) {
  // thread-per-quartet for classes whose scratch fits comfortably; warp otherwise
  return kClassInfo[cls].scratch <= HFX_G1_MAX_SCRATCH ? 1 : 32;
}

static int g32_stride(int cls) {
  const int s = kClassInfo[cls].scratch;
  return s + (s & 1) + 32 * NCOEF + 1;  // +1: stagger the groups' banks
}

size_t eri_smem_bytes(int cls, bool force32) {
  if (!force32 && eri_group_size(cls) == 1) return sizeof(double) * (size_t)kClassInfo[cls].scratch * kBlock;
  return sizeof(double) * (size_t)g32_stride(cls) * (kBlock / 32);
}

int eri_block_size() { return kBlock; }

// classes whose tables fold the accumulation (the thread-per-quartet ones)
static bool class_folds(int cls) { return kClassInfo[cls].scratch <= HFX_G1_MAX_SCRATCH; }

// force32 (mixed precision): warp groups for every class, with the FP32 path compiled in
static const void* kernel_ptr(int cls, int mode, bool force32) {
  const bool g1 = !force32 && eri_group_size(cls) == 1;
  if (g1) return mode == 0 ? (const void*)eri_g1_kernel<0> : (const void*)eri_g1_kernel<1>;
  const bool fold = class_folds(cls);
  if (mode == 1) return fold ? (const void*)eri_g32_kernel<1, true, false> : (const void*)eri_g32_kernel<1, false, false>;
  if (force32) return fold ? (const void*)eri_g32_kernel<0, true, true> : (const void*)eri_g32_kernel<0, false, true>;
  return fold ? (const void*)eri_g32_kernel<0, true, false> : (const void*)eri_g32_kernel<0, false, false>;
}

cudaError_t eri_prepare() {
  // allow the largest dynamic shared memory any class needs
  size_t mx = 0;
  for (int c = 0; c < HFX_N_CLASSES; ++c) mx = std::max(mx, std::max(eri_smem_bytes(c, false), eri_smem_bytes(c, true)));
  const void* ks[8] = {(const void*)eri_g1_kernel<0>, (const void*)eri_g1_kernel<1>,
                       (const void*)eri_g32_kernel<0, false, false>, (const void*)eri_g32_kernel<1, false, false>,
                       (const void*)eri_g32_kernel<0, true, false>, (const void*)eri_g32_kernel<1, true, false>,
                       (const void*)eri_g32_kernel<0, false, true>, (const void*)eri_g32_kernel<0, true, true>};
  for (auto k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int eri_blocks_per_sm(int cls, int mode, bool force32) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_ptr(cls, mode, force32), kBlock,
                                                    eri_smem_bytes(cls, force32)) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

cudaError_t eri_launch(const EriLaunch& L, int cls, int mode, int grid, cudaStream_t stream, bool force32) {
  const size_t smem = eri_smem_bytes(cls, force32);
  if (!force32 && eri_group_size(cls) == 1) {
    if (mode == 0)
      eri_g1_kernel<0><<<grid, kBlock, smem, stream>>>(L);
    else
      eri_g1_kernel<1><<<grid, kBlock, smem, stream>>>(L);
  } else {
    const int gs = g32_stride(cls);
    const bool fold = class_folds(cls);
    if (mode == 1) {
      if (fold) eri_g32_kernel<1, true, false><<<grid, kBlock, smem, stream>>>(L, gs);
      else eri_g32_kernel<1, false, false><<<grid, kBlock, smem, stream>>>(L, gs);
    } else if (force32) {
      if (fold) eri_g32_kernel<0, true, true><<<grid, kBlock, smem, stream>>>(L, gs);
      else eri_g32_kernel<0, false, true><<<grid, kBlock, smem, stream>>>(L, gs);
    } else {
      if (fold) eri_g32_kernel<0, true, false><<<grid, kBlock, smem, stream>>>(L, gs);
      else eri_g32_kernel<0, false, false><<<grid, kBlock, smem, stream>>>(L, gs);
    }
  }
  return cudaGetLastError();
}

}  // namespace hfx
