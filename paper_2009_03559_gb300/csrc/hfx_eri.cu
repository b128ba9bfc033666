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
__device__ __forceinline__ int contract_g32(const EriLaunch& L, int bra, int ket, double* S, double* CF,
                                             int lane) {
  const EriClassInfo& ci = L.ci;
  const PairArrays& pa = L.pa;
  double* V = S + ci.work_base;
  const int nb = __ldg(pa.prim_n + bra), nk = __ldg(pa.prim_n + ket);
  const PrimPair* pb = pa.prim + __ldg(pa.prim_off + bra);
  const PrimPair* pk = pa.prim + __ldg(pa.prim_off + ket);
  for (int a = lane; a < ci.n_acc; a += 32) S[a] = 0.0;
  const int npq = nb * nk;
  int any = 0;
  for (int base = 0; base < npq; base += 32) {
    const int t = base + lane;
    if (t < npq) {
      const int ib = t / nk, ik = t - ib * nk;
      CoefRg c;
      double Gm[kMaxLt + 1];
      const bool ok = prim_setup(pb[ib], pk[ik], ci.E, ci.F, ci.Lt, L.omega2, L.boys, c, Gm);
      store_coef(c, Gm, ci.Lt, ok, CF + lane * NCOEF);
    }
    __syncwarp();
    const int nchunk = min(32, npq - base);
    for (int u = 0; u < nchunk; ++u) {
      const double* cf = CF + u * NCOEF;
      if (cf[CF_SKIP] != 0.0) continue;
      ++any;
      const CoefSm c{cf};
      for (int m = lane; m <= ci.Lt; m += 32) V[m] = cf[CF_G + m];
      __syncwarp();
      for (int lv = 0; lv < ci.n_bra_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = lane; o < n; o += 32) vrr_bra<false>(ld_op(kVrrOps, off + o), V, S, 1, c);
        __syncwarp();
      }
      for (int lv = ci.n_bra_lv; lv < ci.n_bra_lv + ci.n_ket_lv; ++lv) {
        const int off = ci.lv_off[lv], n = ci.lv_n[lv];
        for (int o = lane; o < n; o += 32) vrr_ket<false>(ld_op(kVrrOps, off + o), V, S, 1, c);
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
  double AB[3], CD[3];
  for (int i = 0; i < 3; ++i) {
    AB[i] = __ldg(pa.AB + 3 * bra + i);
    CD[i] = __ldg(pa.AB + 3 * ket + i);
  }
  for (int s = 0; s < ci.n_post; ++s) {
    const int off = ci.post_off[s], n = ci.post_n[s], type = ci.post_type[s];
    for (int o = lane; o < n; o += 32) post_op(ld_op(kPostOps, off + o), type, S, 1, AB, CD);
    __syncwarp();
  }
  return any;
}

#ifndef HFX_G1_MINB
#define HFX_G1_MINB 6
#endif
#ifndef HFX_G32_MINB
#define HFX_G32_MINB 6
#endif

// The digest reads P_bd, P_bc, P_ad, P_ac: if all four blocks are exactly zero the
// quartet contributes exactly nothing.
__device__ __forceinline__ bool zero_p_blocks(const EriLaunch& L, int sa, int sb, int sc, int sd) {
  if (!L.pmax) return false;
  const double* pm = L.pmax;
  const size_t ns = L.ns;
  return __ldg(pm + sb * ns + sd) == 0.0 && __ldg(pm + sb * ns + sc) == 0.0 &&
         __ldg(pm + sa * ns + sd) == 0.0 && __ldg(pm + sa * ns + sc) == 0.0;
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
        if (zero_p_blocks(L, sa, sb, sc, sd)) continue;
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

template <int MODE>
__global__ void __launch_bounds__(64, HFX_G32_MINB) eri_g32_kernel(const EriLaunch L, int group_stride) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gpb = blockDim.x >> 5;
  double* S = smem + warp * group_stride;
  double* CF = S + L.ci.scratch + (L.ci.scratch & 1);
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
        if (zero_p_blocks(L, sa, sb, sc, sd)) continue;
        const int npq = __ldg(L.pa.prim_n + bra) * __ldg(L.pa.prim_n + ket);
        const int ne = contract_g32(L, bra, ket, S, CF, lane);
        n_prim += ne;
        n_skip += npq - ne;
        if (!ne) continue;
        ++n_quart;
        double deg = 1.0;
        if (sa == sb) deg *= 0.5;
        if (sc == sd) deg *= 0.5;
        if (bra_s == ket_s) deg *= 0.5;
        digest(L.ci, S + L.ci.out_base, 1, __ldg(L.sh.bf_off + sa), __ldg(L.sh.bf_off + sb),
               __ldg(L.sh.bf_off + sc), __ldg(L.sh.bf_off + sd), deg, L.P, L.K, L.ld, lane, 32);
        __syncwarp();
      }
    }
  } else {
    for (long long t = gid; t < L.diag_n; t += ng) {
      const int p = __ldg(L.diag_list + t);
      double mx = 0.0;
      if (contract_g32(L, p, p, S, CF, lane)) mx = diag_max(L.ci, S + L.ci.out_base, 1);
      if (lane == 0) L.diag_Q[p] = sqrt(mx);
      __syncwarp();
    }
  }
  record_busy(L, t0);
  if (L.counters && MODE == 0 && lane == 0) {
    atomicAdd(L.counters + 0, n_prim);
    atomicAdd(L.counters + 1, n_quart);
    atomicAdd(L.counters + 2, n_skip);
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

size_t eri_smem_bytes(int cls) {
  if (eri_group_size(cls) == 1) return sizeof(double) * (size_t)kClassInfo[cls].scratch * kBlock;
  return sizeof(double) * (size_t)g32_stride(cls) * (kBlock / 32);
}

int eri_block_size() { return kBlock; }

static const void* kernel_ptr(int cls, int mode) {
  const bool g1 = eri_group_size(cls) == 1;
  if (g1) return mode == 0 ? (const void*)eri_g1_kernel<0> : (const void*)eri_g1_kernel<1>;
  return mode == 0 ? (const void*)eri_g32_kernel<0> : (const void*)eri_g32_kernel<1>;
}

cudaError_t eri_prepare() {
  // allow the largest dynamic shared memory any class needs
  size_t mx = 0;
  for (int c = 0; c < HFX_N_CLASSES; ++c) mx = std::max(mx, eri_smem_bytes(c));
  const void* ks[4] = {(const void*)eri_g1_kernel<0>, (const void*)eri_g1_kernel<1>,
                       (const void*)eri_g32_kernel<0>, (const void*)eri_g32_kernel<1>};
  for (auto k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int eri_blocks_per_sm(int cls, int mode) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel_ptr(cls, mode), kBlock,
                                                    eri_smem_bytes(cls)) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

cudaError_t eri_launch(const EriLaunch& L, int cls, int mode, int grid, cudaStream_t stream) {
  const size_t smem = eri_smem_bytes(cls);
  if (eri_group_size(cls) == 1) {
    if (mode == 0)
      eri_g1_kernel<0><<<grid, kBlock, smem, stream>>>(L);
    else
      eri_g1_kernel<1><<<grid, kBlock, smem, stream>>>(L);
  } else {
    const int gs = g32_stride(cls);
    if (mode == 0)
      eri_g32_kernel<0><<<grid, kBlock, smem, stream>>>(L, gs);
    else
      eri_g32_kernel<1><<<grid, kBlock, smem, stream>>>(L, gs);
  }
  return cudaGetLastError();
}

}  // namespace hfx
