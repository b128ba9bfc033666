// C ABI of the HFX library: context, basis upload, pair-list build, K build.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hfx.h"
#include "hfx_eri.h"
#include "hfx_internal.cuh"
#include "hfx_setup.h"
#include "hfx_ctx.h"

using namespace hfx;

static thread_local std::string g_init_err;

namespace hfx {
// message for hfx_last_error(NULL) from entry points that have no context
void set_global_error(const std::string& msg) { g_init_err = msg; }

// allocation-failure injection: the k-th context allocation from the arming call fails
static std::atomic<int> g_alloc_countdown{0};
bool alloc_fault_due() {
  int c = g_alloc_countdown.load();
  while (c > 0) {
    if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
  }
  return false;
}
}  // namespace hfx

extern "C" int hfx_debug_fail_alloc(int k) {
  if (k < 0) return HFX_ERR_ARG;
  hfx::g_alloc_countdown.store(k);
  return HFX_OK;
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ctx->cuda_fail(#call, e_); \
  } while (0)
#define RK(call)                 \
  do {                           \
    int r_ = (call);             \
    if (r_ != HFX_OK) return r_; \
  } while (0)

extern "C" void hfx_default_options(hfx_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->omega = 0.11;
  opt->schwarz_tau = 1e-10;
  opt->rcut_bohr = 0.0;
  opt->prim_tau = 1e-22;
  opt->precision = HFX_FP64;
  opt->schedule = HFX_SCHED_DYNAMIC;
  opt->skip_zero_p = 1;
  opt->fp32_tau = 1e-6;
  opt->fp32_class_mask = HFX_FP32_CLASSES_DEFAULT;
}

static int init_basis_impl(hfx_ctx** out, int n_atoms, const double* xyz, int n_shells, const int* shell_atom,
                           const int* shell_l, const int* shell_nprim, const double* alpha, const double* coef,
                           const hfx_options* opt, void* stream, bool periodic = false);

extern "C" int hfx_init_basis(hfx_ctx** out, int n_atoms, const double* xyz, int n_shells,
                              const int* shell_atom, const int* shell_l, const int* shell_nprim,
                              const double* alpha, const double* coef, const hfx_options* opt, void* stream) {
  return init_basis_impl(out, n_atoms, xyz, n_shells, shell_atom, shell_l, shell_nprim, alpha, coef, opt, stream);
}

static int init_basis_impl(hfx_ctx** out, int n_atoms, const double* xyz, int n_shells, const int* shell_atom,
                           const int* shell_l, const int* shell_nprim, const double* alpha, const double* coef,
                           const hfx_options* opt, void* stream, bool periodic) {
  g_init_err.clear();
  if (!out) {
    g_init_err = "out is NULL";
    return HFX_ERR_ARG;
  }
  *out = nullptr;
  if (n_atoms <= 0 || n_shells <= 0 || !xyz || !shell_atom || !shell_l || !shell_nprim || !alpha || !coef) {
    g_init_err = "empty basis or NULL array";
    return HFX_ERR_ARG;
  }
  hfx_options o;
  hfx_default_options(&o);
  if (opt) o = *opt;
  if (!(o.omega >= 0.0) || !(o.schwarz_tau >= 0.0) || !(o.prim_tau >= 0.0) || !(o.fp32_tau >= 0.0) ||
      !(o.density_tau >= 0.0) || !(o.dist_tau >= 0.0) ||
      (o.precision != HFX_FP64 && o.precision != HFX_MIXED) ||
      (o.fp32_pmax_global != 0 && o.fp32_pmax_global != 1) ||
      (o.schedule != HFX_SCHED_QUARTET && o.schedule != HFX_SCHED_PAIR && o.schedule != HFX_SCHED_DYNAMIC)) {
    g_init_err = "invalid options";
    return HFX_ERR_ARG;
  }
  std::vector<int> prim_off(n_shells), bf_off(n_shells);
  int np = 0, nb = 0;
  for (int s = 0; s < n_shells; ++s) {
    if (shell_l[s] < 0 || shell_l[s] > 2) {
      g_init_err = "shell " + std::to_string(s) + ": angular momentum " + std::to_string(shell_l[s]) +
                   " outside 0..2";
      return HFX_ERR_UNSUPPORTED_L;
    }
    if (shell_nprim[s] < 1 || shell_nprim[s] > 8 || shell_atom[s] < 0 || shell_atom[s] >= n_atoms) {
      g_init_err = "shell " + std::to_string(s) + ": bad primitive count or atom index";
      return HFX_ERR_ARG;
    }
    prim_off[s] = np;
    bf_off[s] = nb;
    np += shell_nprim[s];
    nb += 2 * shell_l[s] + 1;
  }
  for (int k = 0; k < np; ++k)
    if (!(alpha[k] > 0.0) || !std::isfinite(coef[k])) {
      g_init_err = "primitive " + std::to_string(k) + ": exponent must be > 0 and weight finite";
      return HFX_ERR_ARG;
    }
  for (int a = 0; a < 3 * n_atoms; ++a)
    if (!std::isfinite(xyz[a])) {
      g_init_err = "non-finite coordinate";
      return HFX_ERR_ARG;
    }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_init_err = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return HFX_ERR_CUDA;
  }
  hfx_ctx* ctx = new hfx_ctx();
  ctx->stream = (cudaStream_t)stream;
  ctx->opt = o;
  ctx->n_atoms = n_atoms;
  ctx->n_shells = n_shells;
  ctx->n_bf = nb;
  ctx->n_prim = np;
  ctx->h_l.assign(shell_l, shell_l + n_shells);
  cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, dev);
  auto bail = [&](int code) {
    g_init_err = ctx->err;
    hfx_free(ctx);
    return code;
  };
  int r;
  if ((r = ctx->alloc(&ctx->d_xyz, 3 * (size_t)n_atoms)) || (r = ctx->alloc(&ctx->d_alpha, np)) ||
      (r = ctx->alloc(&ctx->d_coef, np)) || (r = ctx->alloc(&ctx->d_w, np)) ||
      (r = ctx->alloc(&ctx->d_boys, (size_t)(kMaxLt + 1) * kBoysTableLen)) || (r = ctx->alloc(&ctx->d_atom, n_shells)) ||
      (r = ctx->alloc(&ctx->d_l, n_shells)) || (r = ctx->alloc(&ctx->d_nprim, n_shells)) ||
      (r = ctx->alloc(&ctx->d_prim_off, n_shells)) || (r = ctx->alloc(&ctx->d_bf_off, n_shells)) ||
      (r = ctx->alloc(&ctx->d_energy, 1)) || (r = ctx->alloc(&ctx->d_busy, 1024)) ||
      (r = ctx->alloc(&ctx->d_counters, kNCnt * 21)) ||
      (r = ctx->alloc(&ctx->d_pmax, periodic ? 1 : (size_t)n_shells * n_shells)) || (r = ctx->alloc(&ctx->d_work, 64)) ||
      (r = ctx->alloc(&ctx->d_pglob, 1)))
    return bail(r);
  ctx->n_part = 2 * ctx->n_sm;
  if ((r = ctx->alloc(&ctx->d_part, 2 * (size_t)ctx->n_part))) return bail(r);
  cudaStream_t s = ctx->stream;
#define CKI(call)                                                   \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return bail(ctx->cuda_fail(#call, e_)); \
  } while (0)
  CKI(cudaMemcpyAsync(ctx->d_xyz, xyz, sizeof(double) * 3 * n_atoms, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(ctx->d_alpha, alpha, sizeof(double) * np, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(ctx->d_coef, coef, sizeof(double) * np, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(ctx->d_atom, shell_atom, sizeof(int) * n_shells, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(ctx->d_l, shell_l, sizeof(int) * n_shells, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(ctx->d_nprim, shell_nprim, sizeof(int) * n_shells, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(ctx->d_prim_off, prim_off.data(), sizeof(int) * n_shells, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(ctx->d_bf_off, bf_off.data(), sizeof(int) * n_shells, cudaMemcpyHostToDevice, s));
  CKI(launch_normalize(n_shells, ctx->d_l, ctx->d_nprim, ctx->d_prim_off, ctx->d_alpha, ctx->d_coef, ctx->d_w, s));
  CKI(launch_boys_table(ctx->d_boys, s));
  CKI(eri_prepare());
  CKI(cudaStreamSynchronize(s));  // host arrays may be released by the caller after return
  for (auto& ev : ctx->ev) {
    if (cudaEventCreate(&ev) != cudaSuccess) return bail(ctx->fail(HFX_ERR_CUDA, "cudaEventCreate"));
  }
  ctx->ev_ok = true;
#undef CKI
  *out = ctx;
  return HFX_OK;
}

// Flops (add/mul 1, fma 2) of one primitive-quartet set-up as written in prim_core and
// write_set, with the table branch of both Boys evaluations (each: the offset from the
// grid point and two seven-term Horner chains, 25 flops; the asymptotic branch taken for
// T >= 60 costs 7 + 2 Lt and is not counted separately).
static double setup_flops(int E, int F, int Lt, bool erfc) {
  // s, rsqrt(s), 1/s, rho/p, rho/q, rho, PQ, r2, T, pref, Boys(T), 2T
  double f = 1 + 5 + 1 + 2 + 1 + 3 + 5 + 1 + 2 + 25 + 1;
  if (erfc)
    f += 7 + 1 + 1 + 25 + 1 + Lt + 1 + 3 + 5.0 * Lt;  // sqrt(kappa), kappa, kT, Boys(kT), c_m, G recursion
  else
    f += 1 + 1 + 3.0 * Lt;
  if (E > 0) f += 3;   // W - P
  if (F > 0) f += 4;   // W - Q, 3/(2(p+q))
  return f;
}
// a primitive quartet dropped at kappa T >= table end costs the set-up up to that test
static double skip_flops() { return 47 + 7 + 1 + 1; }

EriLaunch hfx::base_launch(hfx_ctx* ctx) {
  EriLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.pa.sa = ctx->d_sa;
  L.pa.sb = ctx->d_sb;
  L.pa.prim_off = ctx->d_pp_off;
  L.pa.prim_n = ctx->d_pp_n;
  L.pa.AB = ctx->d_AB;
  L.pa.prim = ctx->d_pp;
  L.sh.bf_off = ctx->d_bf_off;
  L.sh.atom = ctx->d_atom;
  L.boys = ctx->d_boys;
  L.omega = ctx->opt.omega;
  L.omega2 = ctx->opt.omega * ctx->opt.omega;
  L.schedule = ctx->opt.schedule;
  return L;
}

static int grid_for(hfx_ctx* ctx, int cls, int mode, long long work_items, int gs, int prec = 0,
                    bool batch = false, int streams = 0) {
  const int groups_per_block = eri_groups_per_block(gs);
  long long need = (work_items + groups_per_block - 1) / groups_per_block;
  long long cap = (long long)eri_blocks_per_sm(cls, mode, gs, prec, batch, streams) * ctx->n_sm;
  long long g = std::min(need, cap);
  return (int)std::max(1LL, g);
}

extern "C" int hfx_build_pairs(hfx_ctx* ctx) {
  if (!ctx) return HFX_ERR_ARG;
  ctx->free_pairs();
  cudaStream_t s = ctx->stream;
  CK(cudaEventRecord(ctx->ev[44], s));
  const long long n = ctx->n_shells;
  // candidates: shell pairs I >= J (triangular index), or for a periodic context every
  // (home-cell shell, image shell) pair (rectangular index)
  const long long n_tri = ctx->periodic ? (long long)ctx->n_home_shells * n : n * (n + 1) / 2;
  // 1. candidate pairs passing the orbital cutoff
  int* d_flag;
  long long* d_cand_t;
  int* d_num;
  RK(ctx->alloc(&d_flag, n_tri, true));
  RK(ctx->alloc(&d_cand_t, n_tri, true));
  RK(ctx->alloc(&d_num, 8, true));
  if (ctx->periodic)
    CK(launch_pair_flags_rect(n_tri, (int)n, ctx->d_atom, ctx->d_xyz, ctx->opt.rcut_bohr, d_flag, s));
  else
    CK(launch_pair_flags(n_tri, ctx->d_atom, ctx->d_xyz, ctx->opt.rcut_bohr, d_flag, s));
  size_t tb = 0;
  CK(select_flagged(nullptr, tb, n_tri, d_flag, d_cand_t, d_num, s));
  void* tmp;
  size_t tmp_bytes = std::max<size_t>(tb, 1 << 20);
  // one temp buffer big enough for every CUB call below (sized conservatively)
  {
    size_t t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0;
    int nn = (int)std::min<long long>(n_tri, 0x7fffffff);
    CK(scan_int(nullptr, t2, (int*)nullptr, (int*)nullptr, nn, s));
    CK(sort_int_keys(nullptr, t3, nullptr, nullptr, nullptr, nullptr, nn, 3, s));
    CK(sort_double_desc(nullptr, t4, nullptr, nullptr, nullptr, nullptr, nn, s));
    CK(reduce_max(nullptr, t5, nullptr, nullptr, nn, s));
    CK(scan_ll_inclusive(nullptr, t6, nullptr, nullptr, 6 * nn, s));
    tmp_bytes = std::max({tmp_bytes, t2, t3, t4, t5, t6});
  }
  RK(ctx->alloc((char**)&tmp, tmp_bytes, true));
  tb = tmp_bytes;
  CK(select_flagged(tmp, tb, n_tri, d_flag, d_cand_t, d_num, s));
  int n_cand = 0;
  CK(cudaMemcpyAsync(&n_cand, d_num, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  ctx->n_cand = n_cand;
  if (n_cand == 0) return ctx->fail(HFX_ERR_ARG, "no shell pair passes the orbital cutoff");
  // 2. orientation, class, AB, primitive pairs
  int* d_cap;
  RK(ctx->alloc(&ctx->d_sa, n_cand, true));
  RK(ctx->alloc(&ctx->d_sb, n_cand, true));
  RK(ctx->alloc(&ctx->d_pcls, n_cand, true));
  RK(ctx->alloc(&ctx->d_AB, 3 * (size_t)n_cand, true));
  RK(ctx->alloc(&d_cap, n_cand, true));
  RK(ctx->alloc(&ctx->d_pp_off, n_cand, true));
  RK(ctx->alloc(&ctx->d_pp_n, n_cand, true));
  RK(ctx->alloc(&ctx->d_Q, n_cand, true));
  if (ctx->periodic) {
    RK(ctx->alloc(&ctx->d_home_first, n_cand, true));
    CK(launch_pair_setup_rect(n_cand, d_cand_t, (int)n, ctx->d_l, ctx->d_nprim, ctx->d_atom, ctx->d_xyz, ctx->d_sa,
                              ctx->d_sb, ctx->d_pcls, ctx->d_AB, d_cap, ctx->d_home_first, s));
  } else {
    CK(launch_pair_setup(n_cand, d_cand_t, ctx->d_l, ctx->d_nprim, ctx->d_atom, ctx->d_xyz, ctx->d_sa, ctx->d_sb,
                         ctx->d_pcls, ctx->d_AB, d_cap, s));
  }
  tb = tmp_bytes;
  CK(scan_int(tmp, tb, d_cap, ctx->d_pp_off, n_cand, s));
  int last[2];
  CK(cudaMemcpyAsync(&last[0], ctx->d_pp_off + n_cand - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&last[1], d_cap + n_cand - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const long long n_pp = (long long)last[0] + last[1];
  RK(ctx->alloc(&ctx->d_pp, n_pp, true));
  CK(launch_prim_fill(n_cand, ctx->d_sa, ctx->d_sb, ctx->d_nprim, ctx->d_prim_off, ctx->d_atom, ctx->d_xyz,
                      ctx->d_alpha, ctx->d_w, ctx->d_pp_off, ctx->opt.prim_tau, ctx->d_pp, ctx->d_pp_n, s));
  // 3. group candidates by pair class, Schwarz diagonal per class
  int *d_iota, *d_ckey, *d_cidx, *d_cnt;
  RK(ctx->alloc(&d_iota, n_cand, true));
  RK(ctx->alloc(&d_ckey, n_cand, true));
  RK(ctx->alloc(&d_cidx, n_cand, true));
  RK(ctx->alloc(&d_cnt, 16, true));
  CK(launch_iota(n_cand, d_iota, s));
  tb = tmp_bytes;
  CK(sort_int_keys(tmp, tb, ctx->d_pcls, d_ckey, d_iota, d_cidx, n_cand, 3, s));
  CK(cudaMemsetAsync(d_cnt, 0, 16 * sizeof(int), s));
  CK(launch_hist(n_cand, ctx->d_pcls, d_cnt, s));
  int cnt[8] = {};
  CK(cudaMemcpyAsync(cnt, d_cnt, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  {
    EriLaunch L = base_launch(ctx);
    int start = 0;
    for (int pc = 0; pc < 6; ++pc) {
      if (cnt[pc] > 0) {
        const int cls = pc * (pc + 1) / 2 + pc;
        L.ci = class_info_host()[cls];
        L.diag_list = d_cidx + start;
        L.diag_n = cnt[pc];
        L.diag_Q = ctx->d_Q;
        const int gs = eri_group_size(cls);
        CK(eri_launch(L, cls, 1, grid_for(ctx, cls, 1, cnt[pc], gs), s, gs, 0, false));
      }
      start += cnt[pc];
    }
  }
  // 4. pair Schwarz test and bins: sort by Q descending, then stably by bin
  double* d_qmax;
  double* d_qsorted;
  int *d_ord, *d_bkey, *d_bkey_sorted;
  RK(ctx->alloc(&d_qmax, 1, true));
  RK(ctx->alloc(&d_qsorted, n_cand, true));
  RK(ctx->alloc(&d_ord, n_cand, true));
  RK(ctx->alloc(&d_bkey, n_cand, true));
  RK(ctx->alloc(&d_bkey_sorted, n_cand, true));
  RK(ctx->alloc(&ctx->d_sorted, n_cand, true));
  tb = tmp_bytes;
  CK(reduce_max(tmp, tb, ctx->d_Q, d_qmax, n_cand, s));
  tb = tmp_bytes;
  CK(sort_double_desc(tmp, tb, ctx->d_Q, d_qsorted, d_iota, d_ord, n_cand, s));
  CK(launch_bin_keys(n_cand, ctx->d_Q, d_qmax, ctx->opt.schwarz_tau, ctx->d_pcls, d_ord, d_bkey, s));
  tb = tmp_bytes;
  CK(sort_int_keys(tmp, tb, d_bkey, d_bkey_sorted, d_ord, ctx->d_sorted, n_cand, 3, s));
  CK(cudaMemsetAsync(d_cnt, 0, 16 * sizeof(int), s));
  CK(launch_hist(n_cand, d_bkey, d_cnt, s));
  int bins[8] = {};
  CK(cudaMemcpyAsync(bins, d_cnt, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  RowTable rt{};
  int acc = 0;
  for (int b = 0; b < 6; ++b) {
    rt.bin_start[b] = acc;
    rt.bin_size[b] = bins[b];
    acc += bins[b];
  }
  rt.bin_start[6] = acc;
  rt.bin_size[6] = bins[6];
  ctx->n_kept = acc;
  RK(ctx->alloc(&ctx->d_Qs, std::max(1, acc), true));
  CK(launch_gather_q(acc, ctx->d_sorted, ctx->d_Q, ctx->d_Qs, s));
  if (ctx->opt.dist_tau > 0.0) {
    double* d_dc;
    RK(ctx->alloc(&d_dc, 5 * (size_t)n_cand, true));
    RK(ctx->alloc(&ctx->d_dist, 5 * (size_t)std::max(1, acc), true));
    CK(launch_pair_dist(n_cand, ctx->d_sa, ctx->d_sb, ctx->d_nprim, ctx->d_prim_off, ctx->d_atom, ctx->d_xyz,
                        ctx->d_alpha, d_dc, s));
    CK(launch_gather5(acc, ctx->d_sorted, d_dc, ctx->d_dist, s));
  }
  // 5. quartet task rows and prefix sums
  int rows = 0;
  for (int cp = 0; cp < 21; ++cp) {
    int hi = 0;
    while ((hi + 1) * (hi + 2) / 2 <= cp) ++hi;
    rt.row_base[cp] = rows;
    rows += rt.bin_size[hi];
  }
  rt.row_base[21] = rows;
  ctx->rt = rt;
  ctx->n_rows = rows;
  long long *d_rown, *d_bounds;
  RK(ctx->alloc(&d_rown, std::max(1, rows), true));
  RK(ctx->alloc(&ctx->d_qoff, (size_t)rows + 1, true));
  RK(ctx->alloc(&d_bounds, 32, true));
  CK(launch_count(rows, rt, ctx->d_Qs, ctx->opt.schwarz_tau, d_rown, s, !ctx->periodic));
  CK(cudaMemsetAsync(ctx->d_qoff, 0, sizeof(long long), s));
  if (rows > 0) {
    tb = tmp_bytes;
    CK(scan_ll_inclusive(tmp, tb, d_rown, ctx->d_qoff + 1, rows, s));
  }
  CK(launch_gather_bounds(rt, ctx->d_qoff, d_bounds, s));
  long long bounds[22];
  CK(cudaMemcpyAsync(bounds, d_bounds, 22 * sizeof(long long), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ctx->ev[45], s));
  CK(cudaStreamSynchronize(s));
  cudaEventElapsedTime(&ctx->ms_pairs, ctx->ev[44], ctx->ev[45]);
  long long total = 0;
  for (int cp = 0; cp < 21; ++cp) {
    ctx->cls_qbegin[cp] = bounds[cp];
    ctx->cls_q[cp] = bounds[cp + 1] - bounds[cp];
    ctx->stats.n_quartets_class[cp] = ctx->cls_q[cp];
    total += ctx->cls_q[cp];
  }
  ctx->stats.n_pairs_cutoff = n_cand;
  ctx->stats.n_pairs_kept = ctx->n_kept;
  ctx->stats.n_quartets = total;
  ctx->stats.ms_pairs = ctx->ms_pairs;
  ctx->pairs_ready = true;
  return HFX_OK;
}

// ---------------------------------------------------------------------------
// Periodic images (Eq. vx lattice sums)
// ---------------------------------------------------------------------------
extern "C" int hfx_init_periodic(hfx_ctx** out, int n_atoms, const double* xyz, const double* lattice, int n_shells,
                                 const int* shell_atom, const int* shell_l, const int* shell_nprim,
                                 const double* alpha, const double* coef, const hfx_options* opt, void* stream) {
  g_init_err.clear();
  if (!out || !lattice || n_atoms <= 0 || n_shells <= 0 || !xyz || !shell_atom || !shell_nprim || !alpha || !coef) {
    g_init_err = "NULL argument or empty cell";
    if (out) *out = nullptr;
    return HFX_ERR_ARG;
  }
  *out = nullptr;
  hfx_options o;
  hfx_default_options(&o);
  if (opt) o = *opt;
  if (!(o.rcut_bohr > 0.0)) {
    g_init_err = "a periodic context needs an orbital cutoff (rcut_bohr > 0): it bounds the image sums";
    return HFX_ERR_ARG;
  }
  if (o.precision != HFX_FP64) {
    g_init_err = "periodic builds run in FP64";
    return HFX_ERR_ARG;
  }
  // box of image cells: every cell whose atoms can come within 2 r_c of a home-cell atom
  const double* L = lattice;
  double diam = 0.0;
  for (int a = 0; a < n_atoms; ++a)
    for (int b = 0; b < n_atoms; ++b) {
      double d2 = 0.0;
      for (int i = 0; i < 3; ++i) d2 += (xyz[3 * a + i] - xyz[3 * b + i]) * (xyz[3 * a + i] - xyz[3 * b + i]);
      diam = std::max(diam, std::sqrt(d2));
    }
  auto cross = [](const double* u, const double* v, double* w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
  };
  double c01[3], c12[3], c20[3];
  cross(L + 0, L + 3, c01);
  cross(L + 3, L + 6, c12);
  cross(L + 6, L + 0, c20);
  const double vol = std::fabs(L[0] * c12[0] + L[1] * c12[1] + L[2] * c12[2]);
  if (!(vol > 0.0) || !std::isfinite(vol)) {
    g_init_err = "lattice vectors are degenerate";
    return HFX_ERR_ARG;
  }
  int nr[3];
  const double* cr[3] = {c12, c20, c01};  // normals of the faces spanned by the other two vectors
  for (int i = 0; i < 3; ++i) {
    const double h = vol / std::sqrt(cr[i][0] * cr[i][0] + cr[i][1] * cr[i][1] + cr[i][2] * cr[i][2]);
    nr[i] = (int)std::ceil((2.0 * o.rcut_bohr + diam) / h);
    if (nr[i] > 8) {
      g_init_err = "orbital cutoff reaches more than 8 cells: use a larger cell";
      return HFX_ERR_ARG;
    }
  }
  std::vector<int> cells = {0, 0, 0};
  for (int i = -nr[0]; i <= nr[0]; ++i)
    for (int j = -nr[1]; j <= nr[1]; ++j)
      for (int k = -nr[2]; k <= nr[2]; ++k)
        if (i || j || k) cells.insert(cells.end(), {i, j, k});
  const int nc = (int)cells.size() / 3;
  // the image cluster: the cell's atoms and shells repeated cell after cell
  std::vector<double> cx((size_t)3 * n_atoms * nc), ca, cc;
  std::vector<int> csa((size_t)n_shells * nc), csl((size_t)n_shells * nc), csn((size_t)n_shells * nc);
  int np = 0;
  for (int sh = 0; sh < n_shells; ++sh) np += shell_nprim[sh];
  ca.reserve((size_t)np * nc);
  cc.reserve((size_t)np * nc);
  for (int c = 0; c < nc; ++c) {
    const int* n3 = &cells[3 * c];
    for (int a = 0; a < n_atoms; ++a)
      for (int i = 0; i < 3; ++i)
        cx[(size_t)3 * (c * n_atoms + a) + i] = xyz[3 * a + i] + n3[0] * L[i] + n3[1] * L[3 + i] + n3[2] * L[6 + i];
    for (int sh = 0; sh < n_shells; ++sh) {
      csa[(size_t)c * n_shells + sh] = shell_atom[sh] + c * n_atoms;
      csl[(size_t)c * n_shells + sh] = shell_l[sh];
      csn[(size_t)c * n_shells + sh] = shell_nprim[sh];
    }
    ca.insert(ca.end(), alpha, alpha + np);
    cc.insert(cc.end(), coef, coef + np);
  }
  int r = init_basis_impl(out, n_atoms * nc, cx.data(), n_shells * nc, csa.data(), csl.data(), csn.data(), ca.data(),
                          cc.data(), &o, stream, true);
  if (r != HFX_OK) return r;
  hfx_ctx* ctx = *out;
  ctx->periodic = true;
  ctx->n_home_atoms = n_atoms;
  ctx->n_home_shells = n_shells;
  ctx->n_home_bf = ctx->n_bf / nc;
  ctx->n_cells = nc;
  std::memcpy(ctx->lattice, lattice, sizeof(ctx->lattice));
  ctx->h_cells = cells;
  std::vector<int> shell_cell((size_t)n_shells * nc), shell_bf((size_t)n_shells * nc);
  int bf = 0;
  for (int sh = 0; sh < n_shells; ++sh) {
    for (int c = 0; c < nc; ++c) {
      shell_cell[(size_t)c * n_shells + sh] = c;
      shell_bf[(size_t)c * n_shells + sh] = bf;
    }
    bf += 2 * shell_l[sh] + 1;
  }
  auto bail = [&](int code) {
    g_init_err = ctx->err;
    hfx_free(ctx);
    *out = nullptr;
    return code;
  };
  if ((r = ctx->alloc(&ctx->d_shell_cell, shell_cell.size())) || (r = ctx->alloc(&ctx->d_shell_bf, shell_bf.size())) ||
      (r = ctx->alloc(&ctx->d_cell_xyz, cells.size())))
    return bail(r);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(ctx->d_shell_cell, shell_cell.data(), sizeof(int) * shell_cell.size(),
                           cudaMemcpyHostToDevice, ctx->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ctx->d_shell_bf, shell_bf.data(), sizeof(int) * shell_bf.size(), cudaMemcpyHostToDevice,
                           ctx->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ctx->d_cell_xyz, cells.data(), sizeof(int) * cells.size(), cudaMemcpyHostToDevice,
                           ctx->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
    return bail(ctx->cuda_fail("periodic tables", e));
  return HFX_OK;
}

extern "C" int hfx_periodic_cells(const hfx_ctx* ctx, int* cells, int max_n) {
  if (!ctx || !ctx->periodic) return HFX_ERR_ARG;
  if (cells) std::memcpy(cells, ctx->h_cells.data(), sizeof(int) * 3 * std::min(max_n, ctx->n_cells));
  return ctx->n_cells;
}

extern "C" int hfx_build_K_periodic(hfx_ctx* ctx, int n_R, const int* R_cells, const double* P_R, int n_G,
                                    const int* G_cells, double* K_G) {
  if (!ctx) return HFX_ERR_ARG;
  if (!ctx->periodic) return ctx->fail(HFX_ERR_STATE, "hfx_build_K_periodic needs a context from hfx_init_periodic");
  if (!ctx->pairs_ready) return ctx->fail(HFX_ERR_STATE, "hfx_build_K_periodic before hfx_build_pairs");
  if (n_R <= 0 || n_G <= 0 || !R_cells || !P_R || !G_cells || !K_G)
    return ctx->fail(HFX_ERR_ARG, "empty or NULL density or cell lists");
  int rb = 0;
  for (int i = 0; i < 3 * n_R; ++i) rb = std::max(rb, std::abs(R_cells[i]));
  if (rb > 32) return ctx->fail(HFX_ERR_ARG, "density cell offsets beyond 32 cells");
  const int w = 2 * rb + 1;
  std::vector<int> rmap((size_t)w * w * w, -1);
  for (int r = 0; r < n_R; ++r) {
    const int* R = R_cells + 3 * r;
    int& slot = rmap[((size_t)(R[0] + rb) * w + (R[1] + rb)) * w + (R[2] + rb)];
    if (slot >= 0) return ctx->fail(HFX_ERR_ARG, "a density cell offset appears twice");
    slot = r;
  }
  cudaStream_t s = ctx->stream;
  const int nbf = ctx->n_home_bf;
  CK(cudaStreamSynchronize(s));  // an earlier build may still read the reused tables
  RK(ctx->scratch(&ctx->d_rmap, &ctx->rmap_cap, rmap.size()));
  int* d_rmap = ctx->d_rmap;
  CK(cudaMemcpyAsync(d_rmap, rmap.data(), sizeof(int) * rmap.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(K_G, 0, sizeof(double) * (size_t)n_G * nbf * nbf, s));
  if (ctx->timing) CK(cudaEventRecord(ctx->ev[0], s));
  EriLaunch L = base_launch(ctx);
  L.sorted = ctx->d_sorted;
  L.qoff = ctx->d_qoff;
  L.Qs = ctx->d_Qs;
  L.per.shell_cell = ctx->d_shell_cell;
  L.per.shell_bf = ctx->d_shell_bf;
  L.per.cell_xyz = ctx->d_cell_xyz;
  L.per.home_first = ctx->d_home_first;
  L.per.rmap = d_rmap;
  L.per.rb = rb;
  L.per.P = P_R;
  L.per.nbf = nbf;
  // density-block maxima of every P^R (the home shells are the first n_home_shells of the
  // image basis, so its bf_off / l arrays serve)
  RK(ctx->scratch(&ctx->d_pmaxR, &ctx->pmaxR_cap, (size_t)n_R * ctx->n_home_shells * ctx->n_home_shells));
  double* d_pmaxR = ctx->d_pmaxR;
  CK(launch_pmax_blocks(n_R, ctx->n_home_shells, nbf, ctx->d_bf_off, ctx->d_l, P_R, d_pmaxR, s));
  L.per.pmax = d_pmaxR;
  L.per.nsh = ctx->n_home_shells;
  L.schedule = HFX_SCHED_DYNAMIC;
  for (int g = 0; g < n_G; ++g) {
    const int* G = G_cells + 3 * g;
    // K^{-G} = (K^G)^T (exchanging bra and ket pairs maps the quartets of cell G onto those of
    // cell -G): a cell whose opposite came earlier in the list is a transpose
    int mirror = -1;
    for (int j = 0; j < g && mirror < 0; ++j)
      if (G_cells[3 * j] == -G[0] && G_cells[3 * j + 1] == -G[1] && G_cells[3 * j + 2] == -G[2]) mirror = j;
    if (mirror >= 0) {
      CK(launch_transpose(nbf, K_G + (size_t)mirror * nbf * nbf, K_G + (size_t)g * nbf * nbf, s));
      continue;
    }
    double sh[3];
    for (int i = 0; i < 3; ++i)
      sh[i] = G[0] * ctx->lattice[i] + G[1] * ctx->lattice[3 + i] + G[2] * ctx->lattice[6 + i];
    L.KG = K_G + (size_t)g * nbf * nbf;
    CK(cudaMemsetAsync(ctx->d_work, 0, 64 * sizeof(unsigned long long), s));
    for (int cp = 0; cp < 21; ++cp) {
      if (ctx->cls_q[cp] == 0) continue;
      int hi = 0;
      while ((hi + 1) * (hi + 2) / 2 <= cp) ++hi;
      const int lo = cp - hi * (hi + 1) / 2;
      L.ci = class_info_host()[cp];
      L.row_begin = ctx->rt.row_base[cp];
      L.row_end = ctx->rt.row_base[cp + 1];
      L.bra_bin_start = ctx->rt.bin_start[hi];
      L.ket_bin_start = ctx->rt.bin_start[lo];
      L.q_begin = ctx->cls_qbegin[cp];
      L.q_count = ctx->cls_q[cp];
      const int gs = eri_group_size(cp);
      L.chunk = gs == 1 ? 256 : 8;
      // forward: (p | q + G L) for bra class hi >= ket class lo; reverse (hi > lo): the
      // quartets (p | q + G L) with class(p) = lo < class(q) = hi, evaluated as (q | p - G L)
      for (int rev = 0; rev < (hi > lo ? 2 : 1); ++rev) {
        L.reverse = rev;
        for (int i = 0; i < 3; ++i) {
          L.gcell[i] = G[i];
          L.shift[i] = rev ? -sh[i] : sh[i];
        }
        L.work = ctx->d_work + cp + 21 * rev;
        CK(eri_launch(L, cp, 0, grid_for(ctx, cp, 0, L.q_count, gs, 3), s, gs, 3, false));
      }
    }
  }
  if (ctx->timing) CK(cudaEventRecord(ctx->ev[1], s));
  return HFX_OK;
}

extern "C" int hfx_part_range(int64_t count, int part, int n_parts, int64_t* q0, int64_t* q1) {
  if (!q0 || !q1 || count < 0 || n_parts < 1 || part < 0 || part >= n_parts) return HFX_ERR_ARG;
  // floor(count * p / n_parts) without overflow for count < 2^62
  auto cut = [&](int p) {
    return (count / n_parts) * p + ((count % n_parts) * p) / n_parts;
  };
  *q0 = cut(part);
  *q1 = cut(part + 1);
  return HFX_OK;
}

static int build_K_impl(hfx_ctx* ctx, const double* P, double* K, int ld, int part, int n_parts);

extern "C" int hfx_build_K(hfx_ctx* ctx, const double* P, double* K, int ld) {
  return build_K_impl(ctx, P, K, ld, 0, 1);
}

extern "C" int hfx_build_K_part(hfx_ctx* ctx, const double* P, double* K, int ld, int part, int n_parts) {
  if (!ctx) return HFX_ERR_ARG;
  if (n_parts < 1 || part < 0 || part >= n_parts)
    return ctx->fail(HFX_ERR_ARG, "part must be in 0..n_parts-1");
  if (n_parts > 1 && ctx->opt.schedule == HFX_SCHED_PAIR)
    return ctx->fail(HFX_ERR_ARG, "partitions split the quartet list: use the quartet or dynamic schedule");
  return build_K_impl(ctx, P, K, ld, part, n_parts);
}

static int build_K_impl(hfx_ctx* ctx, const double* P, double* K, int ld, int part, int n_parts) {
  if (!ctx) return HFX_ERR_ARG;
  if (ctx->periodic) return ctx->fail(HFX_ERR_STATE, "a periodic context builds K with hfx_build_K_periodic");
  if (!ctx->pairs_ready) return ctx->fail(HFX_ERR_STATE, "hfx_build_K before hfx_build_pairs");
  if (!P || !K || ld < ctx->n_bf) return ctx->fail(HFX_ERR_ARG, "NULL matrix or ld < n_bf");
  cudaStream_t s = ctx->stream;
  const int n = ctx->n_bf;
  if (ctx->timing) {
    CK(cudaEventRecord(ctx->ev[0], s));
    CK(cudaMemsetAsync(ctx->d_busy, 0, 1024 * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ctx->d_counters, 0, kNCnt * 21 * sizeof(unsigned long long), s));
  }
  if (ld == n)
    CK(cudaMemsetAsync(K, 0, sizeof(double) * (size_t)n * n, s));
  else
    CK(cudaMemset2DAsync(K, sizeof(double) * ld, 0, sizeof(double) * n, n, s));
  EriLaunch L = base_launch(ctx);
  L.sorted = ctx->d_sorted;
  L.qoff = ctx->d_qoff;
  L.P = P;
  L.K = K;
  L.ld = ld;
  if (ctx->opt.schedule == HFX_SCHED_DYNAMIC) CK(cudaMemsetAsync(ctx->d_work, 0, 64 * sizeof(unsigned long long), s));
  const bool mixed = ctx->opt.precision == HFX_MIXED;
  if (ctx->opt.skip_zero_p || mixed || ctx->opt.density_tau > 0.0) {
    const bool glob = mixed && ctx->opt.fp32_pmax_global;
    CK(launch_pmax(ctx->n_shells, ctx->d_bf_off, ctx->d_l, P, ld, ctx->d_pmax, glob ? ctx->d_pglob : nullptr, s));
    L.pmax = ctx->d_pmax;
    L.pglob = glob ? ctx->d_pglob : nullptr;
    L.ns = ctx->n_shells;
  }
  L.skip_zero = ctx->opt.skip_zero_p;
  L.fp32_tau = ctx->opt.fp32_tau;
  L.dens_tau = ctx->opt.density_tau;
  L.dist_tau = ctx->opt.dist_tau;
  L.dist = ctx->d_dist;
  L.Qs = ctx->d_Qs;
  if (ctx->timing) L.busy = ctx->d_busy;
  for (int cp = 0; cp < 21; ++cp) {
    ctx->class_launched[cp] = false;
    if (ctx->cls_q[cp] == 0) continue;
    int hi = 0;
    while ((hi + 1) * (hi + 2) / 2 <= cp) ++hi;
    const int lo = cp - hi * (hi + 1) / 2;
    L.ci = class_info_host()[cp];
    L.row_begin = ctx->rt.row_base[cp];
    L.row_end = ctx->rt.row_base[cp + 1];
    L.bra_bin_start = ctx->rt.bin_start[hi];
    L.ket_bin_start = ctx->rt.bin_start[lo];
    // partition `part` of n_parts: a contiguous 1/n_parts of every class's quartet list
    int64_t p0 = 0, p1 = 0;
    hfx_part_range(ctx->cls_q[cp], part, n_parts, &p0, &p1);
    if (p1 == p0) continue;
    L.q_begin = ctx->cls_qbegin[cp] + p0;
    L.q_count = p1 - p0;
    L.counters = ctx->timing ? ctx->d_counters + kNCnt * cp : nullptr;
    // mixed precision: a class allowed FP32 runs two passes over its quartet list, the
    // quartets that stay FP64 then those whose recurrences run in FP32, each with a kernel
    // compiled for its precision alone (registers, hence resident warps, of its own)
    L.fp32_ok = mixed && ((ctx->opt.fp32_class_mask >> cp) & 1);
    const int gs = ctx->gs_override[cp] ? ctx->gs_override[cp] : eri_group_size(cp);
    ctx->gs_used[cp] = gs;
    const int streams = ctx->streams_override[cp];
    ctx->streams_used[cp] = gs == 32 ? eri_streams(cp, streams) : 0;
    L.chunk = gs == 1 ? 256 : 8;
    const long long items = ctx->opt.schedule == HFX_SCHED_PAIR ? (L.row_end - L.row_begin) : L.q_count;
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[2 + 2 * cp], s));
    for (int pass = 0; pass < (L.fp32_ok ? 2 : 1); ++pass) {
      const int prec = L.fp32_ok ? 1 + pass : 0;
      // the FP32 pass runs on whole warps in every class (packed FP32 recurrences after an
      // FP32 set-up), unless the caller fixed the class's group size
      const int gsp = (prec == 2 && !ctx->gs_override[cp]) ? 32 : gs;
      L.chunk = gsp == 1 ? 256 : 8;
      L.work = ctx->d_work + cp + 21 * pass;
      CK(eri_launch(L, cp, 0, grid_for(ctx, cp, 0, items, gsp, prec, false, streams), s, gsp, prec, false, streams));
    }
    if (ctx->timing) CK(cudaEventRecord(ctx->ev[3 + 2 * cp], s));
    ctx->class_launched[cp] = true;
  }
  CK(launch_finalize(n, ld, P, K, ctx->d_part, ctx->n_part, ctx->d_energy, s));
  if (ctx->timing) CK(cudaEventRecord(ctx->ev[1], s));
  return HFX_OK;
}

extern "C" int hfx_build_K_host(hfx_ctx* ctx, const double* P_host, double* K_host) {
  if (!ctx) return HFX_ERR_ARG;
  if (!P_host || !K_host) return ctx->fail(HFX_ERR_ARG, "NULL host matrix");
  const size_t bytes = sizeof(double) * (size_t)ctx->n_bf * ctx->n_bf;
  if (!ctx->d_Pst) RK(ctx->alloc(&ctx->d_Pst, (size_t)ctx->n_bf * ctx->n_bf));
  if (!ctx->d_Kst) RK(ctx->alloc(&ctx->d_Kst, (size_t)ctx->n_bf * ctx->n_bf));
  CK(cudaMemcpyAsync(ctx->d_Pst, P_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  RK(hfx_build_K(ctx, ctx->d_Pst, ctx->d_Kst, ctx->n_bf));
  CK(cudaMemcpyAsync(K_host, ctx->d_Kst, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return HFX_OK;
}

extern "C" const double* hfx_energy_device(const hfx_ctx* ctx) { return ctx ? ctx->d_energy : nullptr; }

extern "C" int hfx_energy(hfx_ctx* ctx, double* out) {
  if (!ctx || !out) return HFX_ERR_ARG;
  CK(cudaMemcpyAsync(out, ctx->d_energy, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return HFX_OK;
}

extern "C" int hfx_set_group_size(hfx_ctx* ctx, int cls, int gs) {
  if (!ctx) return HFX_ERR_ARG;
  if (cls < 0 || cls >= 21 || (gs != 0 && !eri_group_size_valid(gs)))
    return ctx->fail(HFX_ERR_ARG, "class must be 0..20 and group size 0, 1, 8, 16 or 32");
  ctx->gs_override[cls] = gs;
  return HFX_OK;
}

extern "C" int hfx_set_streams(hfx_ctx* ctx, int cls, int streams) {
  if (!ctx) return HFX_ERR_ARG;
  if (cls < 0 || cls >= 21 || streams < 0 || !eri_streams_valid(cls, streams))
    return ctx->fail(HFX_ERR_ARG, "class must be 0..20 and streams 0 or a variant the class carries");
  ctx->streams_override[cls] = streams;
  return HFX_OK;
}

extern "C" int hfx_set_timing(hfx_ctx* ctx, int enable) {
  if (!ctx) return HFX_ERR_ARG;
  ctx->timing = enable != 0;
  return HFX_OK;
}

extern "C" int hfx_get_stats(hfx_ctx* ctx, hfx_stats* out) {
  if (!ctx || !out) return HFX_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  hfx_stats& st = ctx->stats;
  for (int cp = 0; cp < 21; ++cp) {
    st.group_size_class[cp] = ctx->gs_used[cp] ? ctx->gs_used[cp] : eri_group_size(cp);
    st.streams_class[cp] = ctx->streams_used[cp];
  }
  CK(cudaMemcpy(&st.energy, ctx->d_energy, sizeof(double), cudaMemcpyDeviceToHost));
  if (ctx->timing) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]) == cudaSuccess) st.ms_build = ms;
    unsigned long long cnt[kNCnt * 21];
    CK(cudaMemcpy(cnt, ctx->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost));
    double fl = 0.0, fl32 = 0.0, flr = 0.0, nsp = 0.0;
    for (int cp = 0; cp < 21; ++cp) {
      st.ms_class[cp] = 0.0;
      if (ctx->class_launched[cp] && cudaEventElapsedTime(&ms, ctx->ev[2 + 2 * cp], ctx->ev[3 + 2 * cp]) == cudaSuccess)
        st.ms_class[cp] = ms;
      const EriClassInfo& ci = class_info_host()[cp];
      const unsigned long long* c = cnt + kNCnt * cp;
      st.prim_quartets_class[cp] = (int64_t)c[0];
      st.quartets_evaluated_class[cp] = (int64_t)c[1];
      st.quartets_fp32_class[cp] = (int64_t)c[3];
      // FP64: the set-up and the recurrences of FP64 quartets, every digest; FP32: the set-up
      // and the recurrences of FP32 quartets (the few primitive quartets whose Boys step the
      // FP32 set-up declines are set up in FP64 but counted here as FP32)
      const double su = setup_flops(ci.E, ci.F, ci.Lt, ctx->opt.omega > 0.0);
      const double f64 = (double)(c[0] - c[4]) * (su + ci.flops_prim) +
                         (double)(c[1] - c[3]) * (ci.flops_quartet - ci.flops_digest) +
                         (double)c[1] * ci.flops_digest + (double)c[2] * skip_flops();
      const double f32 = (double)c[4] * (su + ci.flops_prim) + (double)c[3] * (ci.flops_quartet - ci.flops_digest);
      st.flops_class[cp] = f64 + f32;
      fl += f64;
      fl32 += f32;
      st.flops_recurrence_class[cp] = (double)c[0] * ci.flops_prim + (double)c[1] * ci.flops_quartet;
      flr += st.flops_recurrence_class[cp];
      nsp += (double)c[0] * (ctx->opt.omega > 0.0 ? 2.0 : 1.0) + (double)c[2];
    }
    st.flops_fp64 = fl;
    st.flops_fp32 = fl32;
    st.flops_recurrence = flr;
    st.special_evals = nsp;
  }
  *out = st;
  return HFX_OK;
}

extern "C" int hfx_n_basis(const hfx_ctx* ctx) { return ctx ? ctx->n_bf : HFX_ERR_ARG; }

extern "C" int64_t hfx_device_bytes(const hfx_ctx* ctx) {
  return ctx ? (int64_t)(ctx->bytes + ctx->pair_bytes) : HFX_ERR_ARG;
}

extern "C" int64_t hfx_get_pairs(hfx_ctx* ctx, int* shell_a, int* shell_b, double* q, int64_t max_n) {
  if (!ctx) return HFX_ERR_ARG;
  if (!ctx->pairs_ready) return ctx->fail(HFX_ERR_STATE, "no pair list");
  const int n = ctx->n_kept;
  if (max_n < n || !shell_a || !shell_b || !q) return ctx->fail(HFX_ERR_ARG, "output arrays too small");
  std::vector<int> sorted(n), sa(ctx->n_cand), sb(ctx->n_cand);
  std::vector<double> Q(ctx->n_cand);
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(sorted.data(), ctx->d_sorted, sizeof(int) * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(sa.data(), ctx->d_sa, sizeof(int) * ctx->n_cand, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(sb.data(), ctx->d_sb, sizeof(int) * ctx->n_cand, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(Q.data(), ctx->d_Q, sizeof(double) * ctx->n_cand, cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) {
    shell_a[i] = sa[sorted[i]];
    shell_b[i] = sb[sorted[i]];
    q[i] = Q[sorted[i]];
  }
  return n;
}

extern "C" int hfx_get_cta_busy(hfx_ctx* ctx, double* busy_ns, int max_n) {
  if (!ctx || !busy_ns) return HFX_ERR_ARG;
  const int n = std::min(max_n, ctx->n_sm);
  std::vector<unsigned long long> b(n);
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(b.data(), ctx->d_busy, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) busy_ns[i] = (double)b[i];
  return n;
}

extern "C" const char* hfx_last_error(const hfx_ctx* ctx) {
  if (!ctx) return g_init_err.c_str();
  return ctx->err.c_str();
}

extern "C" void hfx_free(hfx_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  ctx->free_pairs();
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->ev_ok)
    for (auto& ev : ctx->ev) cudaEventDestroy(ev);
  delete ctx;
}

extern "C" int hfx_measure_fma_peak(double* fp64_tflops, double* fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) return HFX_ERR_ARG;
  cudaError_t e = fma_peak(fp64_tflops, fp32_tflops);
  if (e != cudaSuccess) {
    g_init_err = std::string("fma probe: ") + cudaGetErrorString(e);
    return HFX_ERR_CUDA;
  }
  return HFX_OK;
}


extern "C" int hfx_measure_fp64_lane_cost(double* ms_all_lanes, double* ms_one_lane) {
  if (!ms_all_lanes || !ms_one_lane) return HFX_ERR_ARG;
  cudaError_t e = fp64_lane_cost(ms_all_lanes, ms_one_lane);
  if (e != cudaSuccess) {
    g_init_err = std::string("lane probe: ") + cudaGetErrorString(e);
    return HFX_ERR_CUDA;
  }
  return HFX_OK;
}
