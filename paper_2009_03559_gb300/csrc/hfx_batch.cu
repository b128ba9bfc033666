// Batched and served K builds: the quartets of several systems go into one launch per
// angular class (hfx_batch_*), and a request loop forms such batches continuously from
// the requests waiting for the GPU (hfx_server_*, hfx_serve_*).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hfx.h"
#include "hfx_ctx.h"
#include "hfx_eri.h"
#include "hfx_internal.cuh"
#include "hfx_setup.h"

using namespace hfx;

namespace {

int class_hi(int cp) {
  int hi = 0;
  while ((hi + 1) * (hi + 2) / 2 <= cp) ++hi;
  return hi;
}

// ---------------------------------------------------------------------------
// BatchWork: the device tables of one batched build over up to `cap` systems and their
// page-locked host mirrors.  Launch records are stored [class][system] with stride cap,
// segment tables [class][cap + 1].  A build copies the mirrors to the device, zeroes K
// and takes the density-block maxima of every system, runs one dynamic-schedule launch
// per class over the concatenated quartet lists, then forms K = A + A^T and E_K.
// ---------------------------------------------------------------------------
struct BatchWork {
  int cap = 0, n = 0, n_sm = 0;
  bool mixed = false, pmax = false;
  bool fp32_class[21] = {};  // some system may run this class with FP32 recurrences
  long long total[21] = {};
  int gs[21] = {}, chunk[21] = {};  // lanes per quartet and dynamic chunk per class
  int streams[21] = {};             // warp kernel: primitive quartets at a time (0 = default)
  EriLaunch *d_launch = nullptr, *h_launch = nullptr;
  BatchSys *d_sys = nullptr, *h_sys = nullptr;
  long long *d_seg = nullptr, *h_seg = nullptr;
  unsigned long long* d_work = nullptr;
  double* d_part = nullptr;  // cap x 2 kBatchPart partial sums of E_K
  size_t bytes = 0;          // device bytes of the tables
};

void bw_free(BatchWork& w) {
  cudaFree(w.d_launch);
  cudaFree(w.d_sys);
  cudaFree(w.d_seg);
  cudaFree(w.d_work);
  cudaFree(w.d_part);
  cudaFreeHost(w.h_launch);
  cudaFreeHost(w.h_sys);
  cudaFreeHost(w.h_seg);
  w = BatchWork();
}

cudaError_t bw_alloc(BatchWork& w, int cap, int n_sm) {
  w.cap = cap;
  w.n_sm = n_sm;
  const size_t nl = 21 * (size_t)cap, ns = 21 * (size_t)(cap + 1);
  cudaError_t e;
  if ((e = cudaMalloc(&w.d_launch, sizeof(EriLaunch) * nl)) != cudaSuccess ||
      (e = cudaMalloc(&w.d_sys, sizeof(BatchSys) * cap)) != cudaSuccess ||
      (e = cudaMalloc(&w.d_seg, sizeof(long long) * ns)) != cudaSuccess ||
      (e = cudaMalloc(&w.d_work, sizeof(unsigned long long) * 64)) != cudaSuccess ||
      (e = cudaMalloc(&w.d_part, sizeof(double) * 2 * kBatchPart * cap)) != cudaSuccess ||
      (e = cudaMallocHost(&w.h_launch, sizeof(EriLaunch) * nl)) != cudaSuccess ||
      (e = cudaMallocHost(&w.h_sys, sizeof(BatchSys) * cap)) != cudaSuccess ||
      (e = cudaMallocHost(&w.h_seg, sizeof(long long) * ns)) != cudaSuccess)
    return e;
  w.bytes = sizeof(EriLaunch) * nl + sizeof(BatchSys) * cap + sizeof(long long) * ns + 256 +
            sizeof(double) * 2 * kBatchPart * cap;
  return cudaSuccess;
}

// the default per-class choices (those of a single-system build)
void bw_default_choices(BatchWork& w) {
  for (int cp = 0; cp < 21; ++cp) {
    w.gs[cp] = eri_group_size(cp);
    w.chunk[cp] = w.gs[cp] == 1 ? 256 : 8;
    w.streams[cp] = 0;
  }
}

// Fills the host mirrors for systems ctxs[0..n): launch records, segment tables and
// system records.  pmax[s], pglob[s], energy[s]: per-build scratch of system s (device).
void bw_fill(BatchWork& w, hfx_ctx* const* ctxs, int n, double* const* pmax, double* const* pglob,
             double* const* energy, bool mixed) {
  w.n = n;
  w.pmax = false;
  for (int s = 0; s < n; ++s)
    w.pmax = w.pmax || mixed || ctxs[s]->opt.skip_zero_p || ctxs[s]->opt.density_tau > 0.0;
  w.mixed = false;
  for (int cp = 0; cp < 21; ++cp) {
    w.fp32_class[cp] = false;
    for (int s = 0; s < n; ++s) w.fp32_class[cp] = w.fp32_class[cp] || (mixed && ((ctxs[s]->opt.fp32_class_mask >> cp) & 1));
    w.mixed = w.mixed || w.fp32_class[cp];
  }
  for (int cp = 0; cp < 21; ++cp) {
    long long acc = 0;
    long long* seg = w.h_seg + (size_t)cp * (w.cap + 1);
    for (int s = 0; s < n; ++s) {
      seg[s] = acc;
      acc += ctxs[s]->cls_q[cp];
    }
    for (int s = n; s <= w.cap; ++s) seg[s] = acc;
    w.total[cp] = acc;
  }
  for (int s = 0; s < n; ++s) {
    hfx_ctx* c = ctxs[s];
    const bool glob = mixed && c->opt.fp32_pmax_global;
    for (int cp = 0; cp < 21; ++cp) {
      const int hi = class_hi(cp), lo = cp - hi * (hi + 1) / 2;
      EriLaunch L = base_launch(c);
      L.ci = class_info_host()[cp];
      L.sorted = c->d_sorted;
      L.qoff = c->d_qoff;
      L.row_begin = c->rt.row_base[cp];
      L.row_end = c->rt.row_base[cp + 1];
      L.bra_bin_start = c->rt.bin_start[hi];
      L.ket_bin_start = c->rt.bin_start[lo];
      L.q_begin = c->cls_qbegin[cp];
      L.q_count = c->cls_q[cp];
      L.pmax = w.pmax ? pmax[s] : nullptr;
      L.ns = c->n_shells;
      L.skip_zero = c->opt.skip_zero_p;
      L.fp32_ok = mixed && ((c->opt.fp32_class_mask >> cp) & 1);
      L.fp32_tau = c->opt.fp32_tau;
      L.pglob = glob ? pglob[s] : nullptr;
      L.dens_tau = c->opt.density_tau;
      L.dist_tau = c->opt.dist_tau;
      L.dist = c->d_dist;
      L.Qs = c->d_Qs;
      w.h_launch[(size_t)cp * w.cap + s] = L;
    }
    BatchSys& y = w.h_sys[s];
    y.P = nullptr;
    y.K = nullptr;
    y.n = c->n_bf;
    y.ld = c->n_bf;
    y.ns = c->n_shells;
    y.bf_off = c->d_bf_off;
    y.l = c->d_l;
    y.pmax = pmax[s];
    y.energy = energy[s];
    y.part = w.d_part + (size_t)s * 2 * kBatchPart;
    y.pglob = glob ? pglob[s] : nullptr;
  }
}

// P/K/ld of every system in the host mirrors
void bw_set_buffers(BatchWork& w, const double* const* P, double* const* K, const int* ld) {
  for (int s = 0; s < w.n; ++s) {
    BatchSys& y = w.h_sys[s];
    y.P = P[s];
    y.K = K[s];
    y.ld = ld ? ld[s] : y.n;
    for (int cp = 0; cp < 21; ++cp) {
      EriLaunch& L = w.h_launch[(size_t)cp * w.cap + s];
      L.P = P[s];
      L.K = K[s];
      L.ld = y.ld;
    }
  }
}

// launch record of class cp, precision pass `pass` (0, or 0/1 for a mixed class's FP64/FP32
// passes: each has its own work counter)
int bw_prec(const BatchWork& w, int cp, int pass) { return w.fp32_class[cp] ? 1 + pass : 0; }

// lanes per quartet of a pass: the class's choice, except the FP32 pass, which runs on whole
// warps in every class (packed FP32 recurrences after an FP32 set-up)
int bw_gs(const BatchWork& w, int cp, int prec) { return prec == 2 ? 32 : w.gs[cp]; }

EriLaunch bw_class_launch(const BatchWork& w, int cp, int pass = 0) {
  EriLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.ci = class_info_host()[cp];
  L.schedule = HFX_SCHED_DYNAMIC;
  L.q_count = w.total[cp];
  L.work = w.d_work + cp + 21 * pass;
  L.chunk = bw_gs(w, cp, bw_prec(w, cp, pass)) == w.gs[cp] ? w.chunk[cp] : 8;
  L.n_sys = w.n;
  L.seg = w.d_seg + (size_t)cp * (w.cap + 1);
  L.batch = w.d_launch + (size_t)cp * w.cap;
  return L;
}

int bw_grid(const BatchWork& w, int cp, long long items, int prec) {
  const int gs = bw_gs(w, cp, prec);
  const long long groups_per_block = eri_groups_per_block(gs);
  const long long need = (items + groups_per_block - 1) / groups_per_block;
  const long long cap = (long long)eri_blocks_per_sm(cp, 0, gs, prec, true, w.streams[cp]) * w.n_sm;
  return (int)std::max(1LL, std::min(need, cap));
}

cudaError_t bw_upload(const BatchWork& w, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemcpyAsync(w.d_launch, w.h_launch, sizeof(EriLaunch) * 21 * (size_t)w.cap, cudaMemcpyHostToDevice,
                           s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(w.d_sys, w.h_sys, sizeof(BatchSys) * w.n, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(w.d_seg, w.h_seg, sizeof(long long) * 21 * (size_t)(w.cap + 1), cudaMemcpyHostToDevice,
                           s)) != cudaSuccess)
    return e;
  return cudaSuccess;
}

// Parallel branches of a batched build: the class launches are spread over the main
// stream and up to kBranches - 1 more, so that the tail of one class (its last chunks,
// when most SMs are idle) overlaps the next classes.  Inside a graph capture the forks
// and joins become edges of the graph.
constexpr int kBranches = 4;
struct Branches {
  cudaStream_t aux[kBranches - 1] = {};
  cudaEvent_t fork = nullptr, join[kBranches - 1] = {};
  int n = 1;  // branches in use (1: everything on the main stream)
};

// the whole batched build on stream s (and the branches' streams, if any)
cudaError_t bw_enqueue(const BatchWork& w, cudaStream_t s, const Branches* br = nullptr) {
  cudaError_t e;
  if ((e = bw_upload(w, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(w.d_work, 0, 64 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
  if ((e = launch_batch_prologue(w.d_sys, w.n, w.n_sm, w.pmax, s)) != cudaSuccess) return e;
  const int nb = br ? br->n : 1;
  // classes by estimated cost (quartets x FP64 flops of a quartet with 81 primitive
  // quartets), each to the branch with the least cost so far
  int order[21];
  double cost[21];
  for (int cp = 0; cp < 21; ++cp) {
    const EriClassInfo& ci = class_info_host()[cp];
    order[cp] = cp;
    cost[cp] = (double)w.total[cp] * (81.0 * ci.flops_prim + ci.flops_quartet);
  }
  std::sort(order, order + 21, [&](int a, int b) { return cost[a] > cost[b]; });
  double load[kBranches] = {};
  if (nb > 1) {
    if ((e = cudaEventRecord(br->fork, s)) != cudaSuccess) return e;
    for (int i = 0; i < nb - 1; ++i)
      if ((e = cudaStreamWaitEvent(br->aux[i], br->fork, 0)) != cudaSuccess) return e;
  }
  for (int oi = 0; oi < 21; ++oi) {
    const int cp = order[oi];
    if (w.total[cp] == 0) continue;
    int bi = 0;
    for (int i = 1; i < nb; ++i)
      if (load[i] < load[bi]) bi = i;
    load[bi] += cost[cp];
    cudaStream_t bs = bi == 0 ? s : br->aux[bi - 1];
    for (int pass = 0; pass < (w.fp32_class[cp] ? 2 : 1); ++pass) {
      const EriLaunch L = bw_class_launch(w, cp, pass);
      const int prec = bw_prec(w, cp, pass);
      e = eri_launch(L, cp, 0, bw_grid(w, cp, w.total[cp], prec), bs, bw_gs(w, cp, prec), prec, true, w.streams[cp]);
      if (e != cudaSuccess) return e;
    }
  }
  if (nb > 1) {
    for (int i = 0; i < nb - 1; ++i) {
      if ((e = cudaEventRecord(br->join[i], br->aux[i])) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(s, br->join[i], 0)) != cudaSuccess) return e;
    }
  }
  return launch_batch_epilogue(w.d_sys, w.n, w.n_sm, s);
}

double host_ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

// ===========================================================================
// hfx_batch: one fixed set of systems, captured once as a CUDA graph
// ===========================================================================
struct hfx_batch {
  std::vector<hfx_ctx*> ctx;
  cudaStream_t user = nullptr;    // the caller's stream (may be the legacy default stream)
  cudaStream_t stream = nullptr;  // the batch's own stream: graphs are captured and run here
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  BatchWork w;
  bool use_graph = true;
  double tune_ms[21] = {};
  long long tune_window[21] = {};
  double tune_full_default_ms = 0.0, tune_full_tuned_ms = 0.0;
  int tune_kept = 0;
  Branches br;
  float tune_target_ms = 20.f;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ran = false;
  std::string err;
  int fail(int code, const std::string& m) {
    err = m;
    hfx::set_global_error(m);
    return code;
  }
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
};

#define CKB(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return b->fail(HFX_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

extern "C" void hfx_batch_free(hfx_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  b->drop_graph();
  bw_free(b->w);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (int i = 0; i < kBranches - 1; ++i) {
    if (b->br.aux[i]) cudaStreamDestroy(b->br.aux[i]);
    if (b->br.join[i]) cudaEventDestroy(b->br.join[i]);
  }
  if (b->br.fork) cudaEventDestroy(b->br.fork);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

extern "C" int hfx_batch_create(hfx_batch** out, hfx_ctx* const* ctxs, int n, void* stream) {
  if (!out || !ctxs || n <= 0) {
    hfx::set_global_error("hfx_batch_create: NULL argument or n <= 0");
    return HFX_ERR_ARG;
  }
  *out = nullptr;
  for (int s = 0; s < n; ++s)
    if (!ctxs[s] || !ctxs[s]->pairs_ready) {
      hfx::set_global_error("hfx_batch_create: context " + std::to_string(s) + " has no pair list");
      return HFX_ERR_STATE;
    }
  hfx_batch* b = new hfx_batch();
  b->ctx.assign(ctxs, ctxs + n);
  b->user = stream ? (cudaStream_t)stream : ctxs[0]->stream;
  cudaError_t e;
  if ((e = bw_alloc(b->w, n, ctxs[0]->n_sm)) != cudaSuccess || (e = cudaEventCreate(&b->e0)) != cudaSuccess ||
      (e = cudaEventCreate(&b->e1)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->br.fork, cudaEventDisableTiming)) != cudaSuccess) {
    hfx::set_global_error(std::string("hfx_batch_create: ") + cudaGetErrorString(e));
    hfx_batch_free(b);
    return e == cudaErrorMemoryAllocation ? HFX_ERR_OOM : HFX_ERR_CUDA;
  }
  for (int i = 0; i < kBranches - 1; ++i) {
    if ((e = cudaStreamCreateWithFlags(&b->br.aux[i], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->br.join[i], cudaEventDisableTiming)) != cudaSuccess) {
      hfx::set_global_error(std::string("hfx_batch_create: ") + cudaGetErrorString(e));
      hfx_batch_free(b);
      return HFX_ERR_CUDA;
    }
  }
  b->br.n = 1;  // measured faster on the 32-system mix; the tuner also tries kBranches
  // per-build scratch: each context's own (a context belongs to one batch build at a time)
  std::vector<double*> pmax(n), pglob(n), energy(n);
  for (int s = 0; s < n; ++s) {
    pmax[s] = ctxs[s]->d_pmax;
    pglob[s] = ctxs[s]->d_pglob;
    energy[s] = ctxs[s]->d_energy;
  }
  bw_fill(b->w, ctxs, n, pmax.data(), pglob.data(), energy.data(), ctxs[0]->opt.precision == HFX_MIXED);
  bw_default_choices(b->w);
  *out = b;
  return HFX_OK;
}

static int batch_check_args(hfx_batch* b, const double* const* P, double* const* K, const int* ld) {
  for (int s = 0; s < b->w.n; ++s)
    if (!P[s] || !K[s] || (ld && ld[s] < b->ctx[s]->n_bf))
      return b->fail(HFX_ERR_ARG, "NULL matrix or ld < n_bf for system " + std::to_string(s));
  return HFX_OK;
}

extern "C" int hfx_batch_set_tune_target(hfx_batch* b, double ms) {
  if (!b || !(ms > 0.0) || ms > 1e4) return HFX_ERR_ARG;
  b->tune_target_ms = (float)ms;
  return HFX_OK;
}

extern "C" int hfx_batch_set_branches(hfx_batch* b, int n) {
  if (!b || n < 1 || n > kBranches) return HFX_ERR_ARG;
  b->br.n = n;
  b->drop_graph();  // a captured graph holds the previous branches
  return HFX_OK;
}

extern "C" int hfx_batch_set_graph(hfx_batch* b, int enable) {
  if (!b) return HFX_ERR_ARG;
  b->use_graph = enable != 0;
  return HFX_OK;
}

extern "C" int hfx_batch_run(hfx_batch* b, const double* const* P, double* const* K, const int* ld) {
  if (!b || !P || !K) return HFX_ERR_ARG;
  if (int r = batch_check_args(b, P, K, ld)) return r;
  // the mirrors may still be read by a previous run's copies: wait before rewriting
  if (b->ran) CKB(cudaStreamSynchronize(b->stream));
  bw_set_buffers(b->w, P, K, ld);
  cudaStream_t s = b->stream;
  CKB(cudaEventRecord(b->ev_in, b->user));  // the inputs are ready on the caller's stream
  CKB(cudaStreamWaitEvent(s, b->ev_in, 0));
  CKB(cudaEventRecord(b->e0, s));
  if (b->use_graph) {
    if (!b->exec) {
      CKB(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      const cudaError_t r = bw_enqueue(b->w, s, &b->br);
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(s, &g);
      if (r != cudaSuccess || ec != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return b->fail(HFX_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(r != cudaSuccess ? r : ec));
      }
      b->graph = g;
      CKB(cudaGraphInstantiate(&b->exec, g, 0));
    }
    CKB(cudaGraphLaunch(b->exec, s));
  } else {
    CKB(bw_enqueue(b->w, s, &b->br));
  }
  CKB(cudaEventRecord(b->e1, s));
  CKB(cudaEventRecord(b->ev_out, s));  // later work on the caller's stream sees K and E_K
  CKB(cudaStreamWaitEvent(b->user, b->ev_out, 0));
  b->ran = true;
  return HFX_OK;
}

extern "C" int hfx_batch_tune(hfx_batch* b, const double* const* P, double* const* K, const int* ld) {
  if (!b || !P || !K) return HFX_ERR_ARG;
  if (int r = batch_check_args(b, P, K, ld)) return r;
  if (b->ran) CKB(cudaStreamSynchronize(b->stream));
  CKB(cudaStreamSynchronize(b->user));
  BatchWork& w = b->w;
  bw_set_buffers(w, P, K, ld);
  cudaStream_t s = b->stream;
  cudaEvent_t t0, t1;
  CKB(cudaEventCreate(&t0));
  CKB(cudaEventCreate(&t1));
  struct Choice {
    int gs[21], chunk[21], streams[21];
  };
  auto save = [&]() {
    Choice c;
    std::memcpy(c.gs, w.gs, sizeof(c.gs));
    std::memcpy(c.chunk, w.chunk, sizeof(c.chunk));
    std::memcpy(c.streams, w.streams, sizeof(c.streams));
    return c;
  };
  auto restore = [&](const Choice& c) {
    std::memcpy(w.gs, c.gs, sizeof(c.gs));
    std::memcpy(w.chunk, c.chunk, sizeof(c.chunk));
    std::memcpy(w.streams, c.streams, sizeof(c.streams));
  };
  // the whole batched build with the current choices (plain launches on the branches)
  auto time_full = [&](double* ms_out) -> int {
    float ms = 0.f;
    CKB(cudaEventRecord(t0, s));
    CKB(bw_enqueue(w, s, &b->br));
    CKB(cudaEventRecord(t1, s));
    CKB(cudaEventSynchronize(t1));
    CKB(cudaEventElapsedTime(&ms, t0, t1));
    *ms_out = ms;
    return HFX_OK;
  };
  // Each candidate of a class runs on one window of the class's concatenated quartet list
  // (from its middle), sized so that a launch takes about tune_target_ms: the work counters
  // start at the window's first index and the launches stop at its end.
  auto time_window = [&](int cp, long long w0, long long w1, float* ms_out) -> int {
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first repetition warms caches; keep the second
      const unsigned long long start[2] = {(unsigned long long)w0, (unsigned long long)w0};
      CKB(cudaMemcpyAsync(w.d_work + cp, &start[0], sizeof(start[0]), cudaMemcpyHostToDevice, s));
      CKB(cudaMemcpyAsync(w.d_work + cp + 21, &start[1], sizeof(start[1]), cudaMemcpyHostToDevice, s));
      CKB(cudaEventRecord(t0, s));
      for (int pass = 0; pass < (w.fp32_class[cp] ? 2 : 1); ++pass) {
        EriLaunch L = bw_class_launch(w, cp, pass);
        L.q_count = w1;
        const int prec = bw_prec(w, cp, pass);
        CKB(eri_launch(L, cp, 0, bw_grid(w, cp, w1 - w0, prec), s, bw_gs(w, cp, prec), prec, true, w.streams[cp]));
      }
      CKB(cudaEventRecord(t1, s));
      CKB(cudaEventSynchronize(t1));
      CKB(cudaEventElapsedTime(&ms, t0, t1));
    }
    *ms_out = ms;
    return HFX_OK;
  };
  int rc = HFX_OK;
  const Choice incumbent = save();
  double full_inc = 0.0, full_new = 0.0;
  if ((rc = time_full(&full_inc)) != HFX_OK) return rc;
  CKB(bw_upload(w, s));
  CKB(launch_batch_prologue(w.d_sys, w.n, w.n_sm, w.pmax, s));
  for (int cp = 0; cp < 21 && rc == HFX_OK; ++cp) {
    const long long total = w.total[cp];
    if (total == 0) continue;
    struct Cand {
      int gs, streams, chunk;
    };
    std::vector<Cand> cands;
    for (int k : {1, 2, 4})
      if (eri_streams_valid(cp, k))
        for (int c : {4, 8, 16}) cands.push_back({32, k, c});
    if (eri_group_size(cp) == 1)
      for (int c : {128, 256, 512}) cands.push_back({1, 0, c});
    // window size: grow from 16k quartets until the incumbent takes the target, and at
    // least two claims for every resident warp of every candidate, so that a large chunk
    // is not timed on a window that leaves most of the GPU idle
    long long fill = 0;
    for (const Cand& cd : cands) {
      const long long groups = (long long)eri_blocks_per_sm(cp, 0, cd.gs, bw_prec(w, cp, 0), true, cd.streams) *
                               w.n_sm * (eri_block_size() / 32);
      fill = std::max(fill, 2 * groups * cd.chunk);
    }
    long long win = std::min(total, std::max(16384LL, fill));
    for (int it = 0; it < 4 && win < total && rc == HFX_OK; ++it) {
      float ms = 0.f;
      const long long w0 = (total - win) / 2;
      if ((rc = time_window(cp, w0, w0 + win, &ms)) != HFX_OK) break;
      if (ms >= 0.5f * b->tune_target_ms) break;
      const double grow = ms > 0.f ? b->tune_target_ms / ms : 64.0;
      win = std::min(total, (long long)(win * std::min(64.0, std::max(2.0, grow))));
    }
    if (rc != HFX_OK) break;
    const long long w0 = (total - win) / 2;
    // the current choice is the incumbent; a candidate must beat it by 5% to replace it
    Cand bc = {w.gs[cp], w.streams[cp], w.chunk[cp]};
    float inc = 0.f;
    if ((rc = time_window(cp, w0, w0 + win, &inc)) != HFX_OK) break;
    double best = inc;
    for (const Cand& cd : cands) {
      if (rc != HFX_OK) break;
      if (cd.gs == bc.gs && cd.chunk == bc.chunk && eri_streams(cp, cd.streams) == eri_streams(cp, bc.streams))
        continue;
      w.gs[cp] = cd.gs;
      w.streams[cp] = cd.streams;
      w.chunk[cp] = cd.chunk;
      float ms = 0.f;
      if ((rc = time_window(cp, w0, w0 + win, &ms)) != HFX_OK) break;
      if (ms < best && ms < 0.95 * inc) {
        best = ms;
        bc = cd;
      }
    }
    w.gs[cp] = bc.gs;
    w.streams[cp] = bc.streams;
    w.chunk[cp] = bc.chunk;
    b->tune_ms[cp] = best * (double)total / (double)win;  // projected to the whole class
    b->tune_window[cp] = win;
  }
  // the tuned choices replace the incumbent only if the whole batch runs faster with them;
  // the number of parallel branches is chosen the same way (the incumbent's, or 1 or all)
  const int br_inc = b->br.n;
  int br_best = br_inc;
  if (rc == HFX_OK) rc = time_full(&full_new);
  for (int nb : {1, kBranches}) {
    if (rc != HFX_OK || nb == br_inc) continue;
    b->br.n = nb;
    double ms = 0.0;
    if ((rc = time_full(&ms)) == HFX_OK && ms < full_new) {
      full_new = ms;
      br_best = nb;
    }
  }
  if (rc == HFX_OK) {
    b->tune_full_default_ms = full_inc;
    b->tune_full_tuned_ms = full_new;
    b->tune_kept = full_new < full_inc;
    b->br.n = b->tune_kept ? br_best : br_inc;
    if (!b->tune_kept) restore(incumbent);
  } else {
    b->br.n = br_inc;
    restore(incumbent);
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (rc != HFX_OK) return rc;
  b->drop_graph();  // a captured graph holds the previous choices
  CKB(cudaStreamSynchronize(s));
  return HFX_OK;
}

extern "C" int hfx_batch_get_stats(hfx_batch* b, hfx_batch_stats* out) {
  if (!b || !out) return HFX_ERR_ARG;
  CKB(cudaStreamSynchronize(b->stream));
  std::memset(out, 0, sizeof(*out));
  for (int cp = 0; cp < 21; ++cp) {
    out->n_quartets += b->w.total[cp];
    out->group_size_class[cp] = b->w.gs[cp];
    out->chunk_class[cp] = b->w.chunk[cp];
    out->streams_class[cp] = b->w.gs[cp] == 32 ? eri_streams(cp, b->w.streams[cp]) : 0;
    out->tune_ms_class[cp] = b->tune_ms[cp];
    out->tune_window_class[cp] = b->tune_window[cp];
  }
  out->tune_full_default_ms = b->tune_full_default_ms;
  out->tune_full_tuned_ms = b->tune_full_tuned_ms;
  out->tune_kept = b->tune_kept;
  out->branches = b->br.n;
  float ms = 0.f;
  if (b->ran && cudaEventElapsedTime(&ms, b->e0, b->e1) == cudaSuccess) out->ms_last = ms;
  return HFX_OK;
}

extern "C" int hfx_build_K_batched(hfx_ctx* const* ctxs, const double* const* P, double* const* K, const int* ld,
                                   int n) {
  hfx_batch* b = nullptr;
  int r = hfx_batch_create(&b, ctxs, n, nullptr);
  if (r != HFX_OK) return r;
  hfx_batch_set_graph(b, 0);
  r = hfx_batch_run(b, P, K, ld);
  if (r == HFX_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) r = HFX_ERR_CUDA;
  hfx_batch_free(b);
  return r;
}

// ===========================================================================
// hfx_server: continuous batching over registered systems
// ===========================================================================
namespace {

struct Request {
  uint64_t ticket = 0;
  int sys = 0;
  const double* P_src = nullptr;
  double* K_dst = nullptr;
  cudaEvent_t ready = nullptr;  // P is ready (recorded on the submitter's stream)
  int status = HFX_REQ_QUEUED;
  int step_size = 0;
  size_t bytes = 0;
  char* mem = nullptr;  // server-owned P | K | pmax | pglob
  double energy = 0.0, t_submit = 0.0, t_admit = 0.0, t_done = 0.0, ms_step = 0.0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;
  BatchWork w;
  double* d_energy = nullptr;  // cap
  double* h_energy = nullptr;  // cap, page-locked
  std::vector<uint64_t> reqs;
  bool busy = false;
};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct hfx_server {
  std::mutex mu;
  hfx_server_options opt{};
  int n_sm = 0;
  std::vector<hfx_ctx*> systems;
  std::vector<long long> sys_quartets;
  std::vector<Slot> slots;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<cudaEvent_t> event_pool;
  uint64_t next_ticket = 1;
  size_t budget = 0, bytes_resident = 0, bytes_requests = 0, bytes_peak = 0;
  cudaMemPool_t pool = nullptr;
  cudaEvent_t epoch = nullptr;
  std::chrono::steady_clock::time_point t0;
  double epoch_host_ms = 0.0;
  hfx_server_stats st{};
  std::string err;
  int fail(int code, const std::string& m) {
    err = m;
    hfx::set_global_error(m);
    return code;
  }
};

#define CKS(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return srv->fail(HFX_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

extern "C" void hfx_server_default_options(hfx_server_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->hbm_budget_gb = 120.0;
  opt->max_step_quartets = 1e7;
  opt->max_inflight = 4;
  opt->max_batch = 16;
  opt->precision = HFX_FP64;
}

extern "C" void hfx_server_free(hfx_server* srv) {
  if (!srv) return;
  for (Slot& sl : srv->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    bw_free(sl.w);
    cudaFree(sl.d_energy);
    cudaFreeHost(sl.h_energy);
    if (sl.start) cudaEventDestroy(sl.start);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  for (auto& kv : srv->reqs)
    if (kv.second.ready) cudaEventDestroy(kv.second.ready);
  for (cudaEvent_t e : srv->event_pool) cudaEventDestroy(e);
  if (srv->epoch) cudaEventDestroy(srv->epoch);
  if (srv->pool) cudaMemPoolDestroy(srv->pool);
  delete srv;
}

extern "C" int hfx_server_create(hfx_server** out, const hfx_server_options* opt) {
  if (!out) return HFX_ERR_ARG;
  *out = nullptr;
  hfx_server_options o;
  hfx_server_default_options(&o);
  if (opt) o = *opt;
  if (!(o.hbm_budget_gb > 0.0) || !(o.max_step_quartets >= 0.0) || o.max_inflight < 1 || o.max_inflight > 64 || o.max_batch < 1 ||
      o.max_batch > 1024 || (o.precision != HFX_FP64 && o.precision != HFX_MIXED)) {
    hfx::set_global_error("hfx_server_create: invalid options");
    return HFX_ERR_ARG;
  }
  hfx_server* srv = new hfx_server();
  srv->opt = o;
  srv->budget = (size_t)(o.hbm_budget_gb * 1e9);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&srv->n_sm, cudaDevAttrMultiProcessorCount, dev);
  // a memory pool of the server's own: stream-ordered allocation without device-wide
  // synchronisation, memory kept in the pool up to the budget between steps
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  if (e == cudaSuccess) e = cudaMemPoolCreate(&srv->pool, &props);
  if (e == cudaSuccess) {
    uint64_t keep = srv->budget;
    e = cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  // Memory freed at the end of a step on one slot's stream must not be handed to a step on
  // another slot by making that stream wait for the first: that would chain the slots.
  // Reuse only what is known to be free (stream order or completed events).
  int no = 0;
  if (e == cudaSuccess) e = cudaMemPoolSetAttribute(srv->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  if (e == cudaSuccess) e = cudaMemPoolSetAttribute(srv->pool, cudaMemPoolReuseAllowOpportunistic, &no);
  srv->slots.resize(o.max_inflight);
  for (Slot& sl : srv->slots) {
    if (e != cudaSuccess) break;
    if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&sl.start)) != cudaSuccess || (e = cudaEventCreate(&sl.done)) != cudaSuccess ||
        (e = bw_alloc(sl.w, o.max_batch, srv->n_sm)) != cudaSuccess ||
        (e = cudaMalloc(&sl.d_energy, sizeof(double) * o.max_batch)) != cudaSuccess ||
        (e = cudaMallocHost(&sl.h_energy, sizeof(double) * o.max_batch)) != cudaSuccess)
      break;
    srv->bytes_resident += sl.w.bytes + sizeof(double) * o.max_batch;
  }
  if (e == cudaSuccess) e = cudaEventCreate(&srv->epoch);
  if (e == cudaSuccess) e = cudaEventRecord(srv->epoch, srv->slots[0].stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(srv->epoch);
  if (e != cudaSuccess) {
    hfx::set_global_error(std::string("hfx_server_create: ") + cudaGetErrorString(e));
    hfx_server_free(srv);
    return e == cudaErrorMemoryAllocation ? HFX_ERR_OOM : HFX_ERR_CUDA;
  }
  srv->t0 = std::chrono::steady_clock::now();  // host time of the epoch event (just completed)
  if (srv->bytes_resident > srv->budget) {
    hfx::set_global_error("hfx_server_create: the step workspaces alone exceed the memory budget");
    hfx_server_free(srv);
    return HFX_ERR_ADMISSION;
  }
  srv->bytes_peak = srv->bytes_resident;
  *out = srv;
  return HFX_OK;
}

extern "C" int hfx_server_add_system(hfx_server* srv, hfx_ctx* ctx, int* id) {
  if (!srv || !ctx || !id) return HFX_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (!ctx->pairs_ready) return srv->fail(HFX_ERR_STATE, "hfx_server_add_system: context has no pair list");
  const size_t b = ctx->bytes + ctx->pair_bytes;
  if (srv->bytes_resident + srv->bytes_requests + b > srv->budget)
    return srv->fail(HFX_ERR_ADMISSION, "hfx_server_add_system: the system does not fit the memory budget");
  CKS(cudaStreamSynchronize(ctx->stream));
  long long q = 0;
  for (int cp = 0; cp < 21; ++cp) q += ctx->cls_q[cp];
  *id = (int)srv->systems.size();
  srv->systems.push_back(ctx);
  srv->sys_quartets.push_back(q);
  srv->bytes_resident += b;
  srv->bytes_peak = std::max(srv->bytes_peak, srv->bytes_resident + srv->bytes_requests);
  return HFX_OK;
}

static size_t request_bytes(const hfx_ctx* c) {
  const size_t nn = (size_t)c->n_bf * c->n_bf, ss = (size_t)c->n_shells * c->n_shells;
  return 2 * align_up(nn * sizeof(double)) + align_up(ss * sizeof(double)) + 256;
}

// device pointer or page-locked host pointer
static bool servable_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged;
}

// Retires finished steps: results, memory accounting, slots.
static int server_retire(hfx_server* srv) {
  for (Slot& sl : srv->slots) {
    if (!sl.busy) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    float ms_epoch = 0.f, ms_step = 0.f;
    cudaError_t e = q;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_epoch, srv->epoch, sl.done);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_step, sl.start, sl.done);
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
      Request& r = srv->reqs[sl.reqs[i]];
      srv->bytes_requests -= r.bytes;
      r.mem = nullptr;
      if (e == cudaSuccess) {
        r.status = HFX_REQ_DONE;
        r.energy = sl.h_energy[i];
        r.t_done = srv->epoch_host_ms + ms_epoch;
        r.ms_step = ms_step;
        srv->st.n_done++;
        srv->st.quartets_done += srv->sys_quartets[r.sys];
      } else {
        r.status = HFX_ERR_CUDA;
        srv->st.n_failed++;
      }
    }
    sl.reqs.clear();
    sl.busy = false;
    if (e != cudaSuccess) {
      cudaGetLastError();
      return srv->fail(HFX_ERR_CUDA, std::string("server step failed: ") + cudaGetErrorString(e));
    }
  }
  return HFX_OK;
}

// Enqueues one step for the requests `take` on the slot's stream: server-owned P/K/maxima
// from the pool, P copied in after the submitter's stream, the batched build, K copied
// out, memory given back, E_K of every request to the slot's host array, the done event.
static cudaError_t step_enqueue(hfx_server* srv, Slot& sl, const std::vector<uint64_t>& take) {
  cudaStream_t s = sl.stream;
  const int n = (int)take.size();
  std::vector<hfx_ctx*> ctxs(n);
  std::vector<const double*> P(n);
  std::vector<double*> K(n), pmax(n), pglob(n), energy(n);
  cudaError_t e;
  if ((e = cudaEventRecord(sl.start, s)) != cudaSuccess) return e;
  for (int i = 0; i < n; ++i) {
    Request& r = srv->reqs[take[i]];
    hfx_ctx* c = srv->systems[r.sys];
    const size_t nn = (size_t)c->n_bf * c->n_bf;
    void* m = nullptr;
    if ((e = cudaMallocFromPoolAsync(&m, r.bytes, srv->pool, s)) != cudaSuccess) return e;
    r.mem = (char*)m;
    double* Pd = (double*)r.mem;
    if ((e = cudaStreamWaitEvent(s, r.ready, 0)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(Pd, r.P_src, nn * sizeof(double), cudaMemcpyDefault, s)) != cudaSuccess) return e;
    ctxs[i] = c;
    P[i] = Pd;
    K[i] = (double*)(r.mem + align_up(nn * sizeof(double)));
    pmax[i] = (double*)(r.mem + 2 * align_up(nn * sizeof(double)));
    pglob[i] = (double*)(r.mem + r.bytes - 256);
    energy[i] = sl.d_energy + i;
  }
  bw_fill(sl.w, ctxs.data(), n, pmax.data(), pglob.data(), energy.data(), srv->opt.precision == HFX_MIXED);
  bw_default_choices(sl.w);
  bw_set_buffers(sl.w, P.data(), K.data(), nullptr);
  if ((e = bw_enqueue(sl.w, s)) != cudaSuccess) return e;
  for (int i = 0; i < n; ++i) {
    Request& r = srv->reqs[take[i]];
    const size_t nn = (size_t)ctxs[i]->n_bf * ctxs[i]->n_bf;
    if ((e = cudaMemcpyAsync(r.K_dst, K[i], nn * sizeof(double), cudaMemcpyDefault, s)) != cudaSuccess) return e;
    if ((e = cudaFreeAsync(r.mem, s)) != cudaSuccess) return e;
    r.mem = nullptr;  // given back in stream order
  }
  if ((e = cudaMemcpyAsync(sl.h_energy, sl.d_energy, sizeof(double) * n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  return cudaEventRecord(sl.done, s);
}

// Starts one step on a free slot with the queued requests that fit; false if none started.
static int server_launch_step(hfx_server* srv, Slot& sl, bool* started) {
  *started = false;
  std::vector<uint64_t> take;
  size_t add = 0;
  double step_q = 0.0;
  while (!srv->queue.empty() && (int)take.size() < srv->opt.max_batch) {
    const Request& r = srv->reqs[srv->queue.front()];
    if (srv->bytes_resident + srv->bytes_requests + add + r.bytes > srv->budget) break;  // FIFO: wait
    const double q = (double)srv->sys_quartets[r.sys];
    if (!take.empty() && step_q + q > srv->opt.max_step_quartets) break;
    step_q += q;
    add += r.bytes;
    take.push_back(srv->queue.front());
    srv->queue.pop_front();
  }
  if (take.empty()) return HFX_OK;
  const double now = host_ms_since(srv->t0);
  const cudaError_t e = step_enqueue(srv, sl, take);
  if (e != cudaSuccess) {
    // the step's requests fail (their waits return); memory already taken is given back
    for (uint64_t t : take) {
      Request& r = srv->reqs[t];
      if (r.mem) cudaFreeAsync(r.mem, sl.stream);
      r.mem = nullptr;
      r.status = HFX_ERR_CUDA;
      srv->st.n_failed++;
    }
    cudaGetLastError();
    return srv->fail(HFX_ERR_CUDA, std::string("server step launch failed: ") + cudaGetErrorString(e));
  }
  for (uint64_t t : take) {
    Request& r = srv->reqs[t];
    r.status = HFX_REQ_RUNNING;
    r.step_size = (int)take.size();
    r.t_admit = now;
  }
  const int n = (int)take.size();
  sl.reqs = take;
  sl.busy = true;
  srv->bytes_requests += add;
  srv->bytes_peak = std::max(srv->bytes_peak, srv->bytes_resident + srv->bytes_requests);
  srv->st.n_steps++;
  srv->st.max_step_size = std::max(srv->st.max_step_size, n);
  int inflight = 0;
  for (const Slot& x : srv->slots) inflight += x.busy;
  srv->st.max_steps_inflight = std::max(srv->st.max_steps_inflight, inflight);
  *started = true;
  return HFX_OK;
}

static int server_progress_locked(hfx_server* srv) {
  if (int r = server_retire(srv)) return r;
  for (Slot& sl : srv->slots) {
    if (srv->queue.empty()) break;
    if (sl.busy) continue;
    bool started = false;
    if (int r = server_launch_step(srv, sl, &started)) return r;
    if (!started) break;  // the queue head waits for memory
  }
  return HFX_OK;
}

static int server_pending(const hfx_server* srv) {
  int n = (int)srv->queue.size();
  for (const Slot& sl : srv->slots) n += (int)sl.reqs.size();
  return n;
}

extern "C" int hfx_serve_submit(hfx_server* srv, int id, const double* P, double* K_out, void* stream,
                                uint64_t* ticket) {
  if (!srv || !P || !K_out || !ticket) return HFX_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (id < 0 || id >= (int)srv->systems.size()) return srv->fail(HFX_ERR_ARG, "hfx_serve_submit: unknown system");
  if (!servable_pointer(P) || !servable_pointer(K_out))
    return srv->fail(HFX_ERR_ARG, "hfx_serve_submit: P and K_out must be device or page-locked host memory");
  Request r;
  r.ticket = srv->next_ticket++;
  r.sys = id;
  r.P_src = P;
  r.K_dst = K_out;
  r.bytes = request_bytes(srv->systems[id]);
  if (srv->bytes_resident + r.bytes > srv->budget)
    return srv->fail(HFX_ERR_ADMISSION, "hfx_serve_submit: the request can never fit the memory budget");
  if (!srv->event_pool.empty()) {
    r.ready = srv->event_pool.back();
    srv->event_pool.pop_back();
  } else {
    CKS(cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming));
  }
  CKS(cudaEventRecord(r.ready, (cudaStream_t)stream));
  r.t_submit = host_ms_since(srv->t0);
  *ticket = r.ticket;
  srv->queue.push_back(r.ticket);
  srv->reqs.emplace(r.ticket, r);
  srv->st.n_submitted++;
  return server_progress_locked(srv);
}

static void fill_result(const hfx_server* srv, const Request& r, hfx_result* out) {
  std::memset(out, 0, sizeof(*out));
  out->ticket = r.ticket;
  out->status = r.status;
  out->system_id = r.sys;
  out->step_size = r.step_size;
  out->energy = r.energy;
  out->t_submit_ms = r.t_submit;
  out->t_admit_ms = r.t_admit;
  out->t_done_ms = r.t_done;
  out->ms_step = r.ms_step;
  out->n_quartets = srv->sys_quartets[r.sys];
}

// a finished request gives its event back to the pool
static void recycle_event(hfx_server* srv, Request& r) {
  if (r.status != HFX_REQ_QUEUED && r.status != HFX_REQ_RUNNING && r.ready) {
    srv->event_pool.push_back(r.ready);
    r.ready = nullptr;
  }
}

extern "C" int hfx_serve_poll(hfx_server* srv, uint64_t ticket, hfx_result* out) {
  if (!srv || !out) return HFX_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return srv->fail(HFX_ERR_ARG, "hfx_serve_poll: unknown ticket");
  const int r = server_progress_locked(srv);
  recycle_event(srv, it->second);
  fill_result(srv, it->second, out);
  return r;
}

extern "C" int hfx_serve_release(hfx_server* srv, uint64_t ticket) {
  if (!srv) return HFX_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return srv->fail(HFX_ERR_ARG, "hfx_serve_release: unknown ticket");
  Request& r = it->second;
  if (r.status == HFX_REQ_QUEUED || r.status == HFX_REQ_RUNNING)
    return srv->fail(HFX_ERR_STATE, "hfx_serve_release: the request is not finished");
  recycle_event(srv, r);
  srv->reqs.erase(it);
  return HFX_OK;
}

extern "C" int hfx_serve_progress(hfx_server* srv) {
  if (!srv) return HFX_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (int r = server_progress_locked(srv)) return r;
  return server_pending(srv);
}

extern "C" int hfx_serve_wait(hfx_server* srv, uint64_t ticket, double timeout_ms, hfx_result* out) {
  if (!srv || !out) return HFX_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      auto it = srv->reqs.find(ticket);
      if (it == srv->reqs.end()) return srv->fail(HFX_ERR_ARG, "hfx_serve_wait: unknown ticket");
      if (int r = server_progress_locked(srv)) return r;
      Request& q = it->second;
      if (q.status != HFX_REQ_QUEUED && q.status != HFX_REQ_RUNNING) {
        recycle_event(srv, q);
        fill_result(srv, q, out);
        return q.status == HFX_REQ_DONE ? HFX_OK : q.status;
      }
      if (timeout_ms >= 0.0 && host_ms_since(t0) > timeout_ms) {
        fill_result(srv, q, out);
        return srv->fail(HFX_ERR_TIMEOUT, "hfx_serve_wait: timed out");
      }
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

extern "C" int hfx_serve_drain(hfx_server* srv, double timeout_ms) {
  if (!srv) return HFX_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      if (int r = server_progress_locked(srv)) return r;
      if (server_pending(srv) == 0) return HFX_OK;
      if (timeout_ms >= 0.0 && host_ms_since(t0) > timeout_ms)
        return srv->fail(HFX_ERR_TIMEOUT, "hfx_serve_drain: timed out");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

extern "C" int hfx_server_get_stats(hfx_server* srv, hfx_server_stats* out) {
  if (!srv || !out) return HFX_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  *out = srv->st;
  out->n_queued = (int64_t)srv->queue.size();
  out->n_running = 0;
  for (const Slot& sl : srv->slots) out->n_running += (int64_t)sl.reqs.size();
  out->bytes_resident = (int64_t)srv->bytes_resident;
  out->bytes_requests = (int64_t)srv->bytes_requests;
  out->bytes_peak = (int64_t)srv->bytes_peak;
  return HFX_OK;
}

extern "C" const char* hfx_server_last_error(const hfx_server* srv) { return srv ? srv->err.c_str() : ""; }
