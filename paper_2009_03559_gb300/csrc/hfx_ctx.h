// Internal: the context record shared by the library's translation units.
#pragma once
#include <string>
#include <vector>

#include "hfx.h"
#include "hfx_internal.cuh"
#include "hfx_setup.h"

namespace hfx {
// allocation-failure injection (hfx_debug_fail_alloc): true when this allocation must fail
bool alloc_fault_due();
}  // namespace hfx

// device counters per class: primitive quartets evaluated, quartets evaluated, primitive
// quartets dropped at the Boys step, quartets in FP32, primitive quartets in FP32
constexpr int kNCnt = 5;

struct hfx_ctx {
  cudaStream_t stream = nullptr;
  hfx_options opt{};
  std::string err;
  int n_atoms = 0, n_shells = 0, n_bf = 0, n_prim = 0, n_sm = 0;
  std::vector<int> h_l;
  // basis (device)
  double *d_xyz = nullptr, *d_alpha = nullptr, *d_coef = nullptr, *d_w = nullptr, *d_boys = nullptr;
  int *d_atom = nullptr, *d_l = nullptr, *d_nprim = nullptr, *d_prim_off = nullptr, *d_bf_off = nullptr;
  // pairs (device)
  int n_cand = 0, n_kept = 0;
  int *d_sa = nullptr, *d_sb = nullptr, *d_pcls = nullptr, *d_pp_off = nullptr, *d_pp_n = nullptr;
  double *d_AB = nullptr, *d_Q = nullptr, *d_Qs = nullptr;
  double* d_dist = nullptr;  // distance-aware test data per sorted pair (5 doubles)
  hfx::PrimPair* d_pp = nullptr;
  int* d_sorted = nullptr;
  hfx::RowTable rt{};
  int n_rows = 0;
  long long* d_qoff = nullptr;
  long long cls_q[21] = {}, cls_qbegin[21] = {};
  bool pairs_ready = false;
  // per build
  double *d_energy = nullptr, *d_part = nullptr, *d_pmax = nullptr, *d_pglob = nullptr;
  int n_part = 0;
  double *d_Pst = nullptr, *d_Kst = nullptr;
  unsigned long long* d_busy = nullptr;      // per SM
  unsigned long long* d_counters = nullptr;  // kNCnt per class
  unsigned long long* d_work = nullptr;      // dynamic-schedule claim counter per class
  bool timing = false;
  cudaEvent_t ev[2 * 21 + 4] = {};
  bool ev_ok = false;
  bool class_launched[21] = {};
  int gs_override[21] = {};  // lanes per quartet chosen by the caller per class (0 = default)
  int gs_used[21] = {};      // lanes per quartet of each class in the last build
  int streams_override[21] = {};  // warp kernel: primitive quartets at a time (0 = default)
  int streams_used[21] = {};
  hfx_stats stats{};
  // periodic context (hfx_init_periodic): the basis above is the image cluster, the home
  // cell's shells repeated over n_cells cells (home cell first)
  bool periodic = false;
  int n_home_atoms = 0, n_home_shells = 0, n_home_bf = 0, n_cells = 0;
  double lattice[9] = {};
  std::vector<int> h_cells;              // 3 per cell
  int *d_shell_cell = nullptr, *d_shell_bf = nullptr, *d_cell_xyz = nullptr;
  unsigned char* d_home_first = nullptr;  // per candidate pair (pair scope)
  // per periodic build, reused while large enough: cell map of the density blocks, their
  // block maxima
  int* d_rmap = nullptr;
  size_t rmap_cap = 0;
  double* d_pmaxR = nullptr;
  size_t pmaxR_cap = 0;
  // a context-lifetime buffer of at least n elements in *p (capacity *cap), reallocated when short
  template <class T>
  int scratch(T** p, size_t* cap, size_t n) {
    if (*p && *cap >= n) return HFX_OK;
    if (*p) {
      for (auto it = allocs.begin(); it != allocs.end(); ++it)
        if (*it == (void*)*p) {
          allocs.erase(it);
          break;
        }
      cudaFree(*p);
      bytes -= *cap * sizeof(T);
      *p = nullptr;
      *cap = 0;
    }
    const int r = alloc(p, n);
    if (r == HFX_OK) *cap = n;
    return r;
  }
  float ms_pairs = 0.f;
  std::vector<void*> allocs;       // owned for the context lifetime
  std::vector<void*> pair_allocs;  // owned until the next build_pairs
  size_t bytes = 0, pair_bytes = 0;  // device bytes held by allocs / pair_allocs

  int fail(int code, const std::string& msg) {
    err = msg;
    return code;
  }
  int cuda_fail(const char* what, cudaError_t e) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? HFX_ERR_OOM : HFX_ERR_CUDA;
  }
  template <class T>
  int alloc(T** p, size_t n, bool pair_scope = false) {
    *p = nullptr;
    if (n == 0) n = 1;
    if (hfx::alloc_fault_due()) return fail(HFX_ERR_OOM, "cudaMalloc: injected allocation failure");
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) return cuda_fail("cudaMalloc", e);
    (pair_scope ? pair_allocs : allocs).push_back(*p);
    (pair_scope ? pair_bytes : bytes) += n * sizeof(T);
    return HFX_OK;
  }
  void free_pairs() {
    for (void* p : pair_allocs) cudaFree(p);
    pair_allocs.clear();
    pair_bytes = 0;
    pairs_ready = false;
  }
};

namespace hfx {
// read-only parts of a context's launch record (pairs, shells, Boys table, omega)
EriLaunch base_launch(hfx_ctx* ctx);
// message for hfx_last_error(NULL) from entry points that have no context
void set_global_error(const std::string& msg);
}  // namespace hfx
