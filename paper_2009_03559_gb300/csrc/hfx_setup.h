// Host wrappers of the set-up / finalisation kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include "hfx_internal.cuh"

namespace hfx {

// One system of a batched K build (device table; read by the batched kernels).
// One system of a batched build: its matrices, shell data and per-build scratch.
constexpr int kBatchPart = 64;  // partial sums of E_K per system (2 doubles each)
struct BatchSys {
  const double* P;
  double* K;
  int n, ld, ns;
  const int* bf_off;
  const int* l;
  double* pmax;    // ns x ns block maxima of |P|
  double* energy;  // E_K
  double* part;    // 2 * kBatchPart doubles
  double* pglob;   // max |P| over the matrix, or NULL when not needed
};

// Rows of the quartet task list: class pair cp = hi(hi+1)/2 + lo owns rows
// [row_base[cp], row_base[cp+1]), one per bra pair of bin hi.
struct RowTable {
  int row_base[22];
  int bin_start[7];
  int bin_size[7];
};

cudaError_t launch_normalize(int n_shells, const int* l, const int* nprim, const int* prim_off,
                             const double* alpha, const double* coef, double* w, cudaStream_t s);
cudaError_t launch_boys_table(double* tab, cudaStream_t s);
cudaError_t launch_pair_flags(long long n_tri, const int* atom, const double* xyz, double rcut, int* flag,
                              cudaStream_t s);
cudaError_t select_flagged(void* tmp, size_t& tmp_bytes, long long n_tri, const int* flag, long long* out,
                           int* d_num, cudaStream_t s);
// periodic pair list (home-cell shell x image shell candidates)
cudaError_t launch_pair_flags_rect(long long n, int n_img, const int* atom, const double* xyz, double rcut, int* flag,
                                   cudaStream_t s);
cudaError_t launch_pair_setup_rect(int n_cand, const long long* cand_t, int n_img, const int* l, const int* nprim,
                                   const int* atom, const double* xyz, int* sa, int* sb, int* pcls, double* AB,
                                   int* cap, unsigned char* home_first, cudaStream_t s);
cudaError_t launch_pair_setup(int n_cand, const long long* cand_t, const int* l, const int* nprim,
                              const int* atom, const double* xyz, int* sa, int* sb, int* pcls, double* AB,
                              int* cap, cudaStream_t s);
cudaError_t scan_int(void* tmp, size_t& tmp_bytes, const int* in, int* out, int n, cudaStream_t s);
cudaError_t scan_ll_inclusive(void* tmp, size_t& tmp_bytes, const long long* in, long long* out, int n,
                              cudaStream_t s);
cudaError_t launch_prim_fill(int n_cand, const int* sa, const int* sb, const int* nprim, const int* prim_off_shell,
                             const int* atom, const double* xyz, const double* alpha, const double* w,
                             const int* pp_off, double prim_tau, PrimPair* pp, int* pp_n, cudaStream_t s);
// distance-aware screening: per candidate pair (centre xyz, spread, smallest exponent sum),
// and the same gathered into sorted-pair order
cudaError_t launch_pair_dist(int n_cand, const int* sa, const int* sb, const int* nprim, const int* prim_off_shell,
                             const int* atom, const double* xyz, const double* alpha, double* out, cudaStream_t s);
cudaError_t launch_gather5(int n, const int* sorted, const double* in, double* out, cudaStream_t s);
cudaError_t launch_iota(int n, int* v, cudaStream_t s);
cudaError_t launch_hist(int n, const int* key, int* counts, cudaStream_t s);
cudaError_t sort_int_keys(void* tmp, size_t& tmp_bytes, const int* kin, int* kout, const int* vin, int* vout,
                          int n, int end_bit, cudaStream_t s);
cudaError_t sort_double_desc(void* tmp, size_t& tmp_bytes, const double* kin, double* kout, const int* vin,
                             int* vout, int n, cudaStream_t s);
cudaError_t reduce_max(void* tmp, size_t& tmp_bytes, const double* in, double* out, int n, cudaStream_t s);
cudaError_t launch_bin_keys(int n, const double* Q, const double* qmax, double tau, const int* pcls,
                            const int* order, int* binkey, cudaStream_t s);
cudaError_t launch_gather_q(int n, const int* sorted, const double* Q, double* Qs, cudaStream_t s);
// triangle: a ket of the bra's own bin only up to the bra (each unordered pair of pairs once);
// off for periodic builds, whose bra and ket pairs are distinct objects (ket shifted by G)
cudaError_t launch_count(int n_rows, const RowTable& rt, const double* Qs, double tau, long long* row_n,
                         cudaStream_t s, bool triangle = true);
cudaError_t launch_gather_bounds(const RowTable& rt, const long long* qoff, long long* out, cudaStream_t s);
cudaError_t launch_finalize(int n, int ld, const double* P, double* K, double* part, int n_part, double* energy,
                            cudaStream_t s);
// block maxima of |P| per shell pair; with pglob != NULL also the maximum over all of P
cudaError_t launch_pmax(int ns, const int* bf_off, const int* l, const double* P, int ld, double* pmax,
                        double* pglob, cudaStream_t s);
cudaError_t launch_batch_prologue(const BatchSys* sys, int n, int n_sm, bool pmax, cudaStream_t s);
cudaError_t launch_batch_epilogue(const BatchSys* sys, int n, int n_sm, cudaStream_t s);
cudaError_t fma_peak(double* fp64_tflops, double* fp32_tflops);
cudaError_t fp64_lane_cost(double* ms_32, double* ms_1);
// periodic: max |P^R| per (R, home shell, home shell) block (bf_off, l of the home shells)
cudaError_t launch_pmax_blocks(int n_R, int ns, int nbf, const int* bf_off, const int* l, const double* P,
                               double* pmax, cudaStream_t s);
// B = A^T (n x n, row-major, distinct buffers)
cudaError_t launch_transpose(int n, const double* A, double* B, cudaStream_t s);

}  // namespace hfx
