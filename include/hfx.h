/*
 * hfx.h -- C ABI of the GB300 (sm_103a) screened HSE exact-exchange library.
 *
 * The library builds the exchange matrix of the paper's hybrid-functional method
 * (Sec. 2, Eq. vx, for one cell and without lattice images or the -1/2 prefactor):
 *
 *     K_{mu nu} = sum_{lambda sigma} (mu lambda | nu sigma)_omega P_{lambda sigma}
 *
 * over contracted Gaussian shells of angular momentum 0..2 with (2l+1) spherical
 * functions each (Sec. 3.1, shell quartets; Cartesian -> spherical step, Sec. 3.1),
 * with the HSE06 short-range kernel erfc(omega r)/r in the two-electron integral
 * (Sec. 2, ERI definition; Sec. 4, HSE06).  A shell quartet (IJ|KL) contributes iff
 * pair IJ and pair KL are kept and Q_IJ Q_KL >= tau (Schwarz screening, Sec. 3.1
 * Eq. schwarz), where Q_IJ = sqrt(max_{mu in I, nu in J} (mu nu|mu nu)).  A pair is
 * kept iff its atoms are closer than 2 r_c (or identical, or r_c <= 0: NAO/orbital-
 * cutoff screening, Sec. 3.1) and Q_IJ Q_max >= tau.  Each unique quartet is evaluated
 * once (eight-fold permutational symmetry, Sec. 3.1) by CUDA kernels.
 *
 * Basis functions: chi_{I,m}(r) = N_I S_m(r - A) sum_k c_k alpha_k^{(2l+3)/4}
 * exp(-alpha_k |r - A|^2), with S_m = 1; x, y, z; xy, yz, (3z^2 - r^2)/(2 sqrt 3), xz,
 * (x^2 - y^2)/2 and N_I such that every function has unit self-overlap.  Function
 * order: shells in input order, components in the order just listed.
 *
 * Conventions for every entry point:
 *   - Return value: HFX_OK (0) on success, a negative HFX_ERR_* code otherwise; the
 *     message of the last failure is available from hfx_last_error().  The library
 *     never aborts the process and has no CPU fallback: without a CUDA device every
 *     call that needs one fails with HFX_ERR_CUDA.
 *   - Device pointers are CUDA global-memory addresses on the current device; host
 *     pointers are ordinary process memory.  The caller owns every buffer it passes;
 *     the library owns what it allocates inside a context and frees it in hfx_free().
 *   - Matrices are dense, FP64, row-major with leading dimension ld >= n_bf.
 *   - Work is ordered on the context's CUDA stream; "async" calls return before the
 *     GPU work ends.  Calls on one context are not thread-safe.
 */
#ifndef HFX_H
#define HFX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define HFX_OK 0
#define HFX_ERR_ARG -1            /* invalid argument (null pointer, bad size or index) */
#define HFX_ERR_UNSUPPORTED_L -2  /* shell angular momentum outside 0..2 */
#define HFX_ERR_OOM -3            /* device allocation failed */
#define HFX_ERR_CUDA -4           /* a CUDA call or kernel launch failed */
#define HFX_ERR_STATE -5          /* call order violated (e.g. build_K before build_pairs) */
#define HFX_ERR_TIMEOUT -6        /* a bounded wait gave up */
#define HFX_ERR_ADMISSION -7      /* a request can never fit the server's memory budget */

/* precision modes */
#define HFX_FP64 0                /* every integral in FP64 */
#define HFX_MIXED 1               /* FP32 recurrences for small-bound quartets, see hfx_options */

/* Default classes allowed FP32 recurrences under HFX_MIXED: every class but (dd|dd), the
 * highest recurrence (L = 8): with FP32 there, E_K of the 64-atom diamond moved by 1.7e-7 and
 * of the 216-atom one by 4.1e-7 (over the 1e-7 tolerance), against at most 1.1e-9 with the
 * other twenty classes in FP32. */
#define HFX_FP32_CLASSES_DEFAULT 0xFFFFF

/* work schedules inside a class launch (paper Sec. 3.2, Algorithms 2 and 3) */
#define HFX_SCHED_QUARTET 0       /* static even split of the screened quartet list */
#define HFX_SCHED_PAIR 1          /* static even split of the bra pair list, screening after */
#define HFX_SCHED_DYNAMIC 2       /* chunks of the quartet list handed out by a device atomic
                                     counter (the paper's "dynamic distribution"; default) */

typedef struct hfx_ctx hfx_ctx;   /* opaque, library-owned */

typedef struct {
  double omega;        /* range-separation parameter (bohr^-1); 0 gives the Coulomb kernel */
  double schwarz_tau;  /* Schwarz threshold tau (>= 0) */
  double rcut_bohr;    /* orbital cutoff radius r_c; <= 0 disables the pair-distance screen */
  double prim_tau;     /* primitive pairs with |prefactor| below this are dropped (default 1e-22) */
  double fp32_tau;     /* HFX_MIXED: a quartet's primitive set-up, recurrences (VRR) and their
                          contraction run in FP32 iff Q_IJ Q_KL Pmax < fp32_tau (default 1e-6),
                          Pmax as set by fp32_pmax_global; HRR, spherical step and all K
                          accumulation stay FP64.  The FP32 Boys step is the difference of two
                          upper incomplete gamma functions (erfc and an upward recursion of
                          positive terms); a primitive quartet where the subtracted one exceeds
                          1/64 of the other (small T (1 - kappa)) takes the FP64 Boys step.  FP32
                          quartets run on whole warps, four primitive quartets per float4 slot
                          (two FFMA2 per op) */
  int precision;       /* HFX_FP64 (default) or HFX_MIXED */
  int schedule;        /* HFX_SCHED_DYNAMIC (default), HFX_SCHED_QUARTET or HFX_SCHED_PAIR */
  int skip_zero_p;     /* 1 (default): skip quartets whose four density blocks P_bd, P_bc,
                          P_ad, P_ac are all exactly zero (their contribution is exactly 0) */
  int fp32_class_mask; /* HFX_MIXED: bit c allows FP32 for quartet class c (index as in
                          n_quartets_class); default HFX_FP32_CLASSES_DEFAULT */
  int fp32_pmax_global;/* HFX_MIXED: 0 (default): Pmax = max(|P_bd|,|P_bc|,|P_ad|,|P_ac|), the
                          largest density element the quartet's four K updates multiply;
                          1: Pmax = max |P| over the whole matrix (more conservative) */
  int reserved[1];     /* set to 0 */
  double density_tau;  /* density-weighted screening (default 0 = off): a quartet is also
                          dropped when Q_IJ Q_KL max(|P_bd|,|P_bc|,|P_ad|,|P_ac|) <
                          density_tau; it changes K by at most that bound per dropped quartet
                          and block element, and extends the exact-zero skip to small
                          densities (Sec. 3.1 screening with the density folded in) */
  double dist_tau;     /* distance-aware screening (default 0 = off): a quartet is also dropped
                          when Q_IJ Q_KL exp(-kappa rho R^2) < dist_tau, the short-range
                          kernel's decay between the two pair distributions (rho from the pairs'
                          smallest exponent sums p, q: pq/(p+q); kappa = omega^2/(omega^2+rho);
                          R the distance of their most diffuse primitive-pair centres less the
                          spread of each pair's primitive-pair centres).  For s-type primitive
                          quartets the factor bounds the integral; for higher angular momentum
                          it is an estimate (measured far below the true factor) */
} hfx_options;

typedef struct {
  int64_t n_pairs_cutoff;      /* shell pairs passing the orbital cutoff */
  int64_t n_pairs_kept;        /* ... and the pair Schwarz test */
  int64_t n_quartets;          /* canonical shell quartets kept (Schwarz + cutoff) */
  int64_t n_quartets_class[21];/* per class, index hi*(hi+1)/2 + lo over pair classes
                                  ss, ps, pp, ds, dp, dd */
  int64_t prim_quartets_class[21]; /* primitive quartets evaluated per class (timed builds) */
  int64_t quartets_evaluated_class[21]; /* quartets evaluated per class (timed builds): the kept
                                  quartets minus those skipped for exactly-zero density blocks */
  int64_t quartets_fp32_class[21]; /* of those, evaluated with FP32 recurrences (HFX_MIXED) */
  double flops_fp32;           /* FP32 flops of the last timed build (same model) */
  double flops_fp64;           /* FP64 flops of the last timed K build (operation-count model
                                  of the kernels: add/mul = 1, fma = 2) */
  double flops_class[21];      /* the same per class */
  int32_t group_size_class[21];/* lanes per quartet of each class in the last build (1 or 32) */
  double ms_pairs;             /* GPU time of the last hfx_build_pairs */
  double ms_build;             /* GPU time of the last hfx_build_K (zero K .. E_K ready) */
  double ms_class[21];         /* GPU time of each class launch in the last K build */
  double energy;               /* E_K = sum_{mu nu} P_{mu nu} K_{mu nu} of the last K build */
  double flops_recurrence;     /* of flops_fp64 + flops_fp32: the recurrences alone (vertical
                                  recurrence, contraction, horizontal recurrence, Cartesian ->
                                  spherical step, digest into K), the primitive set-up excluded */
  double special_evals;        /* Boys-function evaluations of the last timed build (each: F_m at
                                  the top order and exp(-x) from the tables): two per evaluated
                                  primitive quartet with the erfc kernel, one with omega = 0 */
  int32_t streams_class[21];   /* warp kernel: primitive quartets run at a time per class */
  int32_t reserved_stats[1];
  double flops_recurrence_class[21]; /* flops_recurrence per class */
} hfx_stats;

/* ---------------------------------------------------------------------------
 * Periodic images: the lattice sums of Eq. vx (Sec. 2) for a crystal.
 *
 *   K^G_{mu lambda} = sum_{N,H} sum_{nu sigma} (mu^0 nu^N | lambda^G sigma^H) P^{H-N}_{nu sigma}
 *
 * mu, lambda run over the home cell's functions, nu^N over those of cell N, sigma^H of
 * cell H; P^R couples a home-cell function to one of cell R.  The library builds list-IJ
 * in the home cell (every pair with one shell in the home cell and its partner in any cell
 * within the orbital cutoff 2 r_c, Sec. 3.1), Schwarz-screens it like the molecular list
 * (Q_max over the crystal), and for each requested cell G evaluates every quartet (p | q + G)
 * of two such pairs with Q_p Q_q >= tau whose density block exists (list-KL over the
 * supercell, Sec. 3.1), in FP64 by the same kernels with the ket pair translated by G.  A
 * quartet whose density cell offset is not in the given list contributes nothing.
 * ------------------------------------------------------------------------- */

/* Creates a periodic context: the home cell (n_atoms atoms at xyz, shells as in
 * hfx_init_basis) and lattice[9] (rows: the three cell vectors, bohr; host).  The options
 * must set rcut_bohr > 0 (the cutoff bounds the image sums) and precision HFX_FP64.  The
 * library replicates the cell over the box of cells the cutoff can reach (at most 8 in
 * each direction) and keeps that image basis on the device.  Errors: HFX_ERR_ARG (no
 * cutoff, degenerate lattice, cutoff reaching too far), the hfx_init_basis errors. */
int hfx_init_periodic(hfx_ctx** out, int n_atoms, const double* xyz, const double* lattice, int n_shells,
                      const int* shell_atom, const int* shell_l, const int* shell_nprim, const double* alpha,
                      const double* coef, const hfx_options* opt, void* stream);

/* Integer cell coordinates of the image box (3 per cell, home cell first) into cells[3*max_n]
 * (host, may be NULL); returns the number of cells, or HFX_ERR_ARG for a molecular context. */
int hfx_periodic_cells(const hfx_ctx* ctx, int* cells, int max_n);

/* K^G for n_G cells.  R_cells[3*n_R] (host): the cell offsets R of the density blocks;
 * P_R (device): n_R blocks P^R, each n_bf x n_bf row-major (n_bf of the home cell), in the
 * order of R_cells.  G_cells[3*n_G] (host); K_G (device): n_G blocks K^G written in full
 * (zeroed first).  For a cell whose opposite -G comes earlier in G_cells, K^G is the
 * transpose of K^{-G} (exchanging bra and ket pairs maps one lattice sum onto the other;
 * the density blocks must satisfy P^{-R} = (P^R)^T, as a real density does).  Asynchronous
 * on the context's stream.  Errors: HFX_ERR_STATE (not a
 * periodic context, no pair list), HFX_ERR_ARG (empty lists, a repeated R, |R_i| > 32). */
int hfx_build_K_periodic(hfx_ctx* ctx, int n_R, const int* R_cells, const double* P_R, int n_G, const int* G_cells,
                         double* K_G);

/* Primitive quartets the warp kernel runs at a time for quartet class cls (0..20) in later
 * builds: 0 = the class default, else one of the variants the library carries (1, 2 or 4;
 * the largest classes carry fewer).  Results do not depend on it (summation order aside).
 * Errors: HFX_ERR_ARG for an unknown class or a variant the class does not carry. */
int hfx_set_streams(hfx_ctx* ctx, int cls, int streams);

/* Fills *opt with defaults: omega 0.11, tau 1e-10, no cutoff, prim_tau 1e-22, FP64,
 * dynamic schedule, zero-density-block skip on. */
void hfx_default_options(hfx_options* opt);

/* Creates a context for one system and uploads its basis.
 *   n_atoms, xyz[3*n_atoms]: atom positions in bohr (host).
 *   n_shells, shell_atom[n_shells] (0-based atom of each shell), shell_l[n_shells]
 *   (0..2), shell_nprim[n_shells] (>= 1, <= 8): host arrays.
 *   alpha[], coef[]: exponents (> 0) and raw contraction weights of all primitives,
 *   shell after shell (host; the library normalises, see the header comment).
 *   opt: options (host, may be NULL for defaults).  stream: cudaStream_t to order
 *   all work of this context on (NULL = default stream).
 * On success *out receives the context.  Basis upload and normalisation are queued
 * on the stream.  Errors: HFX_ERR_ARG, HFX_ERR_UNSUPPORTED_L, HFX_ERR_OOM, HFX_ERR_CUDA. */
int hfx_init_basis(hfx_ctx** out, int n_atoms, const double* xyz, int n_shells,
                   const int* shell_atom, const int* shell_l, const int* shell_nprim,
                   const double* alpha, const double* coef, const hfx_options* opt,
                   void* stream);

/* Builds the screened shell-pair list (Sec. 3.1: list-IJ = list-KL here, one cell):
 * orbital-cutoff test, primitive-pair data, Schwarz diagonal Q_IJ by the ERI kernels,
 * pair Schwarz test, binning by pair class with Q descending, and the per-class
 * quartet task lists (bra pair -> number of ket pairs passing Q_IJ Q_KL >= tau) with
 * their 64-bit prefix sums.  The list depends on the basis only, not on P.
 * Synchronises the stream once (sizes are read back to size the launches). */
int hfx_build_pairs(hfx_ctx* ctx);

/* Builds K for the density P (both device pointers, n_bf x n_bf, leading dimension
 * ld; P symmetric).  K is overwritten completely.  Asynchronous on the context stream;
 * E_K lands in a device scalar (read it with hfx_energy or hfx_get_stats).
 * Errors: HFX_ERR_STATE (no pair list), HFX_ERR_ARG, HFX_ERR_CUDA. */
int hfx_build_K(hfx_ctx* ctx, const double* P_dev, double* K_dev, int ld);

/* Partition `part` (0 <= part < n_parts) of the same K build: only the quartets of a
 * contiguous 1/n_parts of every class's screened quartet list (hfx_part_range) contribute.
 * K_part and E_part = sum P K_part of the parts add up to K and E_K of hfx_build_K; the
 * parts are independent (no communication), which is how the build shards over GPUs
 * (one part per GPU, then one sum of the K_part).  Needs the quartet or dynamic
 * schedule.  Otherwise as hfx_build_K. */
int hfx_build_K_part(hfx_ctx* ctx, const double* P_dev, double* K_dev, int ld, int part, int n_parts);

/* The range [*q0, *q1) of a list of `count` items that part `part` of n_parts owns:
 * q0 = floor(count part / n_parts), q1 = floor(count (part + 1) / n_parts).  Host only. */
int hfx_part_range(int64_t count, int part, int n_parts, int64_t* q0, int64_t* q1);

/* Same computation with host buffers: copies P (host, n_bf x n_bf row-major) to the
 * device, builds K, copies K back into K_host and returns after the copy ends.  The
 * device staging buffers are owned by the context. */
int hfx_build_K_host(hfx_ctx* ctx, const double* P_host, double* K_host);

/* Device pointer to the FP64 scalar E_K of the last K build (valid until hfx_free). */
const double* hfx_energy_device(const hfx_ctx* ctx);

/* Synchronises the stream and copies E_K of the last build to *out. */
int hfx_energy(hfx_ctx* ctx, double* out);

/* Synchronises the stream and fills *out (timings need HFX timing enabled, see
 * hfx_set_timing). */
int hfx_get_stats(hfx_ctx* ctx, hfx_stats* out);

/* Lanes per quartet for class cls (0..20) in later K builds of this context: 1 (a thread
 * owns a quartet), 32 (a warp), 0 = the library's default (1 for the nine classes whose
 * scratch fits the thread kernel, 32 otherwise; in a mixed-precision build the FP32 pass runs
 * 32 in every class).  A value set here applies to both passes of a mixed-precision class.
 * 1 needs a class whose scratch fits the thread kernel, else the build fails with
 * HFX_ERR_CUDA.  Errors: HFX_ERR_ARG. */
int hfx_set_group_size(hfx_ctx* ctx, int cls, int gs);

/* Enables (1) or disables (0) per-class CUDA-event timing of K builds. */
int hfx_set_timing(hfx_ctx* ctx, int enable);

/* Number of basis functions of the context, or a negative error code. */
int hfx_n_basis(const hfx_ctx* ctx);

/* Device bytes the context holds (basis, pair list, per-build scratch), or a negative
 * error code. */
int64_t hfx_device_bytes(const hfx_ctx* ctx);

/* Copies the kept pairs (shell a, shell b with l_a >= l_b, Q) in bin order to host
 * arrays of length >= max_n; returns the number of kept pairs or an error code. */
int64_t hfx_get_pairs(hfx_ctx* ctx, int* shell_a, int* shell_b, double* q, int64_t max_n);

/* Per-SM load record of the last K build: for each of n_slots CTA slots, the
 * globaltimer start and end (ns) of its ERI work, summed over class launches
 * (busy_ns[n]); returns the number of entries written. */
int hfx_get_cta_busy(hfx_ctx* ctx, double* busy_ns, int max_n);

/* Message of the last failure on this context ("" if none); ctx may be NULL for
 * failures of hfx_init_basis. */
const char* hfx_last_error(const hfx_ctx* ctx);

/* Releases the context and all device memory it owns (synchronises the stream). */
void hfx_free(hfx_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Batched K builds: the quartets of several systems (contexts with pair lists) go into
 * one launch per angular class (two under HFX_MIXED: the FP64 and the FP32 share); the
 * class launches can be spread over up to four parallel branches (largest classes first,
 * each to the least loaded branch) so that one class's tail overlaps the next ones; the whole
 * build (zeroing, density block maxima, the class launches, K = A + A^T, E_K per system)
 * is captured once as a CUDA graph and replayed.  The systems' P and K pointers are read from a device table refreshed from
 * host memory before each replay, so new buffers need no new graph.  Precision and
 * zero-block skip follow the first context's options.
 * ------------------------------------------------------------------------- */
typedef struct hfx_batch hfx_batch;

typedef struct {
  int64_t n_quartets;          /* screened quartets of all systems */
  double ms_last;              /* GPU time of the last hfx_batch_run (events around it) */
  int32_t group_size_class[21];/* chosen lanes per quartet (1 or 32) per class */
  int32_t chunk_class[21];     /* chosen quartets per dynamic claim per class */
  double tune_ms_class[21];    /* best tuning time per class, scaled from its window to the class */
  int64_t tune_window_class[21]; /* quartets in the window each candidate was timed on */
  int32_t streams_class[21];   /* warp kernel: primitive quartets at a time per class (0: thread kernel) */
  int32_t tune_kept;           /* 1 if the last hfx_batch_tune kept its choices (they beat the
                                  previous ones on the whole batch), 0 if it restored them */
  double tune_full_default_ms; /* last hfx_batch_tune: whole batch with the previous choices */
  double tune_full_tuned_ms;   /* ... and with the tuned ones */
  int32_t branches;            /* parallel branches the class launches are spread over */
  int32_t reserved_b[1];
} hfx_batch_stats;

/* Creates a batch over n contexts (all with pair lists, same device).  Runs are ordered
 * after earlier work on `stream` (NULL = the first context's stream) and later work on it
 * waits for them; the batch captures and launches its graph on a stream of its own.  The
 * contexts must outlive the batch. */
int hfx_batch_create(hfx_batch** out, hfx_ctx* const* ctxs, int n, void* stream);

/* Autotuner: for every class, times its batched launch with each candidate kernel shape
 * (a warp per quartet with 1, 2 or 4 primitive quartets at a time, or a thread per quartet
 * where the class allows it) and dynamic chunk size (quartets per claim) on one window of
 * the class's quartets, and keeps the fastest; a candidate must beat the current choice by
 * 5% to replace it.  Then it times the whole batch with the previous and with the tuned
 * choices and keeps the tuned ones only if they are faster (the number of parallel branches,
 * 1 or 4, is chosen there too), so tuning never makes a batch slower than its previous
 * configuration as measured by these runs.  Uses P/K like
 * hfx_batch_run (their K contents are overwritten; run hfx_batch_run afterwards).
 * Synchronises. */
int hfx_batch_tune(hfx_batch* b, const double* const* P_dev, double* const* K_dev, const int* ld);

/* Builds K_s for P_s of every system s (device pointers; ld[s] >= n_bf of system s; ld
 * may be NULL for ld = n_bf).  The first call captures the graph, later calls replay it.
 * Asynchronous; E_K of system s lands in its context (hfx_energy). */
int hfx_batch_run(hfx_batch* b, const double* const* P_dev, double* const* K_dev, const int* ld);

/* Launch time the tuner aims at per candidate (default 20 ms): each class's candidates are
 * timed on one window of its quartet list, grown from 16k quartets to about this time. */
int hfx_batch_set_tune_target(hfx_batch* b, double ms);

/* Parallel branches (streams, graph branches) the class launches are spread over: 1..4
 * (default 1).  The autotuner also chooses between 1 and 4 on the whole batch. */
int hfx_batch_set_branches(hfx_batch* b, int n);

/* 1 (default): capture and replay a CUDA graph; 0: plain launches every run. */
int hfx_batch_set_graph(hfx_batch* b, int enable);

int hfx_batch_get_stats(hfx_batch* b, hfx_batch_stats* out);
void hfx_batch_free(hfx_batch* b);

/* One-shot form: create a batch, run it once, free it. */
int hfx_build_K_batched(hfx_ctx* const* ctxs, const double* const* P_dev, double* const* K_dev, const int* ld, int n);

/* ---------------------------------------------------------------------------
 * Serving: a request loop over registered systems with continuous batching.
 *
 * Systems (contexts with pair lists) are registered once and stay resident: basis,
 * pair lists and Boys table live on the device for the server's life.  A request names
 * a system and gives a density P and a destination for K.  The server keeps a FIFO
 * queue and up to max_inflight steps on the device at once, each on a stream of its
 * own.  Whenever a step slot is free, the queued requests that fit (in arrival order, at
 * most max_batch and max_step_quartets, while the memory budget allows) form one step: their P are copied
 * to server-owned device buffers, one batched launch per class evaluates all their
 * quartets (as hfx_batch_run), and each K goes to its destination.  Requests arriving
 * while steps run are admitted as soon as a slot and memory free up, so their work
 * overlaps on the device with the steps still running.
 *
 * Admission by memory: the server holds the resident systems, its step workspaces and,
 * for every admitted request, P, K and the density-block maxima (2 n_bf^2 + n_shells^2
 * doubles).  A queued request is admitted only while the total stays within
 * hbm_budget_gb; a request that could never fit is refused with HFX_ERR_ADMISSION.
 *
 * The server is single-threaded and driven by its callers: every submit, poll, wait and
 * progress call retires finished steps and starts new ones.  Calls are serialised by an
 * internal lock, so several host threads may share one server.
 * ------------------------------------------------------------------------- */
typedef struct hfx_server hfx_server;

typedef struct {
  double hbm_budget_gb;  /* device memory the server may hold (default 120 GB) */
  double max_step_quartets; /* a step takes further queued requests only while its screened
                            quartets stay within this (default 1e7; a larger request runs
                            alone): small systems are batched, large ones do not wait for
                            each other */
  int max_inflight;      /* steps on the device at once, each on its own stream (default 4) */
  int max_batch;         /* most requests in one step (default 16) */
  int precision;         /* HFX_FP64 (default) or HFX_MIXED for every request; the FP32 test
                            uses each system's fp32_tau, fp32_class_mask and fp32_pmax_global */
  int reserved[5];       /* set to 0 */
} hfx_server_options;

#define HFX_REQ_DONE 0
#define HFX_REQ_QUEUED 1
#define HFX_REQ_RUNNING 2

typedef struct {
  uint64_t ticket;
  int32_t status;        /* HFX_REQ_DONE, _QUEUED, _RUNNING or a negative HFX_ERR_* code */
  int32_t system_id;
  int32_t step_size;     /* requests in the step that computed it */
  int32_t pad;
  double energy;         /* E_K = sum P K of this request */
  double t_submit_ms;    /* times since server creation: submit call, */
  double t_admit_ms;     /* step launch (host clock), */
  double t_done_ms;      /* end of the step's work on the device (CUDA events) */
  double ms_step;        /* device time of the step, P copy-in to K copy-out */
  int64_t n_quartets;    /* screened quartets of the system */
} hfx_result;

typedef struct {
  int64_t n_submitted, n_done, n_failed, n_steps, n_queued, n_running;
  int64_t quartets_done;
  int64_t bytes_resident;  /* registered systems + step workspaces */
  int64_t bytes_requests;  /* admitted requests now */
  int64_t bytes_peak;      /* largest resident + requests seen */
  int32_t max_step_size, max_steps_inflight;
} hfx_server_stats;

void hfx_server_default_options(hfx_server_options* opt);

/* Creates a server on the current device.  opt may be NULL for defaults. */
int hfx_server_create(hfx_server** out, const hfx_server_options* opt);

/* Registers a context (with its pair list) as system *id.  The server neither copies nor
 * frees it: the context must outlive the server and must not be rebuilt meanwhile.  Its
 * device bytes count against the budget (HFX_ERR_ADMISSION if they do not fit).
 * Synchronises the context's stream. */
int hfx_server_add_system(hfx_server* srv, hfx_ctx* ctx, int* id);

/* Queues K = K(P) for system `id`.  P (n_bf x n_bf, row-major, ld = n_bf) and K_out (same
 * shape) are device pointers or page-locked host pointers (pageable host memory is refused
 * with HFX_ERR_ARG, because copies to and from it would block the server).  P must stay
 * valid until the request is admitted and K_out until it is done.  The server waits for
 * the work queued on `stream` (the stream that produced P; NULL = legacy default stream)
 * before it reads P.  *ticket identifies the request.  Errors: HFX_ERR_ARG,
 * HFX_ERR_ADMISSION. */
int hfx_serve_submit(hfx_server* srv, int id, const double* P, double* K_out, void* stream, uint64_t* ticket);

/* Drives the server and reports the request's state in *out without waiting. */
int hfx_serve_poll(hfx_server* srv, uint64_t ticket, hfx_result* out);

/* Drives the server until the request is done or failed, or timeout_ms (< 0: no limit)
 * passes (then HFX_ERR_TIMEOUT, with the request still queued or running). */
int hfx_serve_wait(hfx_server* srv, uint64_t ticket, double timeout_ms, hfx_result* out);

/* Forgets a finished (done or failed) request: its ticket becomes unknown.  The server
 * keeps every finished request's result until this call, so long-running callers release
 * each ticket after reading it.  Errors: HFX_ERR_ARG (unknown ticket), HFX_ERR_STATE (still
 * queued or running). */
int hfx_serve_release(hfx_server* srv, uint64_t ticket);

/* Retires finished steps and starts new ones; returns the number of requests not done. */
int hfx_serve_progress(hfx_server* srv);

/* Drives the server until every request is done (HFX_ERR_TIMEOUT after timeout_ms >= 0). */
int hfx_serve_drain(hfx_server* srv, double timeout_ms);

int hfx_server_get_stats(hfx_server* srv, hfx_server_stats* out);
const char* hfx_server_last_error(const hfx_server* srv);

/* Waits for every step, then frees the server's own memory (not the contexts). */
void hfx_server_free(hfx_server* srv);

/* Largest matrix order accepted by hfx_energy_noalloc (rows of its fixed scratch). */
#define HFX_NOALLOC_MAX_N 16384

/* E = sum_{mu nu} P_{mu nu} K_{mu nu} for device matrices P and K (n x n, leading
 * dimension ld), written to the device scalar *E_dev, with NO device allocation: for
 * callers that cannot let a library call cudaMalloc (programs that serve all device
 * memory from their own pool or under a fixed budget, or loops where an allocation
 * would synchronise the device).  The paper has no counterpart of this entry point.
 * Scratch: a fixed library-resident device array of 2 * HFX_NOALLOC_MAX_N doubles
 * (256 KiB) on every device that loads the library, kept until process exit.  The
 * first call on a device looks up that array's address (make it before any stream
 * capture) and keeps it for the process: it assumes the device's primary context (the
 * one the CUDA runtime uses) and no cudaDeviceReset in the process afterwards.  Calls
 * share the array: calls that overlap on the GPU race, so order them (e.g. one stream).
 * Each call writes all scratch it reads; nothing needs clearing.
 * Work is queued on `stream` (cudaStream_t, NULL = default).  Errors: HFX_ERR_ARG for
 * NULL pointers, n < 1, n > HFX_NOALLOC_MAX_N or ld < n (message via
 * hfx_last_error(NULL)); HFX_ERR_CUDA if the address lookup or a launch fails. */
int hfx_energy_noalloc(const double* P_dev, const double* K_dev, int n, int ld, double* E_dev, void* stream);

/* Failure injection for tests (host side: no GPU fault is made): the k-th device
 * allocation a context makes from now on (k >= 1) fails as if cudaMalloc had returned an
 * out-of-memory error, so the calling entry point returns HFX_ERR_OOM and releases what it
 * holds; k = 0 disarms.  Process-wide.  Errors: HFX_ERR_ARG for k < 0. */
int hfx_debug_fail_alloc(int k);

/* Measures the FP64 and FP32 fused-multiply-add throughput of the current device with
 * a register-resident FMA chain (TFLOP/s, FMA = 2 flops).  Used as the roofline
 * denominators for the FP64/FP32 ALU-bound kernels. */
int hfx_measure_fma_peak(double* fp64_tflops, double* fp32_tflops);

/* Times (ms) the same FP64 FMA-chain kernel with all 32 lanes of every warp active and with
 * one lane active: equal times show that the FP64 pipe charges each warp instruction in full
 * whatever the number of active lanes, the property the ERI kernels are laid out around. */
int hfx_measure_fp64_lane_cost(double* ms_all_lanes, double* ms_one_lane);

/* ------------------------------------------------------------------------------------
 * NAO -> GTO fit (paper Sec. "NAO2GTO scheme" and Algorithm 1).  A numerical radial
 * function phi (angular momentum l) sampled on the grid r_i = i h, i = 1..n_r, is expanded as
 *   chi(r) = sum_m D_m r^l exp(-alpha_m r^2),  m = 1..M  (M = n_gauss),
 * with alpha, D minimising err = sum_i (sum_m D_m exp(-alpha_m r_i^2) - phi(r_i)/r_i^l)^2 under
 * alpha_m >= alpha_min.  Algorithm 1: n_restarts times, a constrained genetic search gives a
 * starting point and a constrained local search refines it; the restart with the smallest err
 * is kept (the first one on ties).  The two searches are the paper's in name only (it does not
 * spell them out); how they are read here is stated in csrc/hfx_nao.cu.  One warp per restart,
 * FP64 throughout.  Random draws: SplitMix64 (Steele, Lea and Flood 2014) as a
 * counter-based generator from `seed`.
 *
 * Layouts (all device arrays, row-major, caller-owned; the library allocates nothing):
 *   phi   n_fun x n_r      l  n_fun ints (0..6)
 *   per restart q = f * n_restarts + iter:  r_alpha, r_D  (n_fun * n_restarts) x M,
 *   r_err n_fun * n_restarts, r_steps (n_fun * n_restarts) x 2 ints (trial steps of the
 *   local search, Jacobian evaluations) or NULL, r_ga_err the err after the genetic step or NULL
 *   best per function: alpha, D  n_fun x M, err n_fun.  Exponents come out ascending.
 * Limits: 1 <= n_r <= 1024, 1 <= n_gauss <= 6, 2 <= population <= 64; n_fun = 0 is a no-op
 * (its pointers may then be NULL).  Work is queued on
 * `stream` (cudaStream_t, NULL = default).  Errors: HFX_ERR_ARG (NULL pointer, a size or an
 * option out of range; message via hfx_last_error(NULL)), HFX_ERR_CUDA (launch failed). */
typedef struct {
  int n_gauss;             /* M: Gaussians per radial function, 1..6 */
  int n_restarts;          /* N: iterations of Algorithm 1 per function (the paper: > 500) */
  int population;          /* P: genetic-search population, 2..64 */
  int generations;         /* G: genetic-search generations, >= 0 */
  int max_iter;            /* trial steps of the local search, >= 0 */
  double alpha_min;        /* lower bound of the exponents (the paper: 0.1) */
  double alpha_max;        /* upper end of the genetic search's box (> alpha_min) */
  unsigned long long seed; /* of the counter-based draws */
} hfx_nao_options;

/* M 3, N 512, P 32, G 30, max_iter 100, alpha_min 0.1, alpha_max 1000, a fixed seed. */
void hfx_nao_default_options(hfx_nao_options* opt);

/* The whole of Algorithm 1 for n_fun functions: genetic step, local search, selection. */
int hfx_nao_fit(const double* phi, const int* l, int n_fun, int n_r, double h, const hfx_nao_options* opt,
                double* alpha, double* D, double* err, double* r_alpha, double* r_D, double* r_err, int* r_steps,
                double* r_ga_err, void* stream);

/* Its first step alone: per restart the best individual of the genetic search, alpha and the
 * projected D (the least-squares D for that alpha) with its err. */
int hfx_nao_genetic(const double* phi, const int* l, int n_fun, int n_r, double h, const hfx_nao_options* opt,
                    double* alpha, double* D, double* err, void* stream);

/* Its second step alone: the local search started from alpha, D (per restart, updated in
 * place), err out; steps as r_steps above, or NULL. */
int hfx_nao_local(const double* phi, const int* l, int n_fun, int n_r, double h, const hfx_nao_options* opt,
                  double* alpha, double* D, double* err, int* steps, void* stream);

/* The genetic search's fitness for given exponent sets: for set s (function fun_of_set[s],
 * exponents alpha[s * n_gauss ..]) the least-squares D (ridged normal equations, Cholesky;
 * D = 0 if the factorisation fails) and err at it.  A set whose function index is outside
 * 0..n_fun-1 gets NaN for D and err. */
int hfx_nao_project(const double* phi, const int* l, int n_fun, int n_r, double h, int n_gauss, int n_set,
                    const int* fun_of_set, const double* alpha, double* D, double* err, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HFX_H */
