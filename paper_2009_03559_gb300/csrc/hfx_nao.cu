// NAO -> GTO fit on the GPU (paper Sec. "NAO2GTO scheme": the expansion
//   chi(r) = sum_m D_m r^l exp(-alpha_m r^2),  m = 1..M,
// of a numerical radial function phi, fitted by minimising the residual sum of squares
//   err = sum_i (chi(r_i)/r_i^l - phi(r_i)/r_i^l)^2 = sum_i (sum_m D_m e^{-alpha_m r_i^2} - y_i)^2
// under alpha_m >= alpha_min; Algorithm 1: N restarts, each a constrained genetic search for a
// starting point followed by a constrained local search, the restart with the smallest err kept).
//
// Layout: one warp runs one restart; its lanes share the radial grid r_i = i h (lane j owns the
// points i = j + 1 + 32 t), so every sum over the grid is a per-lane partial sum followed by one
// warp reduction.  Everything is FP64.  Per warp, shared memory holds the targets y_i, the
// reduction scratch, a dense system for the local search and the genetic search's two
// populations.  The genetic step and the local search are separate kernels (each gets its own
// register budget); a third picks the best restart per function.
//
// Gaussians on the grid: for an exponent a and beta = a h^2, exp(-beta i^2) moves along one lane's
// points (i -> i + 32) by the factor exp(-beta (64 i + 1024)), and that factor by exp(-2048 beta):
// two exp() calls per Gaussian and lane plus the lane-independent one, then two multiplies per
// point (the local search).  In the genetic step an individual's alpha = exp(u) and the factors
// exp(-beta), exp(-64 beta), exp(-1024 beta) are made once, by the lane that makes the
// individual, and kept with its genes; a lane's start values are then products over the lanes
// below it (warp product scans), so evaluating an individual calls no exp().
//
// The paper names the two searches but does not spell them out; the readings (shared with the
// CPU reference the tests compare against) are:
//  * genetic search on u_m = ln alpha_m in [ln alpha_min, ln alpha_max]: population P with sorted
//    genes, G generations; fitness = err at the variable-projection D (normal equations of the
//    linear least-squares problem for fixed alpha, relative ridge 1e-12 on the diagonal, Cholesky;
//    a failed factorisation gives D = 0); elitism; binary tournaments in which the second
//    contestant wins only if its fitness is lower by more than a relative 1e-12; blend crossover
//    c = a + w (b - a), w uniform in [-0.25, 1.25); per gene with probability 0.1 a uniform
//    mutation step in [-0.5, 0.5); reflection into the box; sorting;
//  * local search over (alpha, D), Levenberg-Marquardt form of a trust-region method: the step
//    solves (H + lambda diag H) delta = -g, H = J^T J, g = J^T res; exponents on the bound whose
//    gradient points outwards are held, the trial point is projected onto alpha >= alpha_min;
//    accepted if err drops by more than a relative 1e-12 (lambda / 3), else lambda x 4; stop
//    after a relative decrease below 1e-10, at lambda > 1e10 or after max_iter trial steps;
//  * random draws: SplitMix64 (Steele, Lea and Flood 2014) used as a counter-based generator:
//    draw c of seed s is the generator's output number c, mix(s + (c + 1) * 0x9E3779B97F4A7C15),
//    as a double from its top 53 bits; the counter of slot k of individual j in generation g
//    (0: the initial population) of restart q is ((q (G + 1) + g) P + j) (4 + 2M) + k.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "hfx.h"

namespace hfx {
void set_global_error(const std::string& msg);
}

namespace {

constexpr int kMaxM = 6;
constexpr int kMaxUnknowns = 2 * kMaxM;
constexpr int kMatLd = kMaxUnknowns + 1;
constexpr int kMatDoubles = kMaxUnknowns * kMatLd + kMatLd;  // matrix + right-hand side
constexpr int kMaxNr = 1024;
constexpr int kMaxPop = 64;
constexpr int kWarps = 4;  // warps (restarts) per block at most
constexpr size_t kMaxBlockSmem = 227 * 1024;

constexpr double kRidge = 1e-12;
constexpr double kTieFactor = 1.0 - 1e-12;
constexpr double kConv = 1e-10;
constexpr double kLambda0 = 1e-3;
constexpr double kLambdaMax = 1e10;
constexpr double kPMut = 0.1;
constexpr double kMutStep = 0.5;

struct NaoArgs {
  const double* phi;  // n_fun x n_r
  const int* l;       // n_fun
  int n_fun, n_r, npad;
  double h;
  int N, P, G, max_iter;
  double alpha_min, lo, hi;  // lo, hi = ln alpha_min, ln alpha_max
  unsigned long long seed;
  // genetic kernel outputs / local kernel inputs and outputs (per restart)
  double* alpha;  // n_fun N x M
  double* D;      // n_fun N x M
  double* err;    // n_fun N
  int* steps;     // n_fun N x 2 (trial steps, Jacobian passes), or NULL
  double* ga_err; // n_fun N fitness after the genetic step, or NULL
  // projection kernel
  int n_set;
  const int* fun_of_set;
  const double* set_alpha;
  double* set_D;
  double* set_err;
};

__host__ __device__ constexpr int n_tri(int m) { return m * (m + 1) / 2; }
// reduction scratch rows: A0, A1, A2 (three triangles), two gradients, one spare
__host__ __device__ constexpr int n_red(int m) { return 3 * n_tri(m) + 2 * m + 1; }

__host__ __device__ inline int warp_smem_doubles(int M, int npad, int P) {
  return npad + n_red(M) * 33 + kMatDoubles + 10 * P * M + 2 * P;
}

// pop: genes u_m = ln alpha_m; al: alpha_m; fac: per Gaussian exp(-beta), exp(-64 beta) and
// exp(-1024 beta), beta = alpha_m h^2, the factors of the grid recurrence (made once per
// individual by the lane that makes it)
struct WarpMem {
  double* y;
  double* red;
  double* mat;
  double* pop[2];
  double* al[2];
  double* fac[2];
  double* fit[2];
};

__device__ __forceinline__ WarpMem warp_mem(int M, int npad, int P) {
  extern __shared__ double smem[];
  const int w = threadIdx.x >> 5;
  double* base = smem + (size_t)w * warp_smem_doubles(M, npad, P);
  WarpMem m;
  m.y = base;
  m.red = m.y + npad;
  m.mat = m.red + n_red(M) * 33;
  m.pop[0] = m.mat + kMatDoubles;
  m.pop[1] = m.pop[0] + P * M;
  m.al[0] = m.pop[1] + P * M;
  m.al[1] = m.al[0] + P * M;
  m.fac[0] = m.al[1] + P * M;
  m.fac[1] = m.fac[0] + 3 * P * M;
  m.fit[0] = m.fac[1] + 3 * P * M;
  m.fit[1] = m.fit[0] + P;
  return m;
}

// y_i = phi(r_i) / r_i^l on the padded grid (zero beyond n_r)
__device__ __forceinline__ void load_targets(const NaoArgs& A, int f, double* y, int lane) {
  const int l = __ldg(A.l + f);
  for (int i0 = lane; i0 < A.npad; i0 += 32) {
    double v = 0.0;
    if (i0 < A.n_r) {
      const double r = A.h * (double)(i0 + 1);
      double rl = 1.0;
      for (int k = 0; k < l; ++k) rl *= r;
      v = __ldg(A.phi + (size_t)f * A.n_r + i0) / rl;
    }
    y[i0] = v;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Counter-based draws
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long c) {
  unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(unsigned long long seed, unsigned long long c) {
  return (double)(splitmix64(seed, c) >> 11) * (1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------------------
// Warp sums: lanes' partials -> every lane holds the totals (one lane adds each row, so the
// totals are bitwise the same on every lane and every decision taken on them is warp-uniform)
// ---------------------------------------------------------------------------
// totals left in red[k * 33 + 32]
template <int NV>
__device__ __forceinline__ void warp_sum_smem(const double (&v)[NV], double* red, int lane) {
#pragma unroll
  for (int k = 0; k < NV; ++k) red[k * 33 + lane] = v[k];
  __syncwarp();
  for (int k = lane; k < NV; k += 32) {
    const double* row = red + k * 33;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
      s0 += row[j];
      s1 += row[j + 1];
      s2 += row[j + 2];
      s3 += row[j + 3];
    }
    red[k * 33 + 32] = (s0 + s1) + (s2 + s3);
  }
  __syncwarp();
}

template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV], double* red, int lane) {
  warp_sum_smem<NV>(v, red, lane);
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = red[k * 33 + 32];
  __syncwarp();
}

__device__ __forceinline__ double warp_sum1(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);  // lane 0's order for everyone
}

// inclusive product of v over lanes 0..lane
__device__ __forceinline__ double scan_mul(double v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v *= t;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Gaussians along one lane's grid points
// ---------------------------------------------------------------------------
template <int M>
struct LaneGauss {
  double e[M], c[M], d[M];
  __device__ __forceinline__ void init(const double (&alpha)[M], double h2, int lane) {
    const double i0 = (double)(lane + 1);
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const double beta = alpha[m] * h2;
      e[m] = exp(-beta * (i0 * i0));
      c[m] = exp(-beta * (64.0 * i0 + 1024.0));
      d[m] = exp(-2048.0 * beta);
    }
  }
  // the same from the lane-independent factors f = (exp(-beta), exp(-64 beta), exp(-1024 beta))
  // per Gaussian, by product scans over the lanes: with a = exp(-beta), lane j's first point
  // i0 = j + 1 has exp(-beta i0^2) = prod_{k <= j} a^{2k+1} and exp(-beta (64 i0 + 1024)) =
  // exp(-1024 beta) exp(-64 beta)^{j+1}; the step factor is exp(-1024 beta)^2
  __device__ __forceinline__ void init_scan(const double* f, int lane) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const double a = f[3 * m], q = f[3 * m + 1], s = f[3 * m + 2];
      const double r = a * scan_mul(lane == 0 ? 1.0 : a * a, lane);  // a^{2 lane + 1}
      e[m] = scan_mul(r, lane);
      c[m] = s * scan_mul(q, lane);
      d[m] = s * s;
    }
  }
  __device__ __forceinline__ void step() {
#pragma unroll
    for (int m = 0; m < M; ++m) {
      e[m] *= c[m];
      c[m] *= d[m];
    }
  }
};

// err(alpha, D) over the warp's grid, given the lane's Gaussian state at its first point
template <int M>
__device__ __forceinline__ double residual(LaneGauss<M> g, const double (&D)[M], const NaoArgs& A, const double* y,
                                           int lane) {
  double s = 0.0;
  const int T = A.npad >> 5;
  for (int t = 0; t < T; ++t) {
    const int i0 = lane + 32 * t;
    const bool valid = i0 < A.n_r;
    double f = 0.0;
#pragma unroll
    for (int m = 0; m < M; ++m) f = fma(D[m], valid ? g.e[m] : 0.0, f);
    const double res = f - y[i0];
    s = fma(res, res, s);
    g.step();
  }
  return warp_sum1(s);
}

// Cholesky solve of a small SPD system held in registers (every lane the same), packed lower
// triangle a[i (i + 1) / 2 + j]; false on a pivot that is not positive.
template <int N>
__device__ __forceinline__ bool chol_solve_reg(double (&a)[n_tri(N)], double (&b)[N]) {
  double rd[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    double s = a[n_tri(j) + j];
#pragma unroll
    for (int k = 0; k < j; ++k) s = fma(-a[n_tri(j) + k], a[n_tri(j) + k], s);
    if (!(s > 0.0)) return false;
    rd[j] = rsqrt(s);  // the solves need only 1 / L_jj
#pragma unroll
    for (int i = j + 1; i < N; ++i) {
      double t = a[n_tri(i) + j];
#pragma unroll
      for (int k = 0; k < j; ++k) t = fma(-a[n_tri(i) + k], a[n_tri(j) + k], t);
      a[n_tri(i) + j] = t * rd[j];
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double t = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t = fma(-a[n_tri(i) + k], b[k], t);
    b[i] = t * rd[i];
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    double t = b[i];
#pragma unroll
    for (int k = i + 1; k < N; ++k) t = fma(-a[n_tri(k) + i], b[k], t);
    b[i] = t * rd[i];
  }
  return true;
}

// Variable projection: D minimising err for fixed alpha (ridged normal equations), and err there.
template <int M>
__device__ __forceinline__ double project(const double (&alpha)[M], double (&D)[M], const NaoArgs& A,
                                          const WarpMem& wm, int lane, const double* fac = nullptr) {
  constexpr int NA = n_tri(M);
  LaneGauss<M> g0;
  if (fac)
    g0.init_scan(fac, lane);
  else
    g0.init(alpha, A.h * A.h, lane);
  LaneGauss<M> g = g0;
  double acc[NA + M];
#pragma unroll
  for (int k = 0; k < NA + M; ++k) acc[k] = 0.0;
  const int T = A.npad >> 5;
  for (int t = 0; t < T; ++t) {
    const int i0 = lane + 32 * t;
    const bool valid = i0 < A.n_r;
    const double yv = wm.y[i0];
    double ev[M];
#pragma unroll
    for (int m = 0; m < M; ++m) ev[m] = valid ? g.e[m] : 0.0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
#pragma unroll
      for (int j = 0; j <= i; ++j) acc[n_tri(i) + j] = fma(ev[i], ev[j], acc[n_tri(i) + j]);
      acc[NA + i] = fma(yv, ev[i], acc[NA + i]);
    }
    g.step();
  }
  warp_sum(acc, wm.red, lane);
  double a[NA];
#pragma unroll
  for (int i = 0; i < M; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) a[n_tri(i) + j] = acc[n_tri(i) + j];
    a[n_tri(i) + i] += kRidge * acc[n_tri(i) + i];
    D[i] = acc[NA + i];
  }
  if (!chol_solve_reg<M>(a, D)) {
#pragma unroll
    for (int m = 0; m < M; ++m) D[m] = 0.0;
  }
  return residual<M>(g0, D, A, wm.y, lane);
}

// ---------------------------------------------------------------------------
// Genetic step (one warp per restart)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool better(double fa, double fb) { return fa < fb * kTieFactor; }

__device__ __forceinline__ int best_index(const double* fit, int P) {
  int b = 0;
  for (int j = 1; j < P; ++j)
    if (better(fit[j], fit[b])) b = j;
  return b;
}

template <int M>
__device__ __forceinline__ void sort_genes(double (&u)[M]) {
#pragma unroll
  for (int i = 1; i < M; ++i) {
#pragma unroll
    for (int j = i; j > 0; --j) {
      if (u[j] < u[j - 1]) {
        const double t = u[j];
        u[j] = u[j - 1];
        u[j - 1] = t;
      }
    }
  }
}

__device__ __forceinline__ double reflect_box(double c, double lo, double hi) {
  if (c < lo) c = __dsub_rn(__dmul_rn(2.0, lo), c);
  if (c > hi) c = __dsub_rn(__dmul_rn(2.0, hi), c);
  return fmin(fmax(c, lo), hi);
}

template <int M>
__device__ __forceinline__ double eval_individual(const double* al, const double* fac, const NaoArgs& A,
                                                  const WarpMem& wm, int lane) {
  double alpha[M], D[M];
#pragma unroll
  for (int m = 0; m < M; ++m) alpha[m] = al[m];
  return project<M>(alpha, D, A, wm, lane, fac);
}

// alpha = exp(u) and the grid-recurrence factors of one individual, into shared memory
template <int M>
__device__ __forceinline__ void store_individual(const double (&u)[M], double h2, double* pop, double* al,
                                                 double* fac) {
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const double a = exp(u[m]);
    const double beta = a * h2;
    pop[m] = u[m];
    al[m] = a;
    fac[3 * m] = exp(-beta);
    fac[3 * m + 1] = exp(-64.0 * beta);
    fac[3 * m + 2] = exp(-1024.0 * beta);
  }
}

template <int M>
__global__ void __launch_bounds__(kWarps * 32) nao_genetic_kernel(NaoArgs A) {
  const int lane = threadIdx.x & 31;
  const long long q = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= (long long)A.n_fun * A.N) return;  // whole warps leave together
  const int f = (int)(q / A.N);
  const int P = A.P, G = A.G;
  constexpr int S = 4 + 2 * M;
  const WarpMem wm = warp_mem(M, A.npad, P);
  load_targets(A, f, wm.y, lane);
  auto ctr = [&](int g, int j, int k) -> unsigned long long {
    return (((unsigned long long)q * (unsigned long long)(G + 1) + (unsigned long long)g) * (unsigned long long)P +
            (unsigned long long)j) * (unsigned long long)S + (unsigned long long)k;
  };
  const double span = __dsub_rn(A.hi, A.lo);
  const double h2 = A.h * A.h;
  // initial population
  for (int j = lane; j < P; j += 32) {
    double u[M];
#pragma unroll
    for (int m = 0; m < M; ++m) u[m] = __dadd_rn(A.lo, __dmul_rn(uniform01(A.seed, ctr(0, j, m)), span));
    sort_genes<M>(u);
    store_individual<M>(u, h2, wm.pop[0] + j * M, wm.al[0] + j * M, wm.fac[0] + 3 * j * M);
  }
  __syncwarp();
  for (int j = 0; j < P; ++j) {
    const double fj = eval_individual<M>(wm.al[0] + j * M, wm.fac[0] + 3 * j * M, A, wm, lane);
    if (lane == 0) wm.fit[0][j] = fj;
  }
  __syncwarp();
  int cur = 0;
  for (int g = 1; g <= G; ++g) {
    const double* pop = wm.pop[cur];
    const double* fit = wm.fit[cur];
    double* npop = wm.pop[cur ^ 1];
    double* nal = wm.al[cur ^ 1];
    double* nfac = wm.fac[cur ^ 1];
    double* nfit = wm.fit[cur ^ 1];
    const int e = best_index(fit, P);
    for (int j = lane; j < P; j += 32) {
      if (j == 0) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
          npop[m] = pop[e * M + m];
          nal[m] = wm.al[cur][e * M + m];
          for (int k = 0; k < 3; ++k) nfac[3 * m + k] = wm.fac[cur][3 * (e * M + m) + k];
        }
        nfit[0] = fit[e];
        continue;
      }
      double U[S];
#pragma unroll
      for (int k = 0; k < S; ++k) U[k] = uniform01(A.seed, ctr(g, j, k));
      auto tournament = [&](double u1, double u2) {
        const int i1 = min((int)(u1 * (double)P), P - 1);
        const int i2 = min((int)(u2 * (double)P), P - 1);
        return better(fit[i2], fit[i1]) ? i2 : i1;
      };
      const double* a = pop + tournament(U[0], U[1]) * M;
      const double* b = pop + tournament(U[2], U[3]) * M;
      double c[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const double w = __dadd_rn(-0.25, __dmul_rn(1.5, U[4 + m]));
        double v = __dadd_rn(a[m], __dmul_rn(w, __dsub_rn(b[m], a[m])));
        const double r = U[4 + M + m];
        if (r < kPMut) v = __dadd_rn(v, __dmul_rn(kMutStep, __dsub_rn(__dmul_rn(2.0, __ddiv_rn(r, kPMut)), 1.0)));
        c[m] = reflect_box(v, A.lo, A.hi);
      }
      sort_genes<M>(c);
      store_individual<M>(c, h2, npop + j * M, nal + j * M, nfac + 3 * j * M);
    }
    __syncwarp();
    for (int j = 1; j < P; ++j) {
      const double fj = eval_individual<M>(nal + j * M, nfac + 3 * j * M, A, wm, lane);
      if (lane == 0) nfit[j] = fj;
    }
    __syncwarp();
    cur ^= 1;
  }
  const int e = best_index(wm.fit[cur], P);
  double alpha[M], D[M];
#pragma unroll
  for (int m = 0; m < M; ++m) alpha[m] = wm.al[cur][e * M + m];
  const double fe = project<M>(alpha, D, A, wm, lane, wm.fac[cur] + 3 * e * M);
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
      A.alpha[q * M + m] = alpha[m];
      A.D[q * M + m] = D[m];
    }
    if (A.ga_err) A.ga_err[q] = fe;
    A.err[q] = fe;
  }
}

// ---------------------------------------------------------------------------
// Local search (one warp per restart), started from A.alpha / A.D, results written in place
// ---------------------------------------------------------------------------
// Lane-parallel Cholesky solve of the n x n system in shared memory (lower triangle, row stride
// kMatLd; right-hand side after the matrix); false, uniformly, on a pivot that is not positive.
__device__ bool chol_solve_smem(double* mat, int n, int lane) {
  double* rhs = mat + kMaxUnknowns * kMatLd;
  for (int k = 0; k < n; ++k) {
    __syncwarp();
    const double akk = mat[k * kMatLd + k];
    if (!(akk > 0.0)) return false;
    const double dk = sqrt(akk), rk = 1.0 / dk;
    __syncwarp();
    for (int i = k + 1 + lane; i < n; i += 32) mat[i * kMatLd + k] *= rk;
    if (lane == 0) mat[k * kMatLd + k] = dk;
    __syncwarp();
    for (int i = k + 1 + lane; i < n; i += 32) {
      const double lik = mat[i * kMatLd + k];
      for (int j = k + 1; j <= i; ++j) mat[i * kMatLd + j] = fma(-lik, mat[j * kMatLd + k], mat[i * kMatLd + j]);
    }
  }
  __syncwarp();
  for (int k = 0; k < n; ++k) {
    const double zk = rhs[k] / mat[k * kMatLd + k];
    __syncwarp();
    if (lane == 0) rhs[k] = zk;
    for (int i = k + 1 + lane; i < n; i += 32) rhs[i] = fma(-mat[i * kMatLd + k], zk, rhs[i]);
    __syncwarp();
  }
  for (int k = n - 1; k >= 0; --k) {
    const double xk = rhs[k] / mat[k * kMatLd + k];
    __syncwarp();
    if (lane == 0) rhs[k] = xk;
    for (int i = lane; i < k; i += 32) rhs[i] = fma(-mat[k * kMatLd + i], xk, rhs[i]);
    __syncwarp();
  }
  return true;
}

template <int M>
__global__ void __launch_bounds__(kWarps * 32) nao_local_kernel(NaoArgs A) {
  const int lane = threadIdx.x & 31;
  const long long q = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= (long long)A.n_fun * A.N) return;
  const int f = (int)(q / A.N);
  constexpr int NA = n_tri(M);
  constexpr int NU = 2 * M;
  constexpr int NS = 3 * NA + 2 * M;  // sums of one Jacobian pass
  const WarpMem wm = warp_mem(M, A.npad, A.P);
  load_targets(A, f, wm.y, lane);
  const double h2 = A.h * A.h;
  double xa[M], xd[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    xa[m] = A.alpha[q * M + m];
    xd[m] = A.D[q * M + m];
  }
  LaneGauss<M> g;
  g.init(xa, h2, lane);
  double E = residual<M>(g, xd, A, wm.y, lane);
  double lam = kLambda0;
  bool needJ = true;
  int it = 0, jpass = 0;
  // after a Jacobian pass its sums stay in the reduction scratch (row k at red[k * 33 + 32]):
  // k < NA: sum e_a e_b; NA..2NA: sum r^2 e_a e_b; 2NA..3NA: sum r^4 e_a e_b (a >= b, packed);
  // 3NA + m: sum e_m res; 3NA + M + m: sum r^2 e_m res
  const double* Sum = wm.red + 32;
  double* mat = wm.mat;
  unsigned act = 0;
  double hfloor = 0.0;
  double gvec[NU];
#pragma unroll
  for (int k = 0; k < NU; ++k) gvec[k] = 0.0;
  while (it < A.max_iter) {
    if (needJ) {
      ++jpass;
      double acc[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) acc[k] = 0.0;
      LaneGauss<M> gg;
      gg.init(xa, h2, lane);
      const int T = A.npad >> 5;
      for (int t = 0; t < T; ++t) {
        const int i0 = lane + 32 * t;
        const bool valid = i0 < A.n_r;
        const double r = A.h * (double)(i0 + 1);
        const double r2 = r * r, r4 = r2 * r2;
        double ev[M];
        double fv = 0.0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          ev[m] = valid ? gg.e[m] : 0.0;
          fv = fma(xd[m], ev[m], fv);
        }
        const double res = valid ? fv - wm.y[i0] : 0.0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
#pragma unroll
          for (int j = 0; j <= i; ++j) {
            const double p = ev[i] * ev[j];
            acc[n_tri(i) + j] += p;
            acc[NA + n_tri(i) + j] = fma(r2, p, acc[NA + n_tri(i) + j]);
            acc[2 * NA + n_tri(i) + j] = fma(r4, p, acc[2 * NA + n_tri(i) + j]);
          }
          const double qv = res * ev[i];
          acc[3 * NA + i] += qv;
          acc[3 * NA + M + i] = fma(r2, qv, acc[3 * NA + M + i]);
        }
        gg.step();
      }
      warp_sum_smem<NS>(acc, wm.red, lane);
      // g = J^T res: d/d alpha_m = -D_m sum r^2 e_m res, d/d D_m = sum e_m res
      double dmax = 0.0;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        gvec[m] = -xd[m] * Sum[(3 * NA + M + m) * 33];
        gvec[M + m] = Sum[(3 * NA + m) * 33];
        dmax = fmax(dmax, xd[m] * xd[m] * Sum[(2 * NA + n_tri(m) + m) * 33]);
        dmax = fmax(dmax, Sum[(n_tri(m) + m) * 33]);
      }
      hfloor = 1e-12 * dmax;  // damping floor: a relative 1e-12 of the largest diagonal of H
      act = 0;
#pragma unroll
      for (int m = 0; m < M; ++m)
        if (xa[m] <= A.alpha_min && gvec[m] > 0.0) act |= 1u << m;
      needJ = false;
    }
    ++it;
    // the damped system H + lambda diag(max(H_kk, floor)), held exponents as identity rows
    if (lane == 0) {
#pragma unroll
      for (int a = 0; a < NU; ++a) {
#pragma unroll
        for (int b = 0; b <= a; ++b) {
          const int ma = a % M, mb = b % M;
          const int ti = ma >= mb ? n_tri(ma) + mb : n_tri(mb) + ma;
          double h;
          if (a < M)                      // (alpha_a, alpha_b): D_a D_b sum r^4 e_a e_b
            h = xd[ma] * xd[mb] * Sum[(2 * NA + ti) * 33];
          else if (b >= M)                // (D_a, D_b): sum e_a e_b
            h = Sum[ti * 33];
          else                            // (D_a, alpha_b): -D_b sum r^2 e_a e_b
            h = -xd[mb] * Sum[(NA + ti) * 33];
          if (a == b) h += lam * fmax(h, hfloor);
          const bool held = (a < M && ((act >> a) & 1u)) || (b < M && ((act >> b) & 1u));
          if (held) h = (a == b) ? 1.0 : 0.0;
          mat[a * kMatLd + b] = h;
        }
        const bool held_a = a < M && ((act >> a) & 1u);
        mat[kMaxUnknowns * kMatLd + a] = held_a ? 0.0 : -gvec[a];
      }
    }
    __syncwarp();
    if (!chol_solve_smem(mat, NU, lane)) {
      lam *= 4.0;
      if (lam > kLambdaMax) break;
      continue;
    }
    double xta[M], xtd[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      xta[m] = fmax(xa[m] + mat[kMaxUnknowns * kMatLd + m], A.alpha_min);
      xtd[m] = xd[m] + mat[kMaxUnknowns * kMatLd + M + m];
    }
    __syncwarp();
    LaneGauss<M> gt;
    gt.init(xta, h2, lane);
    const double Et = residual<M>(gt, xtd, A, wm.y, lane);
    if (Et < E * kTieFactor) {
      const bool conv = (E - Et) <= kConv * E;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        xa[m] = xta[m];
        xd[m] = xtd[m];
      }
      E = Et;
      lam = fmax(lam / 3.0, 1e-12);
      needJ = true;
      if (conv) break;
    } else {
      lam *= 4.0;
      if (lam > kLambdaMax) break;
    }
  }
  // ascending exponents, coefficients along (stable)
#pragma unroll
  for (int i = 1; i < M; ++i) {
#pragma unroll
    for (int j = i; j > 0; --j) {
      if (xa[j] < xa[j - 1]) {
        double t = xa[j];
        xa[j] = xa[j - 1];
        xa[j - 1] = t;
        t = xd[j];
        xd[j] = xd[j - 1];
        xd[j - 1] = t;
      }
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
      A.alpha[q * M + m] = xa[m];
      A.D[q * M + m] = xd[m];
    }
    A.err[q] = E;
    if (A.steps) {
      A.steps[2 * q] = it;
      A.steps[2 * q + 1] = jpass;
    }
  }
}

// Algorithm 1's selection: per function the first restart with the smallest err.
__global__ void nao_best_kernel(int n_fun, int N, int M, const double* r_alpha, const double* r_D, const double* r_err,
                                double* alpha, double* D, double* err) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_fun) return;
  int b = 0;
  double be = r_err[(size_t)f * N];
  for (int n = 1; n < N; ++n) {
    const double e = r_err[(size_t)f * N + n];
    if (e < be) {
      be = e;
      b = n;
    }
  }
  const size_t q = (size_t)f * N + b;
  for (int m = 0; m < M; ++m) {
    alpha[(size_t)f * M + m] = r_alpha[q * M + m];
    D[(size_t)f * M + m] = r_D[q * M + m];
  }
  err[f] = be;
}

// Variable projection for given exponent sets (one warp per set).
template <int M>
__global__ void __launch_bounds__(kWarps * 32) nao_project_kernel(NaoArgs A) {
  const int lane = threadIdx.x & 31;
  const long long s = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (s >= A.n_set) return;
  const int f = __ldg(A.fun_of_set + s);
  if (f < 0 || f >= A.n_fun) {  // no such function: NaN out, nothing read
    if (lane == 0) {
#pragma unroll
      for (int m = 0; m < M; ++m) A.set_D[s * M + m] = __longlong_as_double(0x7ff8000000000000ll);
      A.set_err[s] = __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  const WarpMem wm = warp_mem(M, A.npad, A.P);
  load_targets(A, f, wm.y, lane);
  double alpha[M], D[M];
#pragma unroll
  for (int m = 0; m < M; ++m) alpha[m] = __ldg(A.set_alpha + s * M + m);
  const double e = project<M>(alpha, D, A, wm, lane);
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) A.set_D[s * M + m] = D[m];
    A.set_err[s] = e;
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
enum Which { kGenetic, kLocal, kProject };

template <int M>
const void* kernel_of(Which w) {
  switch (w) {
    case kGenetic: return (const void*)nao_genetic_kernel<M>;
    case kLocal: return (const void*)nao_local_kernel<M>;
    default: return (const void*)nao_project_kernel<M>;
  }
}

const void* kernel_for(int M, Which w) {
  switch (M) {
    case 1: return kernel_of<1>(w);
    case 2: return kernel_of<2>(w);
    case 3: return kernel_of<3>(w);
    case 4: return kernel_of<4>(w);
    case 5: return kernel_of<5>(w);
    default: return kernel_of<6>(w);
  }
}

int launch(Which w, int M, const NaoArgs& a, long long n_warps, cudaStream_t s) {
  if (n_warps <= 0) return HFX_OK;
  // up to kWarps restarts per block, as many as the shared memory of a block holds
  const size_t per_warp = (size_t)warp_smem_doubles(M, a.npad, a.P) * sizeof(double);
  const int warps = (int)std::max<size_t>(1, std::min<size_t>(kWarps, kMaxBlockSmem / per_warp));
  const size_t smem = warps * per_warp;
  const void* k = kernel_for(M, w);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    hfx::set_global_error(std::string("nao: shared memory request refused: ") + cudaGetErrorString(e));
    return HFX_ERR_CUDA;
  }
  const long long blocks = (n_warps + warps - 1) / warps;
  void* args[] = {(void*)&a};
  e = cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(warps * 32), args, smem, s);
  if (e != cudaSuccess) {
    hfx::set_global_error(std::string("nao: launch failed: ") + cudaGetErrorString(e));
    return HFX_ERR_CUDA;
  }
  return HFX_OK;
}

int check(const double* phi, const int* l, int n_fun, int n_r, double h, const hfx_nao_options* o, bool search,
          NaoArgs& a) {
  if (!o || (n_fun > 0 && (!phi || !l))) {
    hfx::set_global_error("nao: NULL pointer");
    return HFX_ERR_ARG;
  }
  if (n_fun < 0 || n_r < 1 || n_r > kMaxNr || !(h > 0.0) || o->n_gauss < 1 || o->n_gauss > kMaxM) {
    hfx::set_global_error("nao: need n_fun >= 0, 1 <= n_r <= 1024, h > 0, 1 <= n_gauss <= 6");
    return HFX_ERR_ARG;
  }
  if (search && (o->n_restarts < 1 || o->population < 2 || o->population > kMaxPop || o->generations < 0 ||
                 o->max_iter < 0 || !(o->alpha_min > 0.0) || !(o->alpha_max > o->alpha_min))) {
    hfx::set_global_error("nao: need n_restarts >= 1, 2 <= population <= 64, generations >= 0, max_iter >= 0, "
                          "0 < alpha_min < alpha_max");
    return HFX_ERR_ARG;
  }
  if ((long long)n_fun * (search ? o->n_restarts : 1) > (1ll << 30)) {
    hfx::set_global_error("nao: too many restarts");
    return HFX_ERR_ARG;
  }
  a = NaoArgs{};
  a.phi = phi;
  a.l = l;
  a.n_fun = n_fun;
  a.n_r = n_r;
  a.npad = (n_r + 31) & ~31;
  a.h = h;
  a.N = search ? o->n_restarts : 1;
  a.P = search ? o->population : 2;
  a.G = o->generations;
  a.max_iter = o->max_iter;
  a.alpha_min = o->alpha_min;
  a.lo = std::log(o->alpha_min);
  a.hi = std::log(o->alpha_max);
  a.seed = o->seed;
  return HFX_OK;
}

}  // namespace

extern "C" void hfx_nao_default_options(hfx_nao_options* o) {
  if (!o) return;
  o->n_gauss = 3;
  o->n_restarts = 512;
  o->population = 32;
  o->generations = 30;
  o->max_iter = 100;
  o->alpha_min = 0.1;
  o->alpha_max = 1000.0;
  o->seed = 0x5eedull;
}

extern "C" int hfx_nao_genetic(const double* phi, const int* l, int n_fun, int n_r, double h,
                               const hfx_nao_options* opt, double* alpha, double* D, double* err, void* stream) {
  NaoArgs a;
  int rc = check(phi, l, n_fun, n_r, h, opt, true, a);
  if (rc) return rc;
  if (n_fun > 0 && (!alpha || !D || !err)) {
    hfx::set_global_error("nao: NULL output");
    return HFX_ERR_ARG;
  }
  a.alpha = alpha;
  a.D = D;
  a.err = err;
  return launch(kGenetic, opt->n_gauss, a, (long long)n_fun * a.N, (cudaStream_t)stream);
}

extern "C" int hfx_nao_local(const double* phi, const int* l, int n_fun, int n_r, double h,
                             const hfx_nao_options* opt, double* alpha, double* D, double* err, int* steps,
                             void* stream) {
  NaoArgs a;
  int rc = check(phi, l, n_fun, n_r, h, opt, true, a);
  if (rc) return rc;
  if (n_fun > 0 && (!alpha || !D || !err)) {
    hfx::set_global_error("nao: NULL output");
    return HFX_ERR_ARG;
  }
  a.alpha = alpha;
  a.D = D;
  a.err = err;
  a.steps = steps;
  return launch(kLocal, opt->n_gauss, a, (long long)n_fun * a.N, (cudaStream_t)stream);
}

extern "C" int hfx_nao_fit(const double* phi, const int* l, int n_fun, int n_r, double h,
                           const hfx_nao_options* opt, double* alpha, double* D, double* err, double* r_alpha,
                           double* r_D, double* r_err, int* r_steps, double* r_ga_err, void* stream) {
  NaoArgs a;
  int rc = check(phi, l, n_fun, n_r, h, opt, true, a);
  if (rc) return rc;
  if (n_fun > 0 && (!alpha || !D || !err || !r_alpha || !r_D || !r_err)) {
    hfx::set_global_error("nao: NULL output");
    return HFX_ERR_ARG;
  }
  a.alpha = r_alpha;
  a.D = r_D;
  a.err = r_err;
  a.steps = r_steps;
  a.ga_err = r_ga_err;
  const long long nw = (long long)n_fun * a.N;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = launch(kGenetic, opt->n_gauss, a, nw, s))) return rc;
  if ((rc = launch(kLocal, opt->n_gauss, a, nw, s))) return rc;
  if (n_fun > 0) {
    nao_best_kernel<<<(n_fun + 127) / 128, 128, 0, s>>>(n_fun, a.N, opt->n_gauss, r_alpha, r_D, r_err, alpha, D, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      hfx::set_global_error(std::string("nao: launch failed: ") + cudaGetErrorString(e));
      return HFX_ERR_CUDA;
    }
  }
  return HFX_OK;
}

extern "C" int hfx_nao_project(const double* phi, const int* l, int n_fun, int n_r, double h, int n_gauss, int n_set,
                               const int* fun_of_set, const double* alpha, double* D, double* err, void* stream) {
  hfx_nao_options o;
  hfx_nao_default_options(&o);
  o.n_gauss = n_gauss;
  NaoArgs a;
  int rc = check(phi, l, n_fun, n_r, h, &o, false, a);
  if (rc) return rc;
  if (n_set < 0 || (n_set > 0 && (!fun_of_set || !alpha || !D || !err))) {
    hfx::set_global_error("nao: bad projection sets");
    return HFX_ERR_ARG;
  }
  a.n_set = n_set;
  a.fun_of_set = fun_of_set;
  a.set_alpha = alpha;
  a.set_D = D;
  a.set_err = err;
  return launch(kProject, n_gauss, a, n_set, (cudaStream_t)stream);
}
