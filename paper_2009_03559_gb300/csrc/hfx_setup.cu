// Set-up and finalisation kernels of the HFX library: basis normalisation, Boys table,
// shell-pair list (orbital cutoff, primitive-pair data), pair binning, quartet counting
// and prefix sums, K = A + A^T and the exchange energy tr(PK).
#include <cub/cub.cuh>
#include <thrust/iterator/counting_iterator.h>
#include <cmath>
#include "hfx_setup.h"

namespace hfx {

// ---------------------------------------------------------------------------
// Basis normalisation.  Radial part of shell s: R(r) = sum_k w_k exp(-alpha_k r^2) with
// w_k = N c_k alpha_k^{(2l+3)/4}; N makes int (S R)^2 = 1 for S = 1, x and xy
// (s, p, d), i.e. N^-2 = sum_{kl} wt_k wt_l (pi/g)^{3/2} (2g)^{-l}, g = alpha_k + alpha_l.
// The spherical d combinations used by the kernels all have the norm of xy.
// ---------------------------------------------------------------------------
__global__ void k_normalize(int n_shells, const int* __restrict__ l, const int* __restrict__ nprim,
                            const int* __restrict__ prim_off, const double* __restrict__ alpha,
                            const double* __restrict__ coef, double* __restrict__ w) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_shells) return;
  const int L = l[s], n = nprim[s], o = prim_off[s];
  double ov = 0.0;
  for (int k = 0; k < n; ++k) {
    const double wk = coef[o + k] * pow(alpha[o + k], 0.25 * (2 * L + 3));
    for (int kk = 0; kk < n; ++kk) {
      const double wkk = coef[o + kk] * pow(alpha[o + kk], 0.25 * (2 * L + 3));
      const double g = alpha[o + k] + alpha[o + kk];
      ov += wk * wkk * pow(M_PI / g, 1.5) * pow(2.0 * g, -(double)L);
    }
  }
  const double N = 1.0 / sqrt(ov);
  for (int k = 0; k < n; ++k) w[o + k] = N * coef[o + k] * pow(alpha[o + k], 0.25 * (2 * L + 3));
}

// ---------------------------------------------------------------------------
// Boys tables: at x_g = g h, F_15(x_g) from its series exp(-x) sum_k (2x)^k / ((31)(33)...(31+2k)),
// lower orders by the downward recursion F_{m-1} = (2x F_m + e^{-x}) / (2m-1); then for every
// order L = 0..kMaxLt the row of Taylor coefficients [x_g, (-1)^k F_{L+k}/k!, (-1)^k e^{-x_g}/k!].
// ---------------------------------------------------------------------------
__global__ void k_boys_table(double* __restrict__ tab) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= kBoysRows) return;
  const double x = g * kBoysStep;
  const int M = 15;
  double term = 1.0 / (2 * M + 1), sum = term;
  for (int k = 1; k < 4000; ++k) {
    term *= 2.0 * x / (2 * M + 2 * k + 1);
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  const double e = exp(-x);
  double Fm[M + 1];
  Fm[M] = e * sum;
  for (int m = M; m >= 1; --m) Fm[m - 1] = (2.0 * x * Fm[m] + e) / (2 * m - 1);
  const double inv_fact[7] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720};
  for (int L = 0; L <= kMaxLt; ++L) {
    double* row = tab + (size_t)L * kBoysTableLen + (size_t)g * kBoysRowLen;
    row[0] = x;
    for (int k = 0; k < 7; ++k) {
      const double sg = (k & 1) ? -inv_fact[k] : inv_fact[k];
      row[1 + k] = sg * Fm[L + k];
      row[8 + k] = sg * e;
    }
    row[15] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Shell pairs I >= J (triangular index t = I(I+1)/2 + J) passing the orbital cutoff:
// same atom, no cutoff (rcut <= 0), or |R_A - R_B| < 2 rcut.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tri_decode(long long t, int& I, int& J) {
  long long i = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  I = (int)i;
  J = (int)(t - i * (i + 1) / 2);
}

__global__ void k_pair_flags(long long n_tri, const int* __restrict__ atom, const double* __restrict__ xyz,
                             double rcut, int* __restrict__ flag) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tri) return;
  int I, J;
  tri_decode(t, I, J);
  int ok = 1;
  const int a = atom[I], b = atom[J];
  if (rcut > 0.0 && a != b) {
    const double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1],
                 dz = xyz[3 * a + 2] - xyz[3 * b + 2];
    ok = sqrt(dx * dx + dy * dy + dz * dz) < 2.0 * rcut;
  }
  flag[t] = ok;
}

// Periodic pair list: candidates t = s * n_img + u, s a home-cell shell (image index s), u
// any image shell; kept if the shells share an atom (same cell) or their atoms are closer
// than 2 rcut.
__global__ void k_pair_flags_rect(long long n, int n_img, const int* __restrict__ atom, const double* __restrict__ xyz,
                                  double rcut, int* __restrict__ flag) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int s = (int)(t / n_img), u = (int)(t - (long long)s * n_img);
  const int a = atom[s], b = atom[u];
  int ok = 1;
  if (a != b) {
    const double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1], dz = xyz[3 * a + 2] - xyz[3 * b + 2];
    ok = sqrt(dx * dx + dy * dy + dz * dz) < 2.0 * rcut;
  }
  flag[t] = ok;
}

__global__ void k_pair_setup_rect(int n_cand, const long long* __restrict__ cand_t, int n_img,
                                  const int* __restrict__ l, const int* __restrict__ nprim,
                                  const int* __restrict__ atom, const double* __restrict__ xyz, int* __restrict__ sa,
                                  int* __restrict__ sb, int* __restrict__ pcls, double* __restrict__ AB,
                                  int* __restrict__ cap, unsigned char* __restrict__ home_first) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cand) return;
  const long long t = cand_t[c];
  const int s = (int)(t / n_img), u = (int)(t - (long long)s * n_img);
  int a = s, b = u;
  unsigned char hf = 1;
  if (l[u] > l[s]) {
    a = u;
    b = s;
    hf = 0;
  }
  sa[c] = a;
  sb[c] = b;
  home_first[c] = hf;
  const int hi = l[a], lo = l[b];
  pcls[c] = hi * (hi + 1) / 2 + lo;
  for (int i = 0; i < 3; ++i) AB[3 * c + i] = xyz[3 * atom[a] + i] - xyz[3 * atom[b] + i];
  cap[c] = nprim[a] * nprim[b];
}

// Orientation (l_a >= l_b), pair class, AB and primitive capacity of each candidate.
__global__ void k_pair_setup(int n_cand, const long long* __restrict__ cand_t, const int* __restrict__ l,
                             const int* __restrict__ nprim, const int* __restrict__ atom,
                             const double* __restrict__ xyz, int* __restrict__ sa, int* __restrict__ sb,
                             int* __restrict__ pcls, double* __restrict__ AB, int* __restrict__ cap) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cand) return;
  int I, J;
  tri_decode(cand_t[c], I, J);
  int a = I, b = J;
  if (l[J] > l[I]) { a = J; b = I; }
  sa[c] = a;
  sb[c] = b;
  const int hi = l[a], lo = l[b];
  pcls[c] = hi * (hi + 1) / 2 + lo;
  for (int i = 0; i < 3; ++i) AB[3 * c + i] = xyz[3 * atom[a] + i] - xyz[3 * atom[b] + i];
  cap[c] = nprim[a] * nprim[b];
}

// Primitive-pair records; pairs whose prefactor magnitude is below prim_tau are dropped.
__global__ void k_prim_fill(int n_cand, const int* __restrict__ sa, const int* __restrict__ sb,
                            const int* __restrict__ nprim, const int* __restrict__ prim_off_shell,
                            const int* __restrict__ atom, const double* __restrict__ xyz,
                            const double* __restrict__ alpha, const double* __restrict__ w,
                            const int* __restrict__ pp_off, double prim_tau, PrimPair* __restrict__ pp,
                            int* __restrict__ pp_n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cand) return;
  const int a = sa[c], b = sb[c];
  const double A[3] = {xyz[3 * atom[a]], xyz[3 * atom[a] + 1], xyz[3 * atom[a] + 2]};
  const double B[3] = {xyz[3 * atom[b]], xyz[3 * atom[b] + 1], xyz[3 * atom[b] + 2]};
  const double AB2 = (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]);
  const double c0 = 5.914967172795613;  // sqrt(2 pi^{5/2})
  int n = 0;
  PrimPair* out = pp + pp_off[c];
  for (int ia = 0; ia < nprim[a]; ++ia) {
    const double ea = alpha[prim_off_shell[a] + ia], wa = w[prim_off_shell[a] + ia];
    for (int ib = 0; ib < nprim[b]; ++ib) {
      const double eb = alpha[prim_off_shell[b] + ib], wb = w[prim_off_shell[b] + ib];
      const double p = ea + eb;
      const double C = c0 * wa * wb * exp(-ea * eb / p * AB2) / p;
      if (fabs(C) < prim_tau) continue;
      PrimPair r;
      r.p = p;
      r.inv2p = 0.5 / p;
      for (int i = 0; i < 3; ++i) {
        r.P[i] = (ea * A[i] + eb * B[i]) / p;
        r.PA[i] = r.P[i] - A[i];
      }
      r.C = C;
      r.inv2p3 = 1.5 / p;
      r.pf = (float)p;
      r.inv2pf = (float)r.inv2p;
      for (int i = 0; i < 3; ++i) {
        r.PAf[i] = (float)r.PA[i];
        r.Pf[i] = (float)r.P[i];
      }
      out[n++] = r;
    }
  }
  pp_n[c] = n;
}

// Pair data of the distance-aware test, per candidate pair: the centre of its most diffuse
// primitive pair (a, b the smallest exponents of the two shells: (a A + b B)/(a + b)), the
// largest distance of any primitive-pair centre from it (all lie on AB), a + b.
__global__ void k_pair_dist(int n_cand, const int* __restrict__ sa, const int* __restrict__ sb,
                            const int* __restrict__ nprim, const int* __restrict__ prim_off_shell,
                            const int* __restrict__ atom, const double* __restrict__ xyz,
                            const double* __restrict__ alpha, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cand) return;
  const int I = sa[c], J = sb[c];
  const double* A = xyz + 3 * atom[I];
  const double* B = xyz + 3 * atom[J];
  double a = alpha[prim_off_shell[I]], b = alpha[prim_off_shell[J]];
  for (int k = 1; k < nprim[I]; ++k) a = fmin(a, alpha[prim_off_shell[I] + k]);
  for (int k = 1; k < nprim[J]; ++k) b = fmin(b, alpha[prim_off_shell[J] + k]);
  double ab = 0.0;
  for (int i = 0; i < 3; ++i) {
    out[5 * c + i] = (a * A[i] + b * B[i]) / (a + b);
    ab += (A[i] - B[i]) * (A[i] - B[i]);
  }
  ab = sqrt(ab);
  double sp = 0.0;
  for (int k = 0; k < nprim[I]; ++k)
    for (int kk = 0; kk < nprim[J]; ++kk) {
      const double x = alpha[prim_off_shell[I] + k], y = alpha[prim_off_shell[J] + kk];
      sp = fmax(sp, fabs(x / (x + y) - a / (a + b)) * ab);
    }
  out[5 * c + 3] = sp;
  out[5 * c + 4] = a + b;
}

__global__ void k_gather5(int n, const int* __restrict__ sorted, const double* __restrict__ in, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < 5; ++k) out[5 * i + k] = in[5 * sorted[i] + k];
}

__global__ void k_iota(int n, int* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = i;
}

__global__ void k_hist(int n, const int* __restrict__ key, int* __restrict__ counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(counts + key[i], 1);
}

// bin = pair class if the pair passes Q_IJ Q_max >= tau, else 6 (dropped)
__global__ void k_bin_keys(int n, const double* __restrict__ Q, const double* __restrict__ qmax, double tau,
                           const int* __restrict__ pcls, const int* __restrict__ order, int* __restrict__ binkey) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = order[i];
  binkey[i] = (Q[c] * qmax[0] >= tau) ? pcls[c] : 6;
}

__global__ void k_gather_q(int n, const int* __restrict__ sorted, const double* __restrict__ Q,
                           double* __restrict__ Qs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Qs[i] = Q[sorted[i]];
}

// Quartet count of each row (class pair cp = hi(hi+1)/2 + lo, bra position i in bin hi):
// number of ket positions j in bin lo with Q_i Q_j >= tau (a prefix: bins are sorted by
// Q descending), and j <= i when hi == lo (each unordered pair of pairs once).
__global__ void k_count(int n_rows, RowTable rt, const double* __restrict__ Qs, double tau, int triangle,
                        long long* __restrict__ row_n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  int cp = 0;
  while (cp < 20 && rt.row_base[cp + 1] <= r) ++cp;
  int hi = 0;
  while ((hi + 1) * (hi + 2) / 2 <= cp) ++hi;
  const int lo = cp - hi * (hi + 1) / 2;
  const int i = r - rt.row_base[cp];
  const double qi = Qs[rt.bin_start[hi] + i];
  const double* qk = Qs + rt.bin_start[lo];
  int a = 0, b = rt.bin_size[lo];  // first j with qi*qk[j] < tau lies in [a, b]
  while (a < b) {
    const int m = (a + b) >> 1;
    if (qi * qk[m] >= tau) a = m + 1; else b = m;
  }
  long long n = a;
  if (triangle && hi == lo && n > i + 1) n = i + 1;
  row_n[r] = n;
}

__global__ void k_gather_bounds(RowTable rt, const long long* __restrict__ qoff, long long* __restrict__ out) {
  const int i = threadIdx.x;
  if (i < 22) out[i] = qoff[rt.row_base[i]];
}

// max |P| over each shell-pair block (I, J): one thread per block
// max over a warp, then one atomic per warp into *out (values >= 0, so the order of
// their bit patterns as unsigned integers is their numeric order)
__device__ __forceinline__ void warp_max_into(double m, double* out) {
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(m));
}

__global__ void k_pmax(int ns, const int* __restrict__ bf_off, const int* __restrict__ l,
                       const double* __restrict__ P, int ld, double* __restrict__ pmax, double* pglob) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (t < (long long)ns * ns) {
    const int I = (int)(t / ns), J = (int)(t - (long long)I * ns);
    const int oi = bf_off[I], oj = bf_off[J], ni = 2 * l[I] + 1, nj = 2 * l[J] + 1;
    for (int a = 0; a < ni; ++a)
      for (int b = 0; b < nj; ++b) m = fmax(m, fabs(P[(size_t)(oi + a) * ld + oj + b]));
    pmax[t] = m;
  }
  if (pglob) warp_max_into(m, pglob);  // blockDim is a multiple of 32: whole warps get here
}

// max |P^R| over each (home shell, home shell) block of every density block: one thread per
// (R, I, J)
__global__ void k_pmax_blocks(int n_R, int ns, int nbf, const int* __restrict__ bf_off, const int* __restrict__ l,
                              const double* __restrict__ P, double* __restrict__ pmax) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n_R * ns * ns) return;
  const int r = (int)(t / ((long long)ns * ns));
  const int rem = (int)(t - (long long)r * ns * ns);
  const int I = rem / ns, J = rem - I * ns;
  const double* B = P + (size_t)r * nbf * nbf;
  double m = 0.0;
  for (int a = 0; a < 2 * l[I] + 1; ++a)
    for (int b = 0; b < 2 * l[J] + 1; ++b) m = fmax(m, fabs(B[(size_t)(bf_off[I] + a) * nbf + bf_off[J] + b]));
  pmax[t] = m;
}

// ---------------------------------------------------------------------------
// K = A + A^T in place, 32x32 tiles (tile pairs bi <= bj), then E = sum P K with
// compensated (Neumaier) summation.
// ---------------------------------------------------------------------------
__global__ void k_symmetrize(int n, int ld, double* __restrict__ K) {
  __shared__ double ta[32][33], tb[32][33];
  const int nt = (n + 31) / 32;
  long long t = blockIdx.x;
  int bj = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)bj * (bj + 1) / 2 > t) --bj;
  while ((long long)(bj + 1) * (bj + 2) / 2 <= t) ++bj;
  const int bi = (int)(t - (long long)bj * (bj + 1) / 2);  // bi <= bj
  if (bj >= nt) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += blockDim.y) {
    const int i = bi * 32 + r, j = bj * 32 + tx;
    ta[r][tx] = (i < n && j < n) ? K[(size_t)i * ld + j] : 0.0;
    const int i2 = bj * 32 + r, j2 = bi * 32 + tx;
    tb[r][tx] = (i2 < n && j2 < n) ? K[(size_t)i2 * ld + j2] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += blockDim.y) {
    const int i = bi * 32 + r, j = bj * 32 + tx;
    const double s = ta[r][tx] + tb[tx][r];  // A_ij + A_ji
    if (i < n && j < n) K[(size_t)i * ld + j] = s;
    const int i2 = bj * 32 + r, j2 = bi * 32 + tx;
    const double s2 = tb[r][tx] + ta[tx][r];
    if (bi != bj && i2 < n && j2 < n) K[(size_t)i2 * ld + j2] = s2;
  }
}

// B = A^T for n x n row-major blocks (32 x 32 tiles through shared memory)
__global__ void k_transpose(int n, const double* __restrict__ A, double* __restrict__ B) {
  __shared__ double t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = by + r, j = bx + threadIdx.x;
    if (i < n && j < n) t[r][threadIdx.x] = A[(size_t)i * n + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = bx + r, j = by + threadIdx.x;
    if (i < n && j < n) B[(size_t)i * n + j] = t[threadIdx.x][r];
  }
}

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__global__ void k_trace_partial(int n, int ld, const double* __restrict__ P, const double* __restrict__ K,
                                double* __restrict__ part) {
  double s = 0.0, c = 0.0;
  const long long nn = (long long)n * n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t - (long long)i * n);
    double e;
    two_sum(s, P[(size_t)i * ld + j] * K[(size_t)i * ld + j], s, e);
    c += e;
  }
  __shared__ double ss[256], cc[256];
  ss[threadIdx.x] = s;
  cc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double e;
      two_sum(ss[threadIdx.x], ss[threadIdx.x + w], ss[threadIdx.x], e);
      cc[threadIdx.x] += cc[threadIdx.x + w] + e;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ss[0];
    part[2 * blockIdx.x + 1] = cc[0];
  }
}

__global__ void k_trace_final(int nb, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double ss[256], cc[256];
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    double e;
    two_sum(s, part[2 * i], s, e);
    c += e + part[2 * i + 1];
  }
  ss[threadIdx.x] = s;
  cc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double e;
      two_sum(ss[threadIdx.x], ss[threadIdx.x + w], ss[threadIdx.x], e);
      cc[threadIdx.x] += cc[threadIdx.x + w] + e;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = ss[0] + cc[0];
}

// ---------------------------------------------------------------------------
// FMA-chain throughput probe (register-resident independent chains).
// ---------------------------------------------------------------------------
// `active` lanes of every warp run the chains (32: all); the others skip them.
template <typename T>
__global__ void k_fma_chain(T* out, int iters, T a, T b, int active) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  if ((int)(threadIdx.x & 31) < active) {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s == (T)12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ---------------------------------------------------------------------------
// Batched forms: one launch for all systems of a batch (grid.y = system); every pointer
// and size is read from the device table, so a captured graph is independent of them.
// ---------------------------------------------------------------------------
__global__ void k_batch_zero(const BatchSys* __restrict__ sys) {
  const BatchSys b = sys[blockIdx.y];
  if (b.pglob && blockIdx.x == 0 && threadIdx.x == 0) *b.pglob = 0.0;
  const long long nn = (long long)b.n * b.n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / b.n), j = (int)(t - (long long)i * b.n);
    b.K[(size_t)i * b.ld + j] = 0.0;
  }
}

__global__ void k_batch_pmax(const BatchSys* __restrict__ sys) {
  const BatchSys b = sys[blockIdx.y];
  const long long nn = (long long)b.ns * b.ns;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // every thread runs the same number of rounds, so whole warps reach the reduction
  const long long rounds = (nn + stride - 1) / stride;
  double mg = 0.0;
  for (long long k = 0; k < rounds; ++k) {
    const long long t = k * stride + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nn) continue;
    const int I = (int)(t / b.ns), J = (int)(t - (long long)I * b.ns);
    const int oi = b.bf_off[I], oj = b.bf_off[J], ni = 2 * b.l[I] + 1, nj = 2 * b.l[J] + 1;
    double m = 0.0;
    for (int a = 0; a < ni; ++a)
      for (int c = 0; c < nj; ++c) m = fmax(m, fabs(b.P[(size_t)(oi + a) * b.ld + oj + c]));
    b.pmax[t] = m;
    mg = fmax(mg, m);
  }
  if (b.pglob) warp_max_into(mg, b.pglob);
}

__global__ void k_batch_symmetrize(const BatchSys* __restrict__ sys) {
  __shared__ double ta[32][33], tb[32][33];
  const BatchSys b = sys[blockIdx.y];
  const int nt = (b.n + 31) / 32;
  const long long ntp = (long long)nt * (nt + 1) / 2;
  for (long long t = blockIdx.x; t < ntp; t += gridDim.x) {
    int bj = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)bj * (bj + 1) / 2 > t) --bj;
    while ((long long)(bj + 1) * (bj + 2) / 2 <= t) ++bj;
    const int bi = (int)(t - (long long)bj * (bj + 1) / 2);
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += blockDim.y) {
      const int i = bi * 32 + r, j = bj * 32 + tx;
      ta[r][tx] = (i < b.n && j < b.n) ? b.K[(size_t)i * b.ld + j] : 0.0;
      const int i2 = bj * 32 + r, j2 = bi * 32 + tx;
      tb[r][tx] = (i2 < b.n && j2 < b.n) ? b.K[(size_t)i2 * b.ld + j2] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += blockDim.y) {
      const int i = bi * 32 + r, j = bj * 32 + tx;
      if (i < b.n && j < b.n) b.K[(size_t)i * b.ld + j] = ta[r][tx] + tb[tx][r];
      const int i2 = bj * 32 + r, j2 = bi * 32 + tx;
      if (bi != bj && i2 < b.n && j2 < b.n) b.K[(size_t)i2 * b.ld + j2] = tb[r][tx] + ta[tx][r];
    }
    __syncthreads();
  }
}

// compensated partial sums of P K: blockIdx.y = system, kBatchPart blocks per system
__global__ void k_batch_trace_partial(const BatchSys* __restrict__ sys) {
  const BatchSys b = sys[blockIdx.y];
  __shared__ double ss[256], cc[256];
  double s = 0.0, c = 0.0;
  const long long nn = (long long)b.n * b.n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / b.n), j = (int)(t - (long long)i * b.n);
    double e;
    two_sum(s, b.P[(size_t)i * b.ld + j] * b.K[(size_t)i * b.ld + j], s, e);
    c += e;
  }
  ss[threadIdx.x] = s;
  cc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double e;
      two_sum(ss[threadIdx.x], ss[threadIdx.x + w], ss[threadIdx.x], e);
      cc[threadIdx.x] += cc[threadIdx.x + w] + e;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    b.part[2 * blockIdx.x] = ss[0];
    b.part[2 * blockIdx.x + 1] = cc[0];
  }
}

// one block of kBatchPart threads per system: E_K from the partial sums
__global__ void k_batch_trace_final(const BatchSys* __restrict__ sys) {
  const BatchSys b = sys[blockIdx.x];
  __shared__ double ss[kBatchPart], cc[kBatchPart];
  ss[threadIdx.x] = b.part[2 * threadIdx.x];
  cc[threadIdx.x] = b.part[2 * threadIdx.x + 1];
  __syncthreads();
  for (int w = kBatchPart / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double e;
      two_sum(ss[threadIdx.x], ss[threadIdx.x + w], ss[threadIdx.x], e);
      cc[threadIdx.x] += cc[threadIdx.x + w] + e;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) b.energy[0] = ss[0] + cc[0];
}

// ===========================================================================
// Host wrappers
// ===========================================================================
static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

cudaError_t launch_normalize(int n_shells, const int* l, const int* nprim, const int* prim_off,
                             const double* alpha, const double* coef, double* w, cudaStream_t s) {
  if (n_shells <= 0) return cudaSuccess;
  k_normalize<<<nblk(n_shells, 128), 128, 0, s>>>(n_shells, l, nprim, prim_off, alpha, coef, w);
  return cudaGetLastError();
}

cudaError_t launch_transpose(int n, const double* A, double* B, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_transpose<<<dim3(nblk(n, 32), nblk(n, 32)), dim3(32, 8), 0, s>>>(n, A, B);
  return cudaGetLastError();
}

cudaError_t launch_pmax_blocks(int n_R, int ns, int nbf, const int* bf_off, const int* l, const double* P,
                               double* pmax, cudaStream_t s) {
  const long long n = (long long)n_R * ns * ns;
  if (n <= 0) return cudaSuccess;
  k_pmax_blocks<<<nblk(n, 128), 128, 0, s>>>(n_R, ns, nbf, bf_off, l, P, pmax);
  return cudaGetLastError();
}

cudaError_t launch_boys_table(double* tab, cudaStream_t s) {
  k_boys_table<<<nblk(kBoysRows, 128), 128, 0, s>>>(tab);
  return cudaGetLastError();
}

cudaError_t launch_pair_flags(long long n_tri, const int* atom, const double* xyz, double rcut, int* flag,
                              cudaStream_t s) {
  if (n_tri <= 0) return cudaSuccess;
  k_pair_flags<<<nblk(n_tri, 256), 256, 0, s>>>(n_tri, atom, xyz, rcut, flag);
  return cudaGetLastError();
}

cudaError_t select_flagged(void* tmp, size_t& tmp_bytes, long long n_tri, const int* flag, long long* out,
                           int* d_num, cudaStream_t s) {
  thrust::counting_iterator<long long> it(0);
  return cub::DeviceSelect::Flagged(tmp, tmp_bytes, it, flag, out, d_num, n_tri, s);
}

cudaError_t launch_pair_flags_rect(long long n, int n_img, const int* atom, const double* xyz, double rcut, int* flag,
                                   cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_pair_flags_rect<<<nblk(n, 256), 256, 0, s>>>(n, n_img, atom, xyz, rcut, flag);
  return cudaGetLastError();
}

cudaError_t launch_pair_setup_rect(int n_cand, const long long* cand_t, int n_img, const int* l, const int* nprim,
                                   const int* atom, const double* xyz, int* sa, int* sb, int* pcls, double* AB,
                                   int* cap, unsigned char* home_first, cudaStream_t s) {
  if (n_cand <= 0) return cudaSuccess;
  k_pair_setup_rect<<<nblk(n_cand, 256), 256, 0, s>>>(n_cand, cand_t, n_img, l, nprim, atom, xyz, sa, sb, pcls, AB,
                                                      cap, home_first);
  return cudaGetLastError();
}

cudaError_t launch_pair_setup(int n_cand, const long long* cand_t, const int* l, const int* nprim,
                              const int* atom, const double* xyz, int* sa, int* sb, int* pcls, double* AB,
                              int* cap, cudaStream_t s) {
  if (n_cand <= 0) return cudaSuccess;
  k_pair_setup<<<nblk(n_cand, 256), 256, 0, s>>>(n_cand, cand_t, l, nprim, atom, xyz, sa, sb, pcls, AB, cap);
  return cudaGetLastError();
}

cudaError_t scan_int(void* tmp, size_t& tmp_bytes, const int* in, int* out, int n, cudaStream_t s) {
  return cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, in, out, n, s);
}

cudaError_t scan_ll_inclusive(void* tmp, size_t& tmp_bytes, const long long* in, long long* out, int n,
                              cudaStream_t s) {
  return cub::DeviceScan::InclusiveSum(tmp, tmp_bytes, in, out, n, s);
}

cudaError_t launch_prim_fill(int n_cand, const int* sa, const int* sb, const int* nprim, const int* prim_off_shell,
                             const int* atom, const double* xyz, const double* alpha, const double* w,
                             const int* pp_off, double prim_tau, PrimPair* pp, int* pp_n, cudaStream_t s) {
  if (n_cand <= 0) return cudaSuccess;
  k_prim_fill<<<nblk(n_cand, 128), 128, 0, s>>>(n_cand, sa, sb, nprim, prim_off_shell, atom, xyz, alpha, w,
                                                 pp_off, prim_tau, pp, pp_n);
  return cudaGetLastError();
}

cudaError_t launch_pair_dist(int n_cand, const int* sa, const int* sb, const int* nprim, const int* prim_off_shell,
                             const int* atom, const double* xyz, const double* alpha, double* out, cudaStream_t s) {
  if (n_cand <= 0) return cudaSuccess;
  k_pair_dist<<<nblk(n_cand, 128), 128, 0, s>>>(n_cand, sa, sb, nprim, prim_off_shell, atom, xyz, alpha, out);
  return cudaGetLastError();
}

cudaError_t launch_gather5(int n, const int* sorted, const double* in, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather5<<<nblk(n, 128), 128, 0, s>>>(n, sorted, in, out);
  return cudaGetLastError();
}

cudaError_t launch_iota(int n, int* v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_iota<<<nblk(n, 256), 256, 0, s>>>(n, v);
  return cudaGetLastError();
}

cudaError_t launch_hist(int n, const int* key, int* counts, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_hist<<<nblk(n, 256), 256, 0, s>>>(n, key, counts);
  return cudaGetLastError();
}

cudaError_t sort_int_keys(void* tmp, size_t& tmp_bytes, const int* kin, int* kout, const int* vin, int* vout,
                          int n, int end_bit, cudaStream_t s) {
  return cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, kin, kout, vin, vout, n, 0, end_bit, s);
}

cudaError_t sort_double_desc(void* tmp, size_t& tmp_bytes, const double* kin, double* kout, const int* vin,
                             int* vout, int n, cudaStream_t s) {
  return cub::DeviceRadixSort::SortPairsDescending(tmp, tmp_bytes, kin, kout, vin, vout, n, 0, 64, s);
}

cudaError_t reduce_max(void* tmp, size_t& tmp_bytes, const double* in, double* out, int n, cudaStream_t s) {
  return cub::DeviceReduce::Max(tmp, tmp_bytes, in, out, n, s);
}

cudaError_t launch_bin_keys(int n, const double* Q, const double* qmax, double tau, const int* pcls,
                            const int* order, int* binkey, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_bin_keys<<<nblk(n, 256), 256, 0, s>>>(n, Q, qmax, tau, pcls, order, binkey);
  return cudaGetLastError();
}

cudaError_t launch_gather_q(int n, const int* sorted, const double* Q, double* Qs, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather_q<<<nblk(n, 256), 256, 0, s>>>(n, sorted, Q, Qs);
  return cudaGetLastError();
}

cudaError_t launch_count(int n_rows, const RowTable& rt, const double* Qs, double tau, long long* row_n,
                         cudaStream_t s, bool triangle) {
  if (n_rows <= 0) return cudaSuccess;
  k_count<<<nblk(n_rows, 128), 128, 0, s>>>(n_rows, rt, Qs, tau, triangle ? 1 : 0, row_n);
  return cudaGetLastError();
}

cudaError_t launch_gather_bounds(const RowTable& rt, const long long* qoff, long long* out, cudaStream_t s) {
  k_gather_bounds<<<1, 32, 0, s>>>(rt, qoff, out);
  return cudaGetLastError();
}

cudaError_t launch_finalize(int n, int ld, const double* P, double* K, double* part, int n_part, double* energy,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long nt = (n + 31) / 32;
  k_symmetrize<<<(unsigned)(nt * (nt + 1) / 2), dim3(32, 8), 0, s>>>(n, ld, K);
  k_trace_partial<<<n_part, 256, 0, s>>>(n, ld, P, K, part);
  k_trace_final<<<1, 256, 0, s>>>(n_part, part, energy);
  return cudaGetLastError();
}

cudaError_t launch_pmax(int ns, const int* bf_off, const int* l, const double* P, int ld, double* pmax,
                        double* pglob, cudaStream_t s) {
  const long long n = (long long)ns * ns;
  if (n <= 0) return cudaSuccess;
  if (pglob) {
    cudaError_t e = cudaMemsetAsync(pglob, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
  }
  k_pmax<<<nblk(n, 256), 256, 0, s>>>(ns, bf_off, l, P, ld, pmax, pglob);
  return cudaGetLastError();
}

cudaError_t launch_batch_prologue(const BatchSys* sys, int n, int n_sm, bool pmax, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_batch_zero<<<dim3(2 * n_sm, n), 256, 0, s>>>(sys);
  if (pmax) k_batch_pmax<<<dim3(n_sm, n), 256, 0, s>>>(sys);
  return cudaGetLastError();
}

cudaError_t launch_batch_epilogue(const BatchSys* sys, int n, int n_sm, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_batch_symmetrize<<<dim3(n_sm, n), dim3(32, 8), 0, s>>>(sys);
  k_batch_trace_partial<<<dim3(kBatchPart, n), 256, 0, s>>>(sys);
  k_batch_trace_final<<<n, kBatchPart, 0, s>>>(sys);
  return cudaGetLastError();
}

cudaError_t fma_peak(double* fp64_tflops, double* fp32_tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  double* d = nullptr;
  const int blocks = sms * 4, threads = 256;
  e = cudaMalloc(&d, sizeof(double) * blocks * threads);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  const int it64 = 4096, it32 = 65536;
  for (int w = 0; w < 2; ++w) k_fma_chain<double><<<blocks, threads>>>(d, it64, 0.999, 1e-4, 32);
  cudaEventRecord(e0);
  k_fma_chain<double><<<blocks, threads>>>(d, it64, 0.999, 1e-4, 32);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *fp64_tflops = 2.0 * 8 * (double)it64 * blocks * threads / (ms * 1e-3) / 1e12;
  for (int w = 0; w < 2; ++w) k_fma_chain<float><<<blocks, threads>>>((float*)d, it32, 0.999f, 1e-4f, 32);
  cudaEventRecord(e0);
  k_fma_chain<float><<<blocks, threads>>>((float*)d, it32, 0.999f, 1e-4f, 32);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *fp32_tflops = 2.0 * 8 * (double)it32 * blocks * threads / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  e = cudaGetLastError();
  cudaFree(d);
  return e;
}

}  // namespace hfx

namespace hfx {
// Time of the FP64 FMA chains with 1 and with 32 active lanes per warp (the same warp
// instructions; the 1-lane run does 1/32 of the flops): equal times mean the FP64 pipe is
// charged per warp instruction, not per active lane.
cudaError_t fp64_lane_cost(double* ms_32, double* ms_1) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  double* d = nullptr;
  const int blocks = sms * 4, threads = 256, it64 = 4096;
  e = cudaMalloc(&d, sizeof(double) * blocks * threads);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double* outs[2] = {ms_32, ms_1};
  const int act[2] = {32, 1};
  k_fma_chain<double><<<blocks, threads>>>(d, it64, 0.999, 1e-4, 32);
  for (int r = 0; r < 2; ++r) {
    float ms = 0.f;
    cudaEventRecord(e0);
    k_fma_chain<double><<<blocks, threads>>>(d, it64, 0.999, 1e-4, act[r]);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *outs[r] = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  e = cudaGetLastError();
  cudaFree(d);
  return e;
}
}  // namespace hfx
