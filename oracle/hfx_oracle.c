/*
 * hfx_oracle.c -- plain, slow, FP64 CPU reference ("oracle") for the screened,
 * erfc-attenuated exact-exchange build
 *
 *     K_{mu nu} = sum_{lambda sigma} keep * (mu lambda | nu sigma)_omega * P_{lambda sigma}
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it; the CUDA library never does.  It shares no source,
 * table or helper with the CUDA path.
 *
 * What it follows (citations are to the paper's sections / equations):
 *  - exchange matrix, Sec. 2 Eq. (vx): one cell, no lattice images, no -1/2 prefactor;
 *  - the two-electron integral definition, Sec. 2 (ERI equation), with the Coulomb
 *    kernel replaced by the HSE06 short-range kernel erfc(omega r)/r (Sec. 4, HSE06);
 *  - contracted Gaussian shells of (2l+1) spherical functions, Sec. 3.1 (shell quartets)
 *    and the Cartesian -> spherical transformation, Sec. 3.1 (last paragraph);
 *  - Schwarz screening, Sec. 3.1 Eq. (schwarz), and the orbital-cutoff (NAO) screening,
 *    Sec. 3.1;
 *  - eight-fold permutational symmetry, Sec. 3.1 (symmetry equation).
 *
 * Integrals: Obara-Saika vertical recurrence (Obara & Saika, J. Chem. Phys. 84, 3963
 * (1986)) and Head-Gordon-Pople horizontal recurrence (J. Chem. Phys. 89, 5777 (1988)),
 * with the Boys function F_m replaced by the attenuated form
 *     G_m(T) = F_m(T) - kappa^{m+1/2} F_m(kappa T),  kappa = omega^2 / (omega^2 + rho),
 * which is the Coulomb value minus the erf(omega r)/r value.  F_m is evaluated from its
 * convergent series below T = 30 and from erf plus upward recursion above.
 *
 * Basis function definition used here (and stated in the design notes):
 *     chi_{I,m}(r) = N_{I,m} S_m(r - A) sum_k c_k n_l(alpha_k) exp(-alpha_k |r - A|^2)
 * with n_l(alpha) = (2 alpha/pi)^{3/4} (4 alpha)^{l/2} / sqrt((2l-1)!!), the raw weights c_k,
 * S_m the real solid-harmonic polynomial (1; x, y, z; xy, yz, 3z^2-r^2, xz, x^2-y^2) and
 * N_{I,m} chosen so that each function has unit self-overlap.  The self-overlap is
 * computed here from Gaussian moment integrals, one spherical component at a time.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_MAXL 2          /* highest shell angular momentum */
#define ORA_MAXDEG 8        /* highest total degree in a quartet */
#define ORA_NMONO4 35       /* monomials of degree <= 4 */
#define ORA_MAXCART 6
#define ORA_MAXSPH 5

/* ------------------------------------------------------------------------- */
/* Boys function F_m(T) = int_0^1 u^{2m} exp(-T u^2) du                       */
/* ------------------------------------------------------------------------- */

/* Series F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)), then downward
 * recursion F_{m-1} = (2T F_m + exp(-T)) / (2m-1). */
static void boys_series(int mmax, double T, double *F) {
  double term = 1.0 / (2 * mmax + 1), sum = term;
  for (int k = 1; k < 10000; ++k) {
    term *= 2.0 * T / (2 * mmax + 2 * k + 1);
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  double e = exp(-T);
  F[mmax] = e * sum;
  for (int m = mmax - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + e) / (2 * m + 1);
}

/* F_0(T) = (1/2) sqrt(pi/T) erf(sqrt(T)), upward F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T),
 * stable for T > m + 1/2. */
static void boys_erf_up(int mmax, double T, double *F) {
  double e = exp(-T);
  F[0] = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
  for (int m = 0; m < mmax; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);
}

void ora_boys(int mmax, double T, double *F) {
  if (T < 30.0)
    boys_series(mmax, T, F);
  else
    boys_erf_up(mmax, T, F);
}

/* G_m(T) = F_m(T) - kappa^{m+1/2} F_m(kappa T); kappa = 0 gives the Coulomb F_m. */
void ora_gboys(int mmax, double T, double kappa, double *G) {
  double F1[ORA_MAXDEG + 16], F2[ORA_MAXDEG + 16];
  ora_boys(mmax, T, F1);
  if (kappa <= 0.0) {
    for (int m = 0; m <= mmax; ++m) G[m] = F1[m];
    return;
  }
  ora_boys(mmax, kappa * T, F2);
  double km = sqrt(kappa);
  for (int m = 0; m <= mmax; ++m) {
    G[m] = F1[m] - km * F2[m];
    km *= kappa;
  }
}

/* ------------------------------------------------------------------------- */
/* Cartesian monomials                                                        */
/* ------------------------------------------------------------------------- */

/* Monomials of degree l, ordered i = l..0, j = l-i..0, k = l-i-j (xx, xy, xz, yy, yz, zz). */
static int g_mono[165][3];
static int g_deg_off[ORA_MAXDEG + 2];
static int g_mono_idx[ORA_MAXDEG + 1][ORA_MAXDEG + 1][ORA_MAXDEG + 1];
static int g_init = 0;

static void mono_init(void) {
  if (g_init) return;
  int n = 0;
  for (int l = 0; l <= ORA_MAXDEG; ++l) {
    g_deg_off[l] = n;
    for (int i = l; i >= 0; --i)
      for (int j = l - i; j >= 0; --j) {
        int k = l - i - j;
        g_mono[n][0] = i;
        g_mono[n][1] = j;
        g_mono[n][2] = k;
        g_mono_idx[i][j][k] = n;
        ++n;
      }
  }
  g_deg_off[ORA_MAXDEG + 1] = n;
  g_init = 1;
}

static inline int ncart(int l) { return (l + 1) * (l + 2) / 2; }
static inline int nsph(int l) { return 2 * l + 1; }
static inline int midx(int i, int j, int k) { return g_mono_idx[i][j][k]; }

/* Real solid-harmonic polynomials as Cartesian monomial expansions (unnormalised):
 * l=0: 1; l=1: x, y, z; l=2: xy, yz, 3z^2-r^2 = 2zz-xx-yy, xz, x^2-y^2. Coefficient
 * sph_poly[l][m][c] multiplies the c-th monomial of degree l (ordering above). */
static const double sph_poly[3][5][6] = {
    {{1, 0, 0, 0, 0, 0}},
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    /* xx  xy  xz  yy  yz  zz */
    {{0, 1, 0, 0, 0, 0},    /* xy        */
     {0, 0, 0, 0, 1, 0},    /* yz        */
     {-1, 0, 0, -1, 0, 2},  /* 3z^2-r^2  */
     {0, 0, 1, 0, 0, 0},    /* xz        */
     {1, 0, 0, -1, 0, 0}},  /* x^2-y^2   */
};

/* ------------------------------------------------------------------------- */
/* Basis                                                                      */
/* ------------------------------------------------------------------------- */

typedef struct {
  int n_atoms, n_shells, n_bf;
  double *xyz;      /* 3 per atom */
  int *atom, *l, *nprim, *prim_off, *bf_off;
  double *alpha;    /* per primitive */
  double *w;        /* per primitive: c_k * n_l(alpha_k) */
  double *nrm;      /* per shell: ORA_MAXSPH spherical-component normalisers N_{I,m} */
} ora_basis;

static double dfact(int n) { /* n!! with (-1)!! = 1 */
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

/* int x^n exp(-g x^2) dx over the real line */
static double gmoment(int n, double g) {
  if (n & 1) return 0.0;
  return dfact(n - 1) / pow(2.0 * g, n / 2) * sqrt(M_PI / g);
}

void ora_basis_free(void *vb) {
  ora_basis *b = (ora_basis *)vb;
  if (!b) return;
  free(b->xyz); free(b->atom); free(b->l); free(b->nprim); free(b->prim_off);
  free(b->bf_off); free(b->alpha); free(b->w); free(b->nrm);
  free(b);
}

void *ora_basis_new(int n_atoms, const double *xyz, int n_shells, const int *shell_atom,
                    const int *shell_l, const int *shell_nprim, const double *alpha,
                    const double *coef) {
  mono_init();
  ora_basis *b = (ora_basis *)calloc(1, sizeof(ora_basis));
  b->n_atoms = n_atoms;
  b->n_shells = n_shells;
  b->xyz = (double *)malloc(sizeof(double) * 3 * (n_atoms > 0 ? n_atoms : 1));
  memcpy(b->xyz, xyz, sizeof(double) * 3 * n_atoms);
  b->atom = (int *)malloc(sizeof(int) * n_shells);
  b->l = (int *)malloc(sizeof(int) * n_shells);
  b->nprim = (int *)malloc(sizeof(int) * n_shells);
  b->prim_off = (int *)malloc(sizeof(int) * (n_shells + 1));
  b->bf_off = (int *)malloc(sizeof(int) * (n_shells + 1));
  int np = 0, nb = 0;
  for (int s = 0; s < n_shells; ++s) {
    if (shell_l[s] < 0 || shell_l[s] > ORA_MAXL || shell_nprim[s] < 1 || shell_atom[s] < 0 ||
        shell_atom[s] >= n_atoms) {
      ora_basis_free(b);
      return NULL;
    }
    b->atom[s] = shell_atom[s];
    b->l[s] = shell_l[s];
    b->nprim[s] = shell_nprim[s];
    b->prim_off[s] = np;
    b->bf_off[s] = nb;
    np += shell_nprim[s];
    nb += nsph(shell_l[s]);
  }
  b->prim_off[n_shells] = np;
  b->bf_off[n_shells] = nb;
  b->n_bf = nb;
  b->alpha = (double *)malloc(sizeof(double) * (np > 0 ? np : 1));
  b->w = (double *)malloc(sizeof(double) * (np > 0 ? np : 1));
  b->nrm = (double *)malloc(sizeof(double) * ORA_MAXSPH * (n_shells > 0 ? n_shells : 1));
  for (int s = 0; s < n_shells; ++s) {
    int l = b->l[s];
    for (int k = 0; k < b->nprim[s]; ++k) {
      int p = b->prim_off[s] + k;
      double a = alpha[p];
      b->alpha[p] = a;
      b->w[p] = coef[p] * pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * l) / sqrt(dfact(2 * l - 1));
    }
    /* self-overlap of S_m(r) R(r): sum_{k,k'} w_k w_k' sum_{c,c'} t_c t_c' <mono_c mono_c'> */
    int nc = ncart(l);
    for (int m = 0; m < nsph(l); ++m) {
      double ov = 0.0;
      for (int k = 0; k < b->nprim[s]; ++k)
        for (int kk = 0; kk < b->nprim[s]; ++kk) {
          int p1 = b->prim_off[s] + k, p2 = b->prim_off[s] + kk;
          double g = b->alpha[p1] + b->alpha[p2];
          double acc = 0.0;
          for (int c = 0; c < nc; ++c)
            for (int cc = 0; cc < nc; ++cc) {
              double t = sph_poly[l][m][c] * sph_poly[l][m][cc];
              if (t == 0.0) continue;
              const int *u = g_mono[g_deg_off[l] + c], *v = g_mono[g_deg_off[l] + cc];
              acc += t * gmoment(u[0] + v[0], g) * gmoment(u[1] + v[1], g) * gmoment(u[2] + v[2], g);
            }
          ov += b->w[p1] * b->w[p2] * acc;
        }
      b->nrm[ORA_MAXSPH * s + m] = 1.0 / sqrt(ov);
    }
  }
  return b;
}

int ora_n_bf(const void *vb) { return ((const ora_basis *)vb)->n_bf; }

/* N_{I,m} for every shell (ORA_MAXSPH per shell) and radial weights c_k n_l(alpha_k). */
void ora_basis_export(const void *vb, double *nrm_out, double *w_out) {
  const ora_basis *b = (const ora_basis *)vb;
  if (nrm_out) memcpy(nrm_out, b->nrm, sizeof(double) * ORA_MAXSPH * b->n_shells);
  if (w_out) memcpy(w_out, b->w, sizeof(double) * b->prim_off[b->n_shells]);
}

/* ------------------------------------------------------------------------- */
/* Contracted Cartesian shell quartet by OS VRR + HGP HRR                     */
/* ------------------------------------------------------------------------- */

typedef struct {
  int l, n;            /* angular momentum, number of primitives */
  const double *alpha; /* exponents */
  const double *w;     /* contraction weights (include primitive normalisation) */
  double A[3];         /* centre */
} ora_shell;

/* Work space of one thread. */
typedef struct {
  double vrr[ORA_NMONO4][ORA_NMONO4][ORA_MAXDEG + 1];
  double cont[ORA_NMONO4][ORA_NMONO4];
  double lvl[ORA_MAXL + 1][ORA_NMONO4][ORA_MAXCART][ORA_NMONO4]; /* (a b | f) by b degree */
  double kl[ORA_MAXL + 1][ORA_NMONO4][ORA_MAXCART];              /* (a b | c d) by d degree */
  double cart[ORA_MAXCART][ORA_MAXCART][ORA_MAXCART][ORA_MAXCART];
} ora_ws;

/* first axis along which the monomial has a positive power */
static inline int first_axis(const int *e) { return e[0] > 0 ? 0 : (e[1] > 0 ? 1 : 2); }

/* Cartesian contracted (ab|cd) for shells sa..sd; out[a][b][c][d] over Cartesian
 * components (orders per degree as above).  omega = 0 gives the Coulomb integral. */
static void quartet_cart(const ora_shell *sa, const ora_shell *sb, const ora_shell *sc,
                         const ora_shell *sd, double omega, ora_ws *ws) {
  const int la = sa->l, lb = sb->l, lc = sc->l, ld = sd->l;
  const int E = la + lb, F = lc + ld, Lt = E + F;
  const int ne = g_deg_off[E + 1], nf = g_deg_off[F + 1];
  double AB[3], CD[3];
  for (int i = 0; i < 3; ++i) {
    AB[i] = sa->A[i] - sb->A[i];
    CD[i] = sc->A[i] - sd->A[i];
  }
  double AB2 = AB[0] * AB[0] + AB[1] * AB[1] + AB[2] * AB[2];
  double CD2 = CD[0] * CD[0] + CD[1] * CD[1] + CD[2] * CD[2];
  memset(ws->cont, 0, sizeof(ws->cont));
  const double w2 = omega * omega;

  for (int ia = 0; ia < sa->n; ++ia)
    for (int ib = 0; ib < sb->n; ++ib) {
      double a = sa->alpha[ia], b = sb->alpha[ib];
      double p = a + b;
      double P[3], PA[3];
      for (int i = 0; i < 3; ++i) {
        P[i] = (a * sa->A[i] + b * sb->A[i]) / p;
        PA[i] = P[i] - sa->A[i];
      }
      double Kab = exp(-a * b / p * AB2) * sa->w[ia] * sb->w[ib];
      for (int ic = 0; ic < sc->n; ++ic)
        for (int id = 0; id < sd->n; ++id) {
          double c = sc->alpha[ic], d = sd->alpha[id];
          double q = c + d;
          double Q[3], QC[3];
          for (int i = 0; i < 3; ++i) {
            Q[i] = (c * sc->A[i] + d * sd->A[i]) / q;
            QC[i] = Q[i] - sc->A[i];
          }
          double Kcd = exp(-c * d / q * CD2) * sc->w[ic] * sd->w[id];
          double rho = p * q / (p + q);
          double W[3], WP[3], WQ[3], PQ2 = 0.0;
          for (int i = 0; i < 3; ++i) {
            W[i] = (p * P[i] + q * Q[i]) / (p + q);
            WP[i] = W[i] - P[i];
            WQ[i] = W[i] - Q[i];
            PQ2 += (P[i] - Q[i]) * (P[i] - Q[i]);
          }
          double T = rho * PQ2;
          double kappa = (omega > 0.0) ? w2 / (w2 + rho) : 0.0;
          double G[ORA_MAXDEG + 1];
          ora_gboys(Lt, T, kappa, G);
          double pref = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q)) * Kab * Kcd;
          /* [00|00]^(m) */
          for (int m = 0; m <= Lt; ++m) ws->vrr[0][0][m] = pref * G[m];
          /* bra VRR: [e0|00]^(m) */
          for (int e = 1; e < ne; ++e) {
            const int *ev = g_mono[e];
            int de = ev[0] + ev[1] + ev[2];
            int i = first_axis(ev);
            int e1v[3] = {ev[0], ev[1], ev[2]};
            e1v[i] -= 1;
            int e1 = midx(e1v[0], e1v[1], e1v[2]);
            int ni = e1v[i];
            int e2 = -1;
            if (ni > 0) {
              int e2v[3] = {e1v[0], e1v[1], e1v[2]};
              e2v[i] -= 1;
              e2 = midx(e2v[0], e2v[1], e2v[2]);
            }
            for (int m = 0; m <= Lt - de; ++m) {
              double v = PA[i] * ws->vrr[e1][0][m] + WP[i] * ws->vrr[e1][0][m + 1];
              if (e2 >= 0) v += ni / (2.0 * p) * (ws->vrr[e2][0][m] - rho / p * ws->vrr[e2][0][m + 1]);
              ws->vrr[e][0][m] = v;
            }
          }
          /* ket VRR: [e0|f0]^(m) */
          for (int f = 1; f < nf; ++f) {
            const int *fv = g_mono[f];
            int df = fv[0] + fv[1] + fv[2];
            int i = first_axis(fv);
            int f1v[3] = {fv[0], fv[1], fv[2]};
            f1v[i] -= 1;
            int f1 = midx(f1v[0], f1v[1], f1v[2]);
            int ni = f1v[i];
            int f2 = -1;
            if (ni > 0) {
              int f2v[3] = {f1v[0], f1v[1], f1v[2]};
              f2v[i] -= 1;
              f2 = midx(f2v[0], f2v[1], f2v[2]);
            }
            for (int e = 0; e < ne; ++e) {
              const int *ev = g_mono[e];
              int de = ev[0] + ev[1] + ev[2];
              int ei = ev[i];
              int em = -1;
              if (ei > 0) {
                int emv[3] = {ev[0], ev[1], ev[2]};
                emv[i] -= 1;
                em = midx(emv[0], emv[1], emv[2]);
              }
              for (int m = 0; m <= Lt - de - df; ++m) {
                double v = QC[i] * ws->vrr[e][f1][m] + WQ[i] * ws->vrr[e][f1][m + 1];
                if (f2 >= 0) v += ni / (2.0 * q) * (ws->vrr[e][f2][m] - rho / q * ws->vrr[e][f2][m + 1]);
                if (em >= 0) v += ei / (2.0 * (p + q)) * ws->vrr[em][f1][m + 1];
                ws->vrr[e][f][m] = v;
              }
            }
          }
          /* contraction */
          for (int e = g_deg_off[la]; e < ne; ++e)
            for (int f = g_deg_off[lc]; f < nf; ++f) ws->cont[e][f] += ws->vrr[e][f][0];
        }
    }

  /* HRR on the bra: (a, b+1_i | f) = (a+1_i, b | f) + AB_i (a, b | f), built one
   * b degree at a time in lvl[b degree][a][b component][f]. */
  double (*lvl)[ORA_NMONO4][ORA_MAXCART][ORA_NMONO4] = ws->lvl;
  for (int a = 0; a < ne; ++a)
    for (int f = 0; f < nf; ++f) lvl[0][a][0][f] = ws->cont[a][f];
  for (int db = 1; db <= lb; ++db) {
    for (int bc = 0; bc < ncart(db); ++bc) {
      const int *bv = g_mono[g_deg_off[db] + bc];
      int i = first_axis(bv);
      int b1v[3] = {bv[0], bv[1], bv[2]};
      b1v[i] -= 1;
      int b1 = midx(b1v[0], b1v[1], b1v[2]) - g_deg_off[db - 1];
      for (int a = g_deg_off[la]; a < g_deg_off[E - db + 1]; ++a) {
        const int *av = g_mono[a];
        int a1 = midx(av[0] + (i == 0), av[1] + (i == 1), av[2] + (i == 2));
        for (int f = g_deg_off[lc]; f < nf; ++f)
          lvl[db][a][bc][f] = lvl[db - 1][a1][b1][f] + AB[i] * lvl[db - 1][a][b1][f];
      }
    }
  }
  /* HRR on the ket for each (a, b): (ab | c, d+1_i) = (ab | c+1_i, d) + CD_i (ab | c, d) */
  int ncA = ncart(la), ncB = ncart(lb), ncC = ncart(lc), ncD = ncart(ld);
  double (*kl)[ORA_NMONO4][ORA_MAXCART] = ws->kl;
  for (int ac = 0; ac < ncA; ++ac)
    for (int bc = 0; bc < ncB; ++bc) {
      int a = g_deg_off[la] + ac;
      for (int f = 0; f < nf; ++f) kl[0][f][0] = (f >= g_deg_off[lc]) ? lvl[lb][a][bc][f] : 0.0;
      for (int dd = 1; dd <= ld; ++dd)
        for (int dc = 0; dc < ncart(dd); ++dc) {
          const int *dv = g_mono[g_deg_off[dd] + dc];
          int i = first_axis(dv);
          int d1v[3] = {dv[0], dv[1], dv[2]};
          d1v[i] -= 1;
          int d1 = midx(d1v[0], d1v[1], d1v[2]) - g_deg_off[dd - 1];
          for (int c = g_deg_off[lc]; c < g_deg_off[F - dd + 1]; ++c) {
            const int *cv = g_mono[c];
            int c1 = midx(cv[0] + (i == 0), cv[1] + (i == 1), cv[2] + (i == 2));
            kl[dd][c][dc] = kl[dd - 1][c1][d1] + CD[i] * kl[dd - 1][c][d1];
          }
        }
      for (int cc = 0; cc < ncC; ++cc)
        for (int dc = 0; dc < ncD; ++dc) ws->cart[ac][bc][cc][dc] = kl[ld][g_deg_off[lc] + cc][dc];
    }
}

static void make_shell(const ora_basis *b, int s, ora_shell *sh) {
  sh->l = b->l[s];
  sh->n = b->nprim[s];
  sh->alpha = b->alpha + b->prim_off[s];
  sh->w = b->w + b->prim_off[s];
  for (int i = 0; i < 3; ++i) sh->A[i] = b->xyz[3 * b->atom[s] + i];
}

/* Spherical normalised (IJ|KL): out[((a*nJ + b)*nK + c)*nL + d]. */
static void quartet_sph(const ora_basis *B, double omega, int I, int J, int K, int L, ora_ws *ws,
                        double *out) {
  ora_shell s[4];
  make_shell(B, I, &s[0]);
  make_shell(B, J, &s[1]);
  make_shell(B, K, &s[2]);
  make_shell(B, L, &s[3]);
  quartet_cart(&s[0], &s[1], &s[2], &s[3], omega, ws);
  int l[4] = {s[0].l, s[1].l, s[2].l, s[3].l};
  int sh[4] = {I, J, K, L};
  int nc[4], ns[4];
  for (int t = 0; t < 4; ++t) {
    nc[t] = ncart(l[t]);
    ns[t] = nsph(l[t]);
  }
  /* transform index by index: t0[a'][b][c][d] etc. (plain four-fold sums) */
  for (int a = 0; a < ns[0]; ++a)
    for (int bb = 0; bb < ns[1]; ++bb)
      for (int c = 0; c < ns[2]; ++c)
        for (int d = 0; d < ns[3]; ++d) {
          double v = 0.0;
          for (int ca = 0; ca < nc[0]; ++ca) {
            double ta = sph_poly[l[0]][a][ca];
            if (ta == 0.0) continue;
            for (int cb = 0; cb < nc[1]; ++cb) {
              double tb = sph_poly[l[1]][bb][cb];
              if (tb == 0.0) continue;
              for (int cc = 0; cc < nc[2]; ++cc) {
                double tc = sph_poly[l[2]][c][cc];
                if (tc == 0.0) continue;
                for (int cd = 0; cd < nc[3]; ++cd) {
                  double td = sph_poly[l[3]][d][cd];
                  if (td == 0.0) continue;
                  v += ta * tb * tc * td * ws->cart[ca][cb][cc][cd];
                }
              }
            }
          }
          v *= B->nrm[ORA_MAXSPH * sh[0] + a] * B->nrm[ORA_MAXSPH * sh[1] + bb] *
               B->nrm[ORA_MAXSPH * sh[2] + c] * B->nrm[ORA_MAXSPH * sh[3] + d];
          out[((a * ns[1] + bb) * ns[2] + c) * ns[3] + d] = v;
        }
}

static ora_ws *ws_new(void) {
  mono_init();
  return (ora_ws *)malloc(sizeof(ora_ws));
}

/* Public: one spherical, normalised shell quartet. */
int ora_quartet(const void *vb, double omega, int I, int J, int K, int L, double *out) {
  const ora_basis *B = (const ora_basis *)vb;
  if (I < 0 || J < 0 || K < 0 || L < 0 || I >= B->n_shells || J >= B->n_shells ||
      K >= B->n_shells || L >= B->n_shells)
    return -1;
  ora_ws *ws = ws_new();
  quartet_sph(B, omega, I, J, K, L, ws, out);
  free(ws);
  return 0;
}

/* Public: primitive (single Gaussian, weight 1, no normalisation) Cartesian [ab|cd];
 * out[((a*ncb + b)*ncc + c)*ncd + d] over Cartesian components. */
int ora_prim_cart(const int *l4, const double *alpha4, const double *centres12, double omega,
                  double *out) {
  mono_init();
  ora_shell s[4];
  double one = 1.0;
  for (int t = 0; t < 4; ++t) {
    if (l4[t] < 0 || l4[t] > ORA_MAXL) return -1;
    s[t].l = l4[t];
    s[t].n = 1;
    s[t].alpha = &alpha4[t];
    s[t].w = &one;
    for (int i = 0; i < 3; ++i) s[t].A[i] = centres12[3 * t + i];
  }
  ora_ws *ws = ws_new();
  quartet_cart(&s[0], &s[1], &s[2], &s[3], omega, ws);
  int n[4] = {ncart(l4[0]), ncart(l4[1]), ncart(l4[2]), ncart(l4[3])};
  for (int a = 0; a < n[0]; ++a)
    for (int b = 0; b < n[1]; ++b)
      for (int c = 0; c < n[2]; ++c)
        for (int d = 0; d < n[3]; ++d) out[((a * n[1] + b) * n[2] + c) * n[3] + d] = ws->cart[a][b][c][d];
  free(ws);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Screening: orbital cutoff and Schwarz (Sec. 3.1, Eq. schwarz)              */
/* ------------------------------------------------------------------------- */

typedef struct {
  const ora_basis *B;
  double omega, tau, rcut;
  /* density-weighted screening of one K build (ora_build_K_dens): block maxima of |P|
   * (n_shells^2) and the threshold; NULL / 0 otherwise */
  const double *pm;
  double dens_tau;
  /* distance-aware screening (ora_build_K_dist): threshold, and per shell pair (n_shells^2,
   * symmetric) the centre of its most diffuse primitive pair (3), the largest distance of
   * any of its primitive-pair centres from that point, and the smallest exponent sum */
  double dist_tau;
  double *pst;   /* 4 per pair: centre xyz, spread */
  double *pexp;  /* smallest exponent sum */
  double *Q;        /* n_shells^2, symmetric: sqrt(max |(mu nu|mu nu)|) */
  unsigned char *cut_ok; /* n_shells^2: orbital-cutoff test passed */
  unsigned char *kept;   /* n_shells^2: pair kept for the quartet loops */
  double Qmax;
} ora_screen;

/* pair passes the orbital cutoff: same atom, no cutoff, or |R_A - R_B| < 2 rcut */
static int cutoff_ok(const ora_basis *B, int I, int J, double rcut) {
  if (rcut <= 0.0) return 1;
  int a = B->atom[I], b = B->atom[J];
  if (a == b) return 1;
  double d2 = 0.0;
  for (int i = 0; i < 3; ++i) {
    double t = B->xyz[3 * a + i] - B->xyz[3 * b + i];
    d2 += t * t;
  }
  return sqrt(d2) < 2.0 * rcut;
}

void ora_screen_free(void *vs) {
  ora_screen *s = (ora_screen *)vs;
  if (!s) return;
  free(s->Q); free(s->cut_ok); free(s->kept); free(s->pst); free(s->pexp);
  free(s);
}

void *ora_screen_new(const void *vb, double omega, double tau, double rcut, int nthreads) {
  const ora_basis *B = (const ora_basis *)vb;
  int n = B->n_shells;
  ora_screen *s = (ora_screen *)calloc(1, sizeof(ora_screen));
  s->B = B;
  s->omega = omega;
  s->tau = tau;
  s->rcut = rcut;
  size_t nn = (size_t)n * n;
  s->Q = (double *)calloc(nn > 0 ? nn : 1, sizeof(double));
  s->cut_ok = (unsigned char *)calloc(nn > 0 ? nn : 1, 1);
  s->kept = (unsigned char *)calloc(nn > 0 ? nn : 1, 1);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    ora_ws *ws = ws_new();
    double *blk = (double *)malloc(sizeof(double) * 625);
#pragma omp for schedule(dynamic, 4)
    for (int I = 0; I < n; ++I)
      for (int J = 0; J <= I; ++J) {
        int ok = cutoff_ok(B, I, J, rcut);
        s->cut_ok[(size_t)I * n + J] = s->cut_ok[(size_t)J * n + I] = (unsigned char)ok;
        if (!ok) continue;
        quartet_sph(B, omega, I, J, I, J, ws, blk);
        int ni = nsph(B->l[I]), nj = nsph(B->l[J]);
        double mx = 0.0;
        for (int a = 0; a < ni; ++a)
          for (int b = 0; b < nj; ++b) {
            double v = fabs(blk[((a * nj + b) * ni + a) * nj + b]);
            if (v > mx) mx = v;
          }
        double q = sqrt(mx);
        s->Q[(size_t)I * n + J] = s->Q[(size_t)J * n + I] = q;
      }
    free(blk);
    free(ws);
  }
  double qm = 0.0;
  for (size_t i = 0; i < nn; ++i)
    if (s->cut_ok[i] && s->Q[i] > qm) qm = s->Q[i];
  s->Qmax = qm;
  for (size_t i = 0; i < nn; ++i) s->kept[i] = (unsigned char)(s->cut_ok[i] && s->Q[i] * qm >= tau);
  /* pair data of the distance-aware test: a, b the smallest exponents of the two shells,
   * P* = (a A + b B)/(a + b); every primitive-pair centre (x A + y B)/(x + y) lies on AB,
   * at |x/(x+y) - a/(a+b)| |AB| from P* */
  s->pst = (double *)calloc(4 * (nn > 0 ? nn : 1), sizeof(double));
  s->pexp = (double *)calloc(nn > 0 ? nn : 1, sizeof(double));
  for (int I = 0; I < n; ++I)
    for (int J = 0; J < n; ++J) {
      const double *A = B->xyz + 3 * B->atom[I], *Bc = B->xyz + 3 * B->atom[J];
      double a = B->alpha[B->prim_off[I]], b = B->alpha[B->prim_off[J]];
      for (int k = 1; k < B->nprim[I]; ++k)
        if (B->alpha[B->prim_off[I] + k] < a) a = B->alpha[B->prim_off[I] + k];
      for (int k = 1; k < B->nprim[J]; ++k)
        if (B->alpha[B->prim_off[J] + k] < b) b = B->alpha[B->prim_off[J] + k];
      double ab = 0.0;
      for (int i = 0; i < 3; ++i) {
        s->pst[4 * ((size_t)I * n + J) + i] = (a * A[i] + b * Bc[i]) / (a + b);
        ab += (A[i] - Bc[i]) * (A[i] - Bc[i]);
      }
      ab = sqrt(ab);
      double sp = 0.0;
      for (int k = 0; k < B->nprim[I]; ++k)
        for (int kk = 0; kk < B->nprim[J]; ++kk) {
          double x = B->alpha[B->prim_off[I] + k], y = B->alpha[B->prim_off[J] + kk];
          double d = fabs(x / (x + y) - a / (a + b)) * ab;
          if (d > sp) sp = d;
        }
      s->pst[4 * ((size_t)I * n + J) + 3] = sp;
      s->pexp[(size_t)I * n + J] = a + b;
    }
  return s;
}

/* the distance-aware pair data (n_shells^2 x 4 and n_shells^2) */
void ora_screen_export_dist(const void *vs, double *pst, double *pexp) {
  const ora_screen *s = (const ora_screen *)vs;
  size_t nn = (size_t)s->B->n_shells * s->B->n_shells;
  if (pst) memcpy(pst, s->pst, 4 * nn * sizeof(double));
  if (pexp) memcpy(pexp, s->pexp, nn * sizeof(double));
}

/* Distance-aware estimate of the largest |(mu nu|lambda sigma)| of the shell quartet (IJ|KL):
 * Q_IJ Q_KL exp(-kappa rho R^2) with rho = p q / (p + q) from the two pairs' smallest exponent
 * sums p, q, kappa = omega^2 / (omega^2 + rho), and R the distance between their most
 * diffuse primitive-pair centres less both spreads (0 if negative).  For s-type primitive
 * quartets it bounds every primitive term (G_0(T) <= G_0(0) exp(-kappa T), T >= rho R^2 for
 * the slowest-decaying pair); for higher angular momentum it is an estimate. */
double ora_dist_estimate(const void *vs, int I, int J, int K, int L) {
  const ora_screen *s = (const ora_screen *)vs;
  int n = s->B->n_shells;
  size_t ij = (size_t)I * n + J, kl = (size_t)K * n + L;
  double r2 = 0.0;
  for (int i = 0; i < 3; ++i) {
    double t = s->pst[4 * ij + i] - s->pst[4 * kl + i];
    r2 += t * t;
  }
  double r = sqrt(r2) - s->pst[4 * ij + 3] - s->pst[4 * kl + 3];
  if (r < 0.0) r = 0.0;
  double p = s->pexp[ij], q = s->pexp[kl];
  double rho = p * q / (p + q), om2 = s->omega * s->omega;
  double lam = om2 * rho / (om2 + rho);
  return s->Q[ij] * s->Q[kl] * exp(-lam * r * r);
}

void ora_screen_export(const void *vs, double *Q, unsigned char *cut_ok, unsigned char *kept,
                       double *qmax) {
  const ora_screen *s = (const ora_screen *)vs;
  size_t nn = (size_t)s->B->n_shells * s->B->n_shells;
  if (Q) memcpy(Q, s->Q, nn * sizeof(double));
  if (cut_ok) memcpy(cut_ok, s->cut_ok, nn);
  if (kept) memcpy(kept, s->kept, nn);
  if (qmax) *qmax = s->Qmax;
}

double ora_dist_estimate(const void *vs, int I, int J, int K, int L);

static inline int keep4(const ora_screen *s, int I, int J, int K, int L) {
  int n = s->B->n_shells;
  size_t ij = (size_t)I * n + J, kl = (size_t)K * n + L;
  if (!(s->kept[ij] && s->kept[kl] && s->Q[ij] * s->Q[kl] >= s->tau)) return 0;
  if (s->pm) {
    /* density-weighted test: the quartet's K updates multiply the density blocks
     * (J,L), (J,K), (I,L), (I,K); drop it when Q_IJ Q_KL times their largest |P| is below
     * dens_tau (the same value for all eight orderings of the quartet) */
    double m = s->pm[(size_t)J * n + L];
    double t = s->pm[(size_t)J * n + K];
    if (t > m) m = t;
    t = s->pm[(size_t)I * n + L];
    if (t > m) m = t;
    t = s->pm[(size_t)I * n + K];
    if (t > m) m = t;
    if (s->Q[ij] * s->Q[kl] * m < s->dens_tau) return 0;
  }
  if (s->dist_tau > 0.0 && ora_dist_estimate(s, I, J, K, L) < s->dist_tau) return 0;
  return 1;
}

/* pair class index of (l1, l2): ss 0, ps 1, pp 2, ds 3, dp 4, dd 5 */
static inline int pair_class(int l1, int l2) {
  int hi = l1 > l2 ? l1 : l2, lo = l1 > l2 ? l2 : l1;
  return hi * (hi + 1) / 2 + lo;
}
/* quartet class index of two pair classes: (hi, lo) -> hi(hi+1)/2 + lo, 21 classes */
static inline int quartet_class(int pc1, int pc2) {
  int hi = pc1 > pc2 ? pc1 : pc2, lo = pc1 > pc2 ? pc2 : pc1;
  return hi * (hi + 1) / 2 + lo;
}

/* Number of canonical quartets kept (I>=J, K>=L, pair(IJ) >= pair(KL)), per class (21)
 * and in total (counts[21]). */
void ora_count_quartets(const void *vs, long long *counts) {
  const ora_screen *s = (const ora_screen *)vs;
  const ora_basis *B = s->B;
  int n = B->n_shells;
  for (int c = 0; c < 22; ++c) counts[c] = 0;
  for (int I = 0; I < n; ++I)
    for (int J = 0; J <= I; ++J) {
      long long ij = (long long)I * (I + 1) / 2 + J;
      if (!s->kept[(size_t)I * n + J]) continue;
      int pc1 = pair_class(B->l[I], B->l[J]);
      for (int K = 0; K < n; ++K)
        for (int L = 0; L <= K; ++L) {
          long long kl = (long long)K * (K + 1) / 2 + L;
          if (kl > ij) break;
          if (!keep4(s, I, J, K, L)) continue;
          int qc = quartet_class(pc1, pair_class(B->l[K], B->l[L]));
          counts[qc]++;
          counts[21]++;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Exchange matrix                                                            */
/* ------------------------------------------------------------------------- */

/* Plain definition: every ordered shell quartet (I J K L) that is kept contributes
 * K_{mu nu} += (mu lambda | nu sigma) P_{lambda sigma}, mu in I, lambda in J, nu in K,
 * sigma in L. */
static void build_K_plain(const ora_screen *s, const double *P, double *Kout) {
  const ora_basis *B = s->B;
  int n = B->n_shells, nb = B->n_bf;
  memset(Kout, 0, sizeof(double) * (size_t)nb * nb);
#pragma omp parallel
  {
    ora_ws *ws = ws_new();
    double *blk = (double *)malloc(sizeof(double) * 625);
    /* each thread owns whole rows mu in shell I: no races */
#pragma omp for schedule(dynamic, 1)
    for (int I = 0; I < n; ++I)
      for (int Ks = 0; Ks < n; ++Ks)
        for (int J = 0; J < n; ++J)
          for (int L = 0; L < n; ++L) {
            if (!keep4(s, I, J, Ks, L)) continue;
            quartet_sph(B, s->omega, I, J, Ks, L, ws, blk);
            int ni = nsph(B->l[I]), nj = nsph(B->l[J]), nk = nsph(B->l[Ks]), nl = nsph(B->l[L]);
            int oi = B->bf_off[I], oj = B->bf_off[J], ok = B->bf_off[Ks], ol = B->bf_off[L];
            for (int a = 0; a < ni; ++a)
              for (int c = 0; c < nk; ++c) {
                double acc = 0.0;
                for (int b = 0; b < nj; ++b)
                  for (int d = 0; d < nl; ++d)
                    acc += blk[((a * nj + b) * nk + c) * nl + d] * P[(size_t)(oj + b) * nb + ol + d];
                Kout[(size_t)(oi + a) * nb + ok + c] += acc;
              }
          }
    free(blk);
    free(ws);
  }
}

/* Symmetric form: canonical quartets I>=J, K>=L, pair(IJ) >= pair(KL), each evaluated
 * once, scaled by the degeneracy 1/2^[I=J] 1/2^[K=L] 1/2^[IJ=KL], added to four blocks
 * of a half matrix A (the other four permutations are the transposes), K = A + A^T. */
static void build_K_sym(const ora_screen *s, const double *P, double *Kout, int nthreads) {
  const ora_basis *B = s->B;
  int n = B->n_shells, nb = B->n_bf;
  size_t nn = (size_t)nb * nb;
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
  double *priv = (double *)calloc(nn * nt, sizeof(double));
  long long npairs = (long long)n * (n + 1) / 2;
#pragma omp parallel num_threads(nt)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double *A = priv + nn * tid;
    ora_ws *ws = ws_new();
    double *blk = (double *)malloc(sizeof(double) * 625);
#pragma omp for schedule(dynamic, 1)
    for (long long ij = 0; ij < npairs; ++ij) {
      int I = (int)((sqrt(8.0 * ij + 1.0) - 1.0) / 2.0);
      while ((long long)I * (I + 1) / 2 > ij) --I;
      while ((long long)(I + 1) * (I + 2) / 2 <= ij) ++I;
      int J = (int)(ij - (long long)I * (I + 1) / 2);
      if (!s->kept[(size_t)I * n + J]) continue;
      for (int Ks = 0; Ks <= I; ++Ks)
        for (int L = 0; L <= Ks; ++L) {
          long long kl = (long long)Ks * (Ks + 1) / 2 + L;
          if (kl > ij) break;
          if (!keep4(s, I, J, Ks, L)) continue;
          double deg = 1.0;
          if (I == J) deg *= 0.5;
          if (Ks == L) deg *= 0.5;
          if (ij == kl) deg *= 0.5;
          quartet_sph(B, s->omega, I, J, Ks, L, ws, blk);
          int ni = nsph(B->l[I]), nj = nsph(B->l[J]), nk = nsph(B->l[Ks]), nl = nsph(B->l[L]);
          int oi = B->bf_off[I], oj = B->bf_off[J], ok = B->bf_off[Ks], ol = B->bf_off[L];
          for (int a = 0; a < ni; ++a)
            for (int b = 0; b < nj; ++b)
              for (int c = 0; c < nk; ++c)
                for (int d = 0; d < nl; ++d) {
                  double v = deg * blk[((a * nj + b) * nk + c) * nl + d];
                  int mu = oi + a, la = oj + b, nu = ok + c, si = ol + d;
                  A[(size_t)mu * nb + nu] += v * P[(size_t)la * nb + si];
                  A[(size_t)mu * nb + si] += v * P[(size_t)la * nb + nu];
                  A[(size_t)la * nb + nu] += v * P[(size_t)mu * nb + si];
                  A[(size_t)la * nb + si] += v * P[(size_t)mu * nb + nu];
                }
        }
    }
    free(blk);
    free(ws);
  }
  for (int mu = 0; mu < nb; ++mu)
    for (int nu = 0; nu < nb; ++nu) {
      double acc = 0.0;
      for (int t = 0; t < nt; ++t)
        acc += priv[nn * t + (size_t)mu * nb + nu] + priv[nn * t + (size_t)nu * nb + mu];
      Kout[(size_t)mu * nb + nu] = acc;
    }
  free(priv);
}

/* E_K = sum_{mu nu} P_{mu nu} K_{mu nu}, Neumaier-compensated. */
double ora_trace_PK(int nb, const double *P, const double *K) {
  double sum = 0.0, comp = 0.0;
  size_t nn = (size_t)nb * nb;
  for (size_t i = 0; i < nn; ++i) {
    double x = P[i] * K[i];
    double t = sum + x;
    if (fabs(sum) >= fabs(x))
      comp += (sum - t) + x;
    else
      comp += (x - t) + sum;
    sum = t;
  }
  return sum + comp;
}

/* mode 0: plain four-fold loop; mode 1: symmetric canonical loop. Returns E_K. */
double ora_build_K(const void *vs, const double *P, int mode, int nthreads, double *Kout) {
  const ora_screen *s = (const ora_screen *)vs;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  if (mode == 0)
    build_K_plain(s, P, Kout);
  else
    build_K_sym(s, P, Kout, nthreads);
  return ora_trace_PK(s->B->n_bf, P, Kout);
}

/* The same K build with the density-weighted quartet test added to the keep rule
 * (dens_tau > 0): Q_IJ Q_KL max(|P| over the blocks (J,L), (J,K), (I,L), (I,K)) >= dens_tau.
 * pm_out (n_shells^2, may be NULL) receives the block maxima of |P|. */
double ora_build_K_dens(void *vs, const double *P, int mode, int nthreads, double dens_tau, double *Kout,
                        double *pm_out) {
  ora_screen *s = (ora_screen *)vs;
  const ora_basis *B = s->B;
  int n = B->n_shells, nb = B->n_bf;
  double *pm = (double *)calloc((size_t)n * n > 0 ? (size_t)n * n : 1, sizeof(double));
  for (int I = 0; I < n; ++I)
    for (int J = 0; J < n; ++J) {
      double m = 0.0;
      for (int a = 0; a < nsph(B->l[I]); ++a)
        for (int b = 0; b < nsph(B->l[J]); ++b) {
          double v = fabs(P[(size_t)(B->bf_off[I] + a) * nb + B->bf_off[J] + b]);
          if (v > m) m = v;
        }
      pm[(size_t)I * n + J] = m;
    }
  if (pm_out) memcpy(pm_out, pm, sizeof(double) * (size_t)n * n);
  s->pm = pm;
  s->dens_tau = dens_tau;
  double e = ora_build_K(vs, P, mode, nthreads, Kout);
  s->pm = NULL;
  s->dens_tau = 0.0;
  free(pm);
  return e;
}

/* The same K build with the distance-aware quartet test added to the keep rule
 * (dist_tau > 0): ora_dist_estimate(I, J, K, L) >= dist_tau (symmetric in the eight
 * orderings of the quartet). */
double ora_build_K_dist(void *vs, const double *P, int mode, int nthreads, double dist_tau, double *Kout) {
  ora_screen *s = (ora_screen *)vs;
  s->dist_tau = dist_tau;
  double e = ora_build_K(vs, P, mode, nthreads, Kout);
  s->dist_tau = 0.0;
  return e;
}

/* One block K_{mu nu}, mu in shell I, nu in shell Ks, by the plain definition (sum over
 * all J, L).  out is n_sph(I) x n_sph(Ks), row-major. */
int ora_K_block(const void *vs, const double *P, int I, int Ks, double *out) {
  const ora_screen *s = (const ora_screen *)vs;
  const ora_basis *B = s->B;
  int n = B->n_shells, nb = B->n_bf;
  if (I < 0 || I >= n || Ks < 0 || Ks >= n) return -1;
  int ni = nsph(B->l[I]), nk = nsph(B->l[Ks]);
  for (int t = 0; t < ni * nk; ++t) out[t] = 0.0;
  ora_ws *ws = ws_new();
  double *blk = (double *)malloc(sizeof(double) * 625);
  for (int J = 0; J < n; ++J)
    for (int L = 0; L < n; ++L) {
      if (!keep4(s, I, J, Ks, L)) continue;
      quartet_sph(B, s->omega, I, J, Ks, L, ws, blk);
      int nj = nsph(B->l[J]), nl = nsph(B->l[L]);
      int oj = B->bf_off[J], ol = B->bf_off[L];
      for (int a = 0; a < ni; ++a)
        for (int c = 0; c < nk; ++c) {
          double acc = 0.0;
          for (int b = 0; b < nj; ++b)
            for (int d = 0; d < nl; ++d)
              acc += blk[((a * nj + b) * nk + c) * nl + d] * P[(size_t)(oj + b) * nb + ol + d];
          out[a * nk + c] += acc;
        }
    }
  free(blk);
  free(ws);
  return 0;
}

/* Evaluate n_quartets canonical quartets given as (I,J,K,L) rows, return the sum of
 * squares of their values (used only to time the oracle on a bounded sample). */
double ora_eval_quartets(const void *vs, long long n_quartets, const int *ijkl, int nthreads) {
  const ora_screen *s = (const ora_screen *)vs;
  double total = 0.0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : total)
  {
    ora_ws *ws = ws_new();
    double *blk = (double *)malloc(sizeof(double) * 625);
#pragma omp for schedule(dynamic, 16)
    for (long long q = 0; q < n_quartets; ++q) {
      const int *r = ijkl + 4 * q;
      quartet_sph(s->B, s->omega, r[0], r[1], r[2], r[3], ws, blk);
      int nt = nsph(s->B->l[r[0]]) * nsph(s->B->l[r[1]]) * nsph(s->B->l[r[2]]) * nsph(s->B->l[r[3]]);
      for (int t = 0; t < nt; ++t) total += blk[t] * blk[t];
    }
    free(blk);
    free(ws);
  }
  return total;
}

int ora_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
