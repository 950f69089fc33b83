/*
 * FP64 CPU oracle for the Wannier-interpolated electron linewidth.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code with the CUDA path.
 *
 * What it computes (EPW, Ponce et al. 2016):
 *   - Eq. (linewidthel), Sec. "Electron and phonon self-energies": the electron
 *     linewidth Im Sigma_nk(w, T) = pi sum_{m,nu} int dq/Omega_BZ |g_mn,nu(k,q)|^2
 *       { [n_qnu + f_mk+q] delta(w - (e_mk+q - eF) + w_qnu)
 *       + [n_qnu + 1 - f_mk+q] delta(w - (e_mk+q - eF) - w_qnu) },
 *     evaluated on shell, w = e_nk - eF, so E_F cancels inside the deltas
 *     (the Sec. "Examples" discussion of Sigma''(e_nk)).
 *   - n = Bose-Einstein, f = Fermi-Dirac occupations (the definitions that
 *     follow Eq. phselfenergy), with k_B = 8.617333262e-5 eV/K.
 *   - The BZ integral is a weighted sum over the q list (weights w_q).
 *   - Gaussian delta: delta(x) = exp(-(x/sigma)^2) / (sigma sqrt(pi)).
 *   - Wannier interpolation (Sec. "Electron-phonon coupling in polar
 *     materials", step (iii), and the rotation matrices of the overlap
 *     equation there): with phases e^{2 pi i k.R} in crystal coordinates,
 *       H(k)   = sum_Re wRe e^{2pi i k.Re} H(Re),  H(k) U_k = U_k diag(e_k),
 *       D(q)   = sum_R  wR  e^{2pi i q.R} Phi(R) / sqrt(M_kappa M_kappa'),
 *                D(q) e_nu = w_nu^2 e_nu,
 *       g(Re,q)= sum_Rp wRp e^{2pi i q.Rp} g(Re,Rp),
 *       g(k,q) = sum_Re wRe e^{2pi i k.Re} g(Re,q),
 *       g_mn,nu(k,q) = sum_{kappa alpha} [U_k+q^dagger g_{kappa alpha}(k,q) U_k]_mn
 *                       e_{kappa alpha,nu}(q) / sqrt(2 M_kappa w_qnu).
 *     Modes with w_qnu < omega_min are left out (w -> 0 at Gamma).
 *   - The adjoint of L = sum_{k,n} c_nk Im Sigma_nk with respect to g(Re,Rp)
 *     (reported as dL/dRe g + i dL/dIm g), the temperature and the Fermi level.
 *   - Per (q, nu) sums over a k list of the same vertex: the phonon self-energy
 *     Pi''_qnu of Eq. (linewidthph) on shell (w = w_qnu, sign as printed), the
 *     coupling strength lambda_qnu of Eq. (lambdaEQ) with N(E_F) from the k
 *     list, and the nesting function of Eq. (nestingfct); the isotropic
 *     Eliashberg function of Eq. (isotropiceliash) from w_qnu and lambda_qnu.
 *   - The complex electron self-energy of Eq. (elselfenergy) on a frequency grid
 *     and the spectral function of Eq. (spectral_funct).
 *
 * Every eigensolve is a plain cyclic complex Jacobi iteration on the Hermitian
 * part (X + X^dagger)/2, run to full double precision; eigenvalues ascend.
 * Sums of positive linewidth terms are compensated (Neumaier).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define KB_EV 8.617333262e-5
#define TWO_PI 6.283185307179586476925286766559

typedef struct {
  int nw, nat;
  const double *mass;                                          /* [nat] */
  int nRe; const int *Re; const double *wRe; const double *H;  /* H [nRe][nw][nw] complex */
  int nRph; const int *Rph; const double *wRph; const double *Phi; /* [nRph][3nat][3nat] */
  int nRp; const int *Rp; const double *wRp; const double *g;  /* [nRe][nRp][3nat][nw][nw] */
  /* long-range (polar) part, used when polar != 0: lattice vectors A (rows), eps_inf [3][3],
     Born charges Z* [nat][3][3] (Z*_{kappa, b alpha}), damping alpha, prefactor, |n_i| <= gmax */
  int polar;
  const double *pA, *peps, *pZ;
  double palpha, ppref;
  int pgmax;
} oracle_model;

typedef struct {
  double T;         /* K */
  double EF;        /* eV */
  double sigma;     /* eV */
  double omega_min; /* eV */
} oracle_params;

/* ---------------------------------------------------------------- helpers */

static cplx cz(const double *p, long i) { return p[2 * i] + I * p[2 * i + 1]; }

/* e^{2 pi i x.R} with x.R reduced to [-1/2, 1/2] before the trigonometric call. */
static cplx phase(const double x[3], const int R[3]) {
  double a = x[0] * R[0] + x[1] * R[1] + x[2] * R[2];
  a -= nearbyint(a);
  return cexp(I * TWO_PI * a);
}

typedef struct { double s, c; } nsum; /* Neumaier compensated sum */
static void nsum_add(nsum *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double nsum_get(const nsum *a) { return a->s + a->c; }

double oracle_bose(double w, double T) {
  if (T <= 0.0) return 0.0;
  double x = w / (KB_EV * T);
  if (x > 700.0) return 0.0;
  return 1.0 / expm1(x);
}

double oracle_fermi(double e, double EF, double T) {
  double d = e - EF;
  if (T <= 0.0) return d < 0.0 ? 1.0 : (d > 0.0 ? 0.0 : 0.5);
  double x = d / (KB_EV * T);
  if (x > 0.0) { double t = exp(-x); return t / (1.0 + t); }
  return 1.0 / (1.0 + exp(x));
}

/* f (1 - f) = -kT df/de, written as t / (1 + t)^2 with t = exp(-|x|): the same
   value as forming 1 - f, but without its cancellation once f rounds to 1. */
double oracle_fermi_slope(double e, double EF, double T) {
  if (T <= 0.0) return 0.0;
  double t = exp(-fabs((e - EF) / (KB_EV * T)));
  return t / ((1.0 + t) * (1.0 + t));
}

/* f(ea) - f(eb) without the cancellation of subtracting two rounded occupations:
   with a, b = (e - E_F)/kT, d = b - a and S = |a| + |b| (d + S >= 0, S - d >= 0),
     f(a) - f(b) = 2 sinh(d/2) e^{-S/2} / ((1 + e^{-|a|}) (1 + e^{-|b|})),
   the sinh written with expm1 of d or -d so that no exponent is positive.
   T = 0: the step occupations (f(E_F) = 1/2). */
double oracle_fermi_diff(double ea, double eb, double EF, double T) {
  if (T <= 0.0) return oracle_fermi(ea, EF, T) - oracle_fermi(eb, EF, T);
  const double a = (ea - EF) / (KB_EV * T), b = (eb - EF) / (KB_EV * T);
  const double d = b - a, S = fabs(a) + fabs(b);
  const double num = d >= 0.0 ? -exp(0.5 * (d - S)) * expm1(-d) : exp(-0.5 * (d + S)) * expm1(d);
  return num / ((1.0 + exp(-fabs(a))) * (1.0 + exp(-fabs(b))));
}

double oracle_gauss(double x, double sigma) {
  double y = x / sigma;
  return exp(-y * y) / (sigma * sqrt(M_PI));
}

/* delta(x + w) - delta(x - w) for the Gaussian above.  The two exponents differ
   by 4 x w / sigma^2, so with a = x/sigma, b = w/sigma
     delta(x + w) - delta(x - w) = -2 exp(-(a^2 + b^2)) sinh(2 a b) / (sigma sqrt(pi)),
   which keeps full relative accuracy when w << sigma, where the plain difference
   subtracts two nearly equal numbers.  For |2ab| > 1 the plain difference is
   well conditioned (the two values differ by a factor e^2 or more) and the
   product form could overflow in sinh, so that branch takes the difference. */
double oracle_gauss_diff(double x, double w, double sigma) {
  const double a = x / sigma, b = w / sigma;
  if (fabs(2.0 * a * b) > 1.0) return oracle_gauss(x + w, sigma) - oracle_gauss(x - w, sigma);
  return -2.0 * exp(-(a * a + b * b)) * sinh(2.0 * a * b) / (sigma * sqrt(M_PI));
}

/* ------------------------------------------------------------- eigensolver */

/* Cyclic complex Jacobi.  A: n x n row-major (overwritten), w: ascending
 * eigenvalues, V: column j is the eigenvector of w[j].  Returns sweeps used,
 * or -1 if 100 sweeps did not converge. */
int oracle_eigh(int n, cplx *A, double *w, cplx *V) {
  for (int i = 0; i < n; i++) {
    A[i * n + i] = creal(A[i * n + i]);
    for (int j = i + 1; j < n; j++) {
      cplx a = 0.5 * (A[i * n + j] + conj(A[j * n + i]));
      A[i * n + j] = a;
      A[j * n + i] = conj(a);
    }
  }
  for (int i = 0; i < n * n; i++) V[i] = 0.0;
  for (int i = 0; i < n; i++) V[i * n + i] = 1.0;
  int sweep;
  int converged = 0;
  for (sweep = 0; sweep < 100; sweep++) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; i++)
      for (int j = 0; j < n; j++) {
        double m2 = creal(A[i * n + j]) * creal(A[i * n + j]) + cimag(A[i * n + j]) * cimag(A[i * n + j]);
        tot += m2;
        if (i != j) off += m2;
      }
    if (off <= 1e-30 * tot || off == 0.0) { converged = 1; break; }
    for (int p = 0; p < n - 1; p++)
      for (int q = p + 1; q < n; q++) {
        cplx apq = A[p * n + q];
        double ab = cabs(apq);
        if (ab == 0.0) continue;
        cplx e = apq / ab;
        double theta = (creal(A[q * n + q]) - creal(A[p * n + p])) / (2.0 * ab);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        /* G = I except G_pp = c, G_pq = s e, G_qp = -s conj(e), G_qq = c;  A <- G^dagger A G, V <- V G */
        for (int r = 0; r < n; r++) {
          cplx arp = A[r * n + p], arq = A[r * n + q];
          A[r * n + p] = c * arp - s * conj(e) * arq;
          A[r * n + q] = s * e * arp + c * arq;
          cplx vrp = V[r * n + p], vrq = V[r * n + q];
          V[r * n + p] = c * vrp - s * conj(e) * vrq;
          V[r * n + q] = s * e * vrp + c * vrq;
        }
        for (int r = 0; r < n; r++) {
          cplx apr = A[p * n + r], aqr = A[q * n + r];
          A[p * n + r] = c * apr - s * e * aqr;
          A[q * n + r] = s * conj(e) * apr + c * aqr;
        }
      }
  }
  for (int i = 0; i < n; i++) w[i] = creal(A[i * n + i]);
  /* selection sort, ascending, carrying eigenvector columns */
  for (int i = 0; i < n; i++) {
    int m = i;
    for (int j = i + 1; j < n; j++) if (w[j] < w[m]) m = j;
    if (m != i) {
      double tw = w[i]; w[i] = w[m]; w[m] = tw;
      for (int r = 0; r < n; r++) { cplx tv = V[r * n + i]; V[r * n + i] = V[r * n + m]; V[r * n + m] = tv; }
    }
  }
  return converged ? sweep : -1;
}

/* ------------------------------------------------------- interpolation */

/* H(k) = sum_Re wRe e^{2pi i k.Re} H(Re) */
void oracle_hk(const oracle_model *m, const double k[3], cplx *Hk) {
  int nw = m->nw;
  for (int i = 0; i < nw * nw; i++) Hk[i] = 0.0;
  for (int r = 0; r < m->nRe; r++) {
    cplx p = phase(k, m->Re + 3 * r) * (m->wRe ? m->wRe[r] : 1.0);
    for (int i = 0; i < nw * nw; i++) Hk[i] += p * cz(m->H, (long)r * nw * nw + i);
  }
}

/* Bands at k: eps [nk][nw], U [nk][nw][nw] (columns = eigenvectors). */
int oracle_bands(const oracle_model *m, int nk, const double *k, double *eps, double *U) {
  int nw = m->nw, bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
  for (int ik = 0; ik < nk; ik++) {
    cplx *Hk = malloc(sizeof(cplx) * nw * nw), *V = malloc(sizeof(cplx) * nw * nw);
    oracle_hk(m, k + 3 * ik, Hk);
    if (oracle_eigh(nw, Hk, eps + (long)ik * nw, V) < 0) bad++;
    if (U) memcpy(U + 2L * ik * nw * nw, V, sizeof(cplx) * nw * nw);
    free(Hk); free(V);
  }
  return bad ? -1 : 0;
}

/* D(q) (mass scaled) */
void oracle_dynmat(const oracle_model *m, const double q[3], cplx *D) {
  int n = 3 * m->nat;
  for (int i = 0; i < n * n; i++) D[i] = 0.0;
  for (int r = 0; r < m->nRph; r++) {
    cplx p = phase(q, m->Rph + 3 * r) * (m->wRph ? m->wRph[r] : 1.0);
    for (int i = 0; i < n * n; i++) D[i] += p * cz(m->Phi, (long)r * n * n + i);
  }
  for (int a = 0; a < n; a++)
    for (int b = 0; b < n; b++) D[a * n + b] /= sqrt(m->mass[a / 3] * m->mass[b / 3]);
}

/* Phonons at q: omega [nq][3nat] (= sign(w2) sqrt|w2|), evec [nq][3nat][3nat] (columns = modes). */
int oracle_phonons(const oracle_model *m, int nq, const double *q, double *omega, double *evec) {
  int n = 3 * m->nat, bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
  for (int iq = 0; iq < nq; iq++) {
    cplx *D = malloc(sizeof(cplx) * n * n), *V = malloc(sizeof(cplx) * n * n);
    double *w2 = malloc(sizeof(double) * n);
    oracle_dynmat(m, q + 3 * iq, D);
    if (oracle_eigh(n, D, w2, V) < 0) bad++;
    for (int j = 0; j < n; j++) omega[(long)iq * n + j] = (w2[j] >= 0 ? 1.0 : -1.0) * sqrt(fabs(w2[j]));
    if (evec) memcpy(evec + 2L * iq * n * n, V, sizeof(cplx) * n * n);
    free(D); free(V); free(w2);
  }
  return bad ? -1 : 0;
}

/* g(k,q) in the Wannier basis by the direct double sum over (Re, Rp).
 * out [3nat][nw][nw] */
void oracle_g_wannier_direct(const oracle_model *m, const double k[3], const double q[3], double *out) {
  int nw = m->nw, nc = 3 * m->nat * nw * nw;
  cplx *o = (cplx *)out;
  for (int i = 0; i < nc; i++) o[i] = 0.0;
  for (int a = 0; a < m->nRe; a++) {
    cplx pk = phase(k, m->Re + 3 * a) * (m->wRe ? m->wRe[a] : 1.0);
    for (int b = 0; b < m->nRp; b++) {
      cplx p = pk * phase(q, m->Rp + 3 * b) * (m->wRp ? m->wRp[b] : 1.0);
      const double *gab = m->g + 2L * ((long)a * m->nRp + b) * nc;
      for (int i = 0; i < nc; i++) o[i] += p * cz(gab, i);
    }
  }
}

/* First interpolation step: g(Re,q) = sum_Rp wRp e^{2pi i q.Rp} g(Re,Rp); out [nRe][3nat][nw][nw] */
void oracle_g_Re_q(const oracle_model *m, const double q[3], cplx *out) {
  int nc = 3 * m->nat * m->nw * m->nw;
  for (long i = 0; i < (long)m->nRe * nc; i++) out[i] = 0.0;
  for (int b = 0; b < m->nRp; b++) {
    cplx p = phase(q, m->Rp + 3 * b) * (m->wRp ? m->wRp[b] : 1.0);
    for (int a = 0; a < m->nRe; a++) {
      const double *gab = m->g + 2L * ((long)a * m->nRp + b) * nc;
      cplx *oa = out + (long)a * nc;
      for (int i = 0; i < nc; i++) oa[i] += p * cz(gab, i);
    }
  }
}

/* Second step: g(k,q) = sum_Re wRe e^{2pi i k.Re} g(Re,q); out [3nat][nw][nw] */
static void g_k_from_Re_q(const oracle_model *m, const cplx *gReq, const double k[3], cplx *out) {
  int nc = 3 * m->nat * m->nw * m->nw;
  for (int i = 0; i < nc; i++) out[i] = 0.0;
  for (int a = 0; a < m->nRe; a++) {
    cplx p = phase(k, m->Re + 3 * a) * (m->wRe ? m->wRe[a] : 1.0);
    for (int i = 0; i < nc; i++) out[i] += p * gReq[(long)a * nc + i];
  }
}

/* Long-range part of the vertex (Sec. "Electron-phonon coupling in polar materials", Eq. (long-range),
 * with the overlap in its small-(q+G) form [U_k U_k+q^dagger]_nm of that section):
 *   g^L_mn,nu(k,q) = i C_nu(q) [U_k+q^dagger U_k]_mn   (our columns-are-eigenvectors convention),
 *   C_nu(q) = pref sum_{kappa, a} E[kappa a][nu] sum_{G, q+G != 0} damp(q+G) ((q+G) . Z*_kappa)_a / ((q+G) . eps . (q+G)),
 * with E = e / sqrt(2 M w) (the (hbar / 2 M w)^{1/2} e of the equation), (x . Z*_kappa)_a = sum_b x_b Z*_{kappa,b a},
 * damp(x) = exp(-x . eps . x / (4 alpha)) and G = sum_i n_i b_i (|n_i| <= gmax, b_i . a_j = 2 pi delta_ij),
 * q + G Cartesian.  The printed equation has neither the prefactor nor a convergence factor; both are
 * inputs here.  C is zero when the model has no polar part. */
static void polar_factors(const oracle_model *m, const double q[3], const cplx *E, cplx *C) {
  const int nm = 3 * m->nat;
  for (int nu = 0; nu < nm; nu++) C[nu] = 0.0;
  if (!m->polar) return;
  const double *A = m->pA;
  /* b = 2 pi (A^{-1})^T, by cofactors */
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  double inv[9];
  inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  double b[3][3]; /* b[i][c] = 2 pi inv[c][i] */
  for (int i = 0; i < 3; i++)
    for (int c = 0; c < 3; c++) b[i][c] = TWO_PI * inv[c * 3 + i];
  double *F = calloc((size_t)nm, sizeof(double));
  const int G = m->pgmax;
  for (int n1 = -G; n1 <= G; n1++)
    for (int n2 = -G; n2 <= G; n2++)
      for (int n3 = -G; n3 <= G; n3++) {
        double x[3];
        for (int c = 0; c < 3; c++)
          x[c] = (q[0] + n1) * b[0][c] + (q[1] + n2) * b[1][c] + (q[2] + n3) * b[2][c];
        double xex = 0.0;
        for (int c = 0; c < 3; c++)
          for (int d = 0; d < 3; d++) xex += x[c] * m->peps[c * 3 + d] * x[d];
        if (x[0] * x[0] + x[1] * x[1] + x[2] * x[2] == 0.0) continue; /* G = -q */
        const double w = exp(-xex / (4.0 * m->palpha)) / xex;
        for (int kap = 0; kap < m->nat; kap++)
          for (int a = 0; a < 3; a++) {
            double xz = 0.0;
            for (int c = 0; c < 3; c++) xz += x[c] * m->pZ[(kap * 3 + c) * 3 + a];
            F[kap * 3 + a] += w * xz;
          }
      }
  for (int nu = 0; nu < nm; nu++) {
    cplx s = 0.0;
    for (int ka = 0; ka < nm; ka++) s += E[ka * nm + nu] * F[ka];
    C[nu] = m->ppref * s;
  }
  free(F);
}

/* Mode-basis Bloch vertex: gmn[nu][m][n] = sum_{ka} [Ukq^dag g_ka Uk]_mn E[ka][nu] (+ i C_nu [Ukq^dag Uk]_mn
 * when C != NULL), E[ka][nu] = e_{ka,nu} / sqrt(2 M_k w_nu), or 0 for modes below omega_min. */
static void bloch_mode_vertex(int nw, int nm, const cplx *gk, const cplx *Uk, const cplx *Ukq,
                              const cplx *E, cplx *gmn, cplx *tmp, const cplx *C) {
  /* tmp[ka][m][n] = (Ukq^dag g_ka Uk)_mn */
  for (int ka = 0; ka < nm; ka++)
    for (int a = 0; a < nw; a++)
      for (int b = 0; b < nw; b++) {
        cplx s = 0.0;
        for (int i = 0; i < nw; i++)
          for (int j = 0; j < nw; j++)
            s += conj(Ukq[i * nw + a]) * gk[(ka * nw + i) * nw + j] * Uk[j * nw + b];
        tmp[(ka * nw + a) * nw + b] = s;
      }
  for (int nu = 0; nu < nm; nu++)
    for (int i = 0; i < nw * nw; i++) {
      cplx s = 0.0;
      for (int ka = 0; ka < nm; ka++) s += tmp[ka * nw * nw + i] * E[ka * nm + nu];
      gmn[nu * nw * nw + i] = s;
    }
  if (C)
    for (int a = 0; a < nw; a++)
      for (int b = 0; b < nw; b++) {
        cplx o = 0.0; /* [Ukq^dag Uk]_ab */
        for (int i = 0; i < nw; i++) o += conj(Ukq[i * nw + a]) * Uk[i * nw + b];
        for (int nu = 0; nu < nm; nu++) gmn[(nu * nw + a) * nw + b] += I * C[nu] * o;
      }
}

static void mode_factors(const oracle_model *m, const double *w, const cplx *ev, double omega_min, cplx *E) {
  int nm = 3 * m->nat;
  for (int ka = 0; ka < nm; ka++)
    for (int nu = 0; nu < nm; nu++)
      E[ka * nm + nu] = (w[nu] >= omega_min) ? ev[ka * nm + nu] / sqrt(2.0 * m->mass[ka / 3] * w[nu]) : 0.0;
}

/* Interpolated quantities on a k x q product:
 * eps_k [nk][nw], eps_kq [nk][nq][nw], omega [nq][3nat],
 * g [nk][nq][3nat][nw][nw] complex (mode nu, band m at k+q, band n at k). */
int oracle_interp(const oracle_model *m, int nk, const double *k, int nq, const double *q,
                  double omega_min, double *eps_k, double *eps_kq, double *omega, double *g) {
  int nw = m->nw, nm = 3 * m->nat, nc = nm * nw * nw;
  double *Uk = malloc(sizeof(cplx) * (long)nk * nw * nw);
  double *ev = malloc(sizeof(cplx) * (long)nq * nm * nm);
  int bad = oracle_bands(m, nk, k, eps_k, Uk) + oracle_phonons(m, nq, q, omega, ev);
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
  for (int iq = 0; iq < nq; iq++) {
    cplx *gReq = malloc(sizeof(cplx) * (long)m->nRe * nc);
    cplx *gk = malloc(sizeof(cplx) * nc), *tmp = malloc(sizeof(cplx) * nc);
    cplx *Hkq = malloc(sizeof(cplx) * nw * nw), *Ukq = malloc(sizeof(cplx) * nw * nw);
    cplx *E = malloc(sizeof(cplx) * nm * nm);
    double ekq[64];
    oracle_g_Re_q(m, q + 3 * iq, gReq);
    mode_factors(m, omega + (long)iq * nm, (cplx *)ev + (long)iq * nm * nm, omega_min, E);
    cplx Cp[64];
    polar_factors(m, q + 3 * iq, E, Cp);
    for (int ik = 0; ik < nk; ik++) {
      double kq[3] = {k[3 * ik] + q[3 * iq], k[3 * ik + 1] + q[3 * iq + 1], k[3 * ik + 2] + q[3 * iq + 2]};
      oracle_hk(m, kq, Hkq);
      if (oracle_eigh(nw, Hkq, ekq, Ukq) < 0) bad++;
      memcpy(eps_kq + ((long)ik * nq + iq) * nw, ekq, sizeof(double) * nw);
      g_k_from_Re_q(m, gReq, k + 3 * ik, gk);
      bloch_mode_vertex(nw, nm, gk, (cplx *)Uk + (long)ik * nw * nw, Ukq, E,
                        (cplx *)g + ((long)ik * nq + iq) * nc, tmp, m->polar ? Cp : NULL);
    }
    free(gReq); free(gk); free(tmp); free(Hkq); free(Ukq); free(E);
  }
  free(Uk); free(ev);
  return bad ? -1 : 0;
}

/* ------------------------------------------------------------- linewidth */

/* Im Sigma [nk][nw] (eV).  wq == NULL means 1/nq. */
int oracle_linewidth(const oracle_model *m, int nk, const double *k, int nq, const double *q,
                     const double *wq, const oracle_params *pr, double *imsig) {
  int nw = m->nw, nm = 3 * m->nat, nc = nm * nw * nw;
  double *epsk = malloc(sizeof(double) * (long)nk * nw);
  double *Uk = malloc(sizeof(cplx) * (long)nk * nw * nw);
  int bad = oracle_bands(m, nk, k, epsk, Uk);
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  nsum *acc = calloc((size_t)nthr * nk * nw, sizeof(nsum));
#pragma omp parallel reduction(+ : bad)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    nsum *my = acc + (long)tid * nk * nw;
    cplx *gReq = malloc(sizeof(cplx) * (long)m->nRe * nc);
    cplx *gk = malloc(sizeof(cplx) * nc), *tmp = malloc(sizeof(cplx) * nc), *gmn = malloc(sizeof(cplx) * nc);
    cplx *Hkq = malloc(sizeof(cplx) * nw * nw), *Ukq = malloc(sizeof(cplx) * nw * nw);
    cplx *D = malloc(sizeof(cplx) * nm * nm), *ev = malloc(sizeof(cplx) * nm * nm), *E = malloc(sizeof(cplx) * nm * nm);
    double w2[64], w[64], ekq[64];
#pragma omp for schedule(dynamic)
    for (int iq = 0; iq < nq; iq++) {
      const double *qq = q + 3 * iq;
      double wqi = wq ? wq[iq] : 1.0 / nq;
      oracle_dynmat(m, qq, D);
      if (oracle_eigh(nm, D, w2, ev) < 0) bad++;
      for (int j = 0; j < nm; j++) w[j] = (w2[j] >= 0 ? 1.0 : -1.0) * sqrt(fabs(w2[j]));
      mode_factors(m, w, ev, pr->omega_min, E);
      cplx Cp[64];
      polar_factors(m, qq, E, Cp);
      oracle_g_Re_q(m, qq, gReq);
      for (int ik = 0; ik < nk; ik++) {
        double kq[3] = {k[3 * ik] + qq[0], k[3 * ik + 1] + qq[1], k[3 * ik + 2] + qq[2]};
        oracle_hk(m, kq, Hkq);
        if (oracle_eigh(nw, Hkq, ekq, Ukq) < 0) bad++;
        g_k_from_Re_q(m, gReq, k + 3 * ik, gk);
        bloch_mode_vertex(nw, nm, gk, (cplx *)Uk + (long)ik * nw * nw, Ukq, E, gmn, tmp, m->polar ? Cp : NULL);
        for (int n = 0; n < nw; n++) {
          double en = epsk[(long)ik * nw + n];
          for (int nu = 0; nu < nm; nu++) {
            if (w[nu] < pr->omega_min) continue;
            double nb = oracle_bose(w[nu], pr->T);
            for (int mm = 0; mm < nw; mm++) {
              double f = oracle_fermi(ekq[mm], pr->EF, pr->T);
              cplx gv = gmn[(nu * nw + mm) * nw + n];
              double g2 = creal(gv) * creal(gv) + cimag(gv) * cimag(gv);
              double term = (nb + f) * oracle_gauss(en - ekq[mm] + w[nu], pr->sigma) +
                            (nb + 1.0 - f) * oracle_gauss(en - ekq[mm] - w[nu], pr->sigma);
              nsum_add(&my[(long)ik * nw + n], M_PI * wqi * g2 * term);
            }
          }
        }
      }
    }
    free(gReq); free(gk); free(tmp); free(gmn); free(Hkq); free(Ukq); free(D); free(ev); free(E);
  }
  for (long i = 0; i < (long)nk * nw; i++) {
    nsum s = {0.0, 0.0};
    for (int t = 0; t < nthr; t++) {
      nsum_add(&s, acc[(long)t * nk * nw + i].s);
      nsum_add(&s, acc[(long)t * nk * nw + i].c);
    }
    imsig[i] = nsum_get(&s);
  }
  free(acc); free(epsk); free(Uk);
  return bad ? -1 : 0;
}

/* ------------------------------------------------- phonon self-energy */

/* Per (q, nu), sums over k of the same interpolated vertex (Sec. "Theory"):
 *   pi_im[q][nu] = Pi''_qnu(w_qnu) of Eq. (linewidthph), on shell, as printed:
 *                  2 pi sum_k w_k sum_mn |g_mn,nu(k,q)|^2 (f_nk - f_mk+q) delta(e_nk - e_mk+q - w_qnu)
 *   lam[q][nu]   = lambda_qnu of Eq. (lambdaEQ):
 *                  sum_k w_k sum_mn |g|^2 delta(e_nk - E_F) delta(e_mk+q - E_F) / (N(E_F) w_qnu)
 *   zeta[q]      = nesting function of Eq. (nestingfct): sum_k w_k sum_nm delta(e_nk - E_F) delta(e_mk+q - E_F)
 *   dos[0]       = N(E_F) = sum_k w_k sum_n delta(e_nk - E_F)   (per spin)
 * Modes below omega_min get 0 in pi_im and lam.  wk == NULL means 1/nk.
 * Any of pi_im, lam, zeta, dos may be NULL. */
int oracle_phonon_self(const oracle_model *m, int nk, const double *k, const double *wk, int nq, const double *q,
                       const oracle_params *pr, double *pi_im, double *lam, double *zeta, double *dos) {
  int nw = m->nw, nm = 3 * m->nat, nc = nm * nw * nw;
  double *epsk = malloc(sizeof(double) * (long)nk * nw);
  double *Uk = malloc(sizeof(cplx) * (long)nk * nw * nw);
  int bad = oracle_bands(m, nk, k, epsk, Uk);
  nsum nd = {0.0, 0.0};
  for (int ik = 0; ik < nk; ik++)
    for (int n = 0; n < nw; n++)
      nsum_add(&nd, (wk ? wk[ik] : 1.0 / nk) * oracle_gauss(epsk[(long)ik * nw + n] - pr->EF, pr->sigma));
  const double nef = nsum_get(&nd);
  if (dos) dos[0] = nef;
#pragma omp parallel reduction(+ : bad)
  {
    cplx *gReq = malloc(sizeof(cplx) * (long)m->nRe * nc);
    cplx *gk = malloc(sizeof(cplx) * nc), *tmp = malloc(sizeof(cplx) * nc), *gmn = malloc(sizeof(cplx) * nc);
    cplx *Hkq = malloc(sizeof(cplx) * nw * nw), *Ukq = malloc(sizeof(cplx) * nw * nw);
    cplx *D = malloc(sizeof(cplx) * nm * nm), *ev = malloc(sizeof(cplx) * nm * nm), *E = malloc(sizeof(cplx) * nm * nm);
    double w2[64], w[64], ekq[64];
    nsum sp[64], sl[64], sz;
#pragma omp for schedule(dynamic)
    for (int iq = 0; iq < nq; iq++) {
      const double *qq = q + 3 * iq;
      oracle_dynmat(m, qq, D);
      if (oracle_eigh(nm, D, w2, ev) < 0) bad++;
      for (int j = 0; j < nm; j++) w[j] = (w2[j] >= 0 ? 1.0 : -1.0) * sqrt(fabs(w2[j]));
      mode_factors(m, w, ev, pr->omega_min, E);
      cplx Cp[64];
      polar_factors(m, qq, E, Cp);
      oracle_g_Re_q(m, qq, gReq);
      for (int nu = 0; nu < nm; nu++) sp[nu] = sl[nu] = (nsum){0.0, 0.0};
      sz = (nsum){0.0, 0.0};
      for (int ik = 0; ik < nk; ik++) {
        const double wki = wk ? wk[ik] : 1.0 / nk;
        double kq[3] = {k[3 * ik] + qq[0], k[3 * ik + 1] + qq[1], k[3 * ik + 2] + qq[2]};
        oracle_hk(m, kq, Hkq);
        if (oracle_eigh(nw, Hkq, ekq, Ukq) < 0) bad++;
        g_k_from_Re_q(m, gReq, k + 3 * ik, gk);
        bloch_mode_vertex(nw, nm, gk, (cplx *)Uk + (long)ik * nw * nw, Ukq, E, gmn, tmp, m->polar ? Cp : NULL);
        for (int n = 0; n < nw; n++) {
          const double en = epsk[(long)ik * nw + n];
          const double dn = oracle_gauss(en - pr->EF, pr->sigma);
          for (int mm = 0; mm < nw; mm++) {
            const double dfnm = oracle_fermi_diff(en, ekq[mm], pr->EF, pr->T);  /* f_nk - f_mk+q */
            const double dd = dn * oracle_gauss(ekq[mm] - pr->EF, pr->sigma);
            nsum_add(&sz, wki * dd);
            for (int nu = 0; nu < nm; nu++) {
              if (w[nu] < pr->omega_min) continue;
              cplx gv = gmn[(nu * nw + mm) * nw + n];
              double g2 = creal(gv) * creal(gv) + cimag(gv) * cimag(gv);
              nsum_add(&sp[nu], wki * g2 * dfnm * oracle_gauss(en - ekq[mm] - w[nu], pr->sigma));
              nsum_add(&sl[nu], wki * g2 * dd);
            }
          }
        }
      }
      for (int nu = 0; nu < nm; nu++) {
        const int keep = w[nu] >= pr->omega_min;
        if (pi_im) pi_im[(long)iq * nm + nu] = keep ? 2.0 * M_PI * nsum_get(&sp[nu]) : 0.0;
        if (lam) lam[(long)iq * nm + nu] = (keep && nef > 0.0) ? nsum_get(&sl[nu]) / (nef * w[nu]) : 0.0;
      }
      if (zeta) zeta[iq] = nsum_get(&sz);
    }
    free(gReq); free(gk); free(tmp); free(gmn); free(Hkq); free(Ukq); free(D); free(ev); free(E);
  }
  free(epsk); free(Uk);
  return bad ? -1 : 0;
}

/* Complex electron self-energy of Eq. (elselfenergy) on a frequency grid (omega measured from E_F),
 * with the broadening i delta:
 *   sig[k][n][i] = sum_q w_q sum_{m,nu} |g_mn,nu(k,q)|^2 [ (n_qnu + f_mk+q) / (w_i - x_m + w_qnu + i delta)
 *                                                     + (n_qnu + 1 - f_mk+q) / (w_i - x_m - w_qnu + i delta) ],
 *   x_m = e_mk+q - E_F; sig [nk][nw][nomega] complex (re, im interleaved).  With spec != NULL also the
 * spectral function of Eq. (spectral_funct), with Sigma'' = -Im Sigma and the real part shifted by
 * Sigma'(omega = 0) (Eq. realpartselfenergy):
 *   spec[k][n][i] = (1/pi) |Sigma''| / ((w_i - (e_nk - E_F) - Sigma~'(w_i))^2 + Sigma''^2). */
int oracle_selfenergy(const oracle_model *m, int nk, const double *k, int nq, const double *q, const double *wq,
                      const oracle_params *pr, double delta, int nom, const double *omega, double *sig,
                      double *spec) {
  int nw = m->nw, nm = 3 * m->nat, nc = nm * nw * nw;
  const int nw1 = nom + 1;  /* the grid and omega = 0 */
  double *epsk = malloc(sizeof(double) * (long)nk * nw);
  double *Uk = malloc(sizeof(cplx) * (long)nk * nw * nw);
  int bad = oracle_bands(m, nk, k, epsk, Uk);
  cplx *acc = calloc((size_t)nk * nw * nw1, sizeof(cplx));
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
  for (int ik = 0; ik < nk; ik++) {
    cplx *gReq = malloc(sizeof(cplx) * (long)m->nRe * nc);
    cplx *gk = malloc(sizeof(cplx) * nc), *tmp = malloc(sizeof(cplx) * nc), *gmn = malloc(sizeof(cplx) * nc);
    cplx *Hkq = malloc(sizeof(cplx) * nw * nw), *Ukq = malloc(sizeof(cplx) * nw * nw);
    cplx *D = malloc(sizeof(cplx) * nm * nm), *ev = malloc(sizeof(cplx) * nm * nm), *E = malloc(sizeof(cplx) * nm * nm);
    double w2[64], w[64], ekq[64];
    cplx *my = acc + (long)ik * nw * nw1;
    for (int iq = 0; iq < nq; iq++) {
      const double *qq = q + 3 * iq;
      const double wqi = wq ? wq[iq] : 1.0 / nq;
      oracle_dynmat(m, qq, D);
      if (oracle_eigh(nm, D, w2, ev) < 0) bad++;
      for (int j = 0; j < nm; j++) w[j] = (w2[j] >= 0 ? 1.0 : -1.0) * sqrt(fabs(w2[j]));
      mode_factors(m, w, ev, pr->omega_min, E);
      cplx Cp[64];
      polar_factors(m, qq, E, Cp);
      oracle_g_Re_q(m, qq, gReq);
      double kq[3] = {k[3 * ik] + qq[0], k[3 * ik + 1] + qq[1], k[3 * ik + 2] + qq[2]};
      oracle_hk(m, kq, Hkq);
      if (oracle_eigh(nw, Hkq, ekq, Ukq) < 0) bad++;
      g_k_from_Re_q(m, gReq, k + 3 * ik, gk);
      bloch_mode_vertex(nw, nm, gk, (cplx *)Uk + (long)ik * nw * nw, Ukq, E, gmn, tmp, m->polar ? Cp : NULL);
      for (int nu = 0; nu < nm; nu++) {
        if (w[nu] < pr->omega_min) continue;
        const double nb = oracle_bose(w[nu], pr->T);
        for (int mm = 0; mm < nw; mm++) {
          const double f = oracle_fermi(ekq[mm], pr->EF, pr->T);
          const double x = ekq[mm] - pr->EF;
          for (int n = 0; n < nw; n++) {
            cplx gv = gmn[(nu * nw + mm) * nw + n];
            const double g2 = wqi * (creal(gv) * creal(gv) + cimag(gv) * cimag(gv));
            for (int i = 0; i < nw1; i++) {
              const double om = i < nom ? omega[i] : 0.0;
              my[(long)n * nw1 + i] += g2 * ((nb + f) / (om - x + w[nu] + I * delta) +
                                             (nb + 1.0 - f) / (om - x - w[nu] + I * delta));
            }
          }
        }
      }
    }
    free(gReq); free(gk); free(tmp); free(gmn); free(Hkq); free(Ukq); free(D); free(ev); free(E);
  }
  for (int ik = 0; ik < nk; ik++)
    for (int n = 0; n < nw; n++) {
      const cplx *a = acc + ((long)ik * nw + n) * nw1;
      const double re0 = creal(a[nom]);
      for (int i = 0; i < nom; i++) {
        const long o = ((long)ik * nw + n) * nom + i;
        sig[2 * o] = creal(a[i]);
        sig[2 * o + 1] = cimag(a[i]);
        if (spec) {
          const double s2 = -cimag(a[i]);
          const double den = omega[i] - (epsk[(long)ik * nw + n] - pr->EF) - (creal(a[i]) - re0);
          spec[o] = fabs(s2) / (M_PI * (den * den + s2 * s2));
        }
      }
    }
  free(acc); free(epsk); free(Uk);
  return bad ? -1 : 0;
}

/* Isotropic Eliashberg function of Eq. (isotropiceliash) on an omega grid:
 *   a2f[i] = 1/2 sum_q w_q sum_nu w_qnu lambda_qnu delta_ph(omega_i - w_qnu),
 * delta_ph the Gaussian of width sigma_ph; omega [nq][nm], lambda [nq][nm] (eV, 1);
 * wq == NULL means 1/nq. */
void oracle_eliashberg(int nq, int nm, const double *omega, const double *lambda, const double *wq, int nw,
                       const double *grid, double sigma_ph, double *a2f) {
  for (int i = 0; i < nw; i++) {
    nsum s = {0.0, 0.0};
    for (int iq = 0; iq < nq; iq++)
      for (int nu = 0; nu < nm; nu++) {
        const double w = omega[(long)iq * nm + nu];
        nsum_add(&s, 0.5 * (wq ? wq[iq] : 1.0 / nq) * w * lambda[(long)iq * nm + nu] *
                         oracle_gauss(grid[i] - w, sigma_ph));
      }
    a2f[i] = nsum_get(&s);
  }
}

/* ------------------------------------------------------------- adjoint */

/* L = sum_{k,n} cot[k][n] Im Sigma_nk.  dg [nRe][nRp][3nat][nw][nw] complex gets
 * dL/dRe g + i dL/dIm g; dT = dL/dT, dEF = dL/dE_F.  T must be > 0. */
int oracle_linewidth_grad(const oracle_model *m, int nk, const double *k, int nq, const double *q,
                          const double *wq, const oracle_params *pr, const double *cot,
                          double *dg, double *dT, double *dEF) {
  int nw = m->nw, nm = 3 * m->nat, nc = nm * nw * nw;
  long ng = (long)m->nRe * m->nRp * nc;
  double *epsk = malloc(sizeof(double) * (long)nk * nw);
  double *Uk = malloc(sizeof(cplx) * (long)nk * nw * nw);
  int bad = oracle_bands(m, nk, k, epsk, Uk);
  double kT = KB_EV * pr->T;
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  cplx *dgt = calloc((size_t)nthr * ng, sizeof(cplx));
  nsum *sT = calloc(nthr, sizeof(nsum)), *sE = calloc(nthr, sizeof(nsum));
#pragma omp parallel reduction(+ : bad)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    cplx *mydg = dgt + (long)tid * ng;
    cplx *gReq = malloc(sizeof(cplx) * (long)m->nRe * nc), *barReq = malloc(sizeof(cplx) * (long)m->nRe * nc);
    cplx *gk = malloc(sizeof(cplx) * nc), *tmp = malloc(sizeof(cplx) * nc), *gmn = malloc(sizeof(cplx) * nc);
    cplx *Wg = malloc(sizeof(cplx) * nc), *bar = malloc(sizeof(cplx) * nc);
    cplx *Hkq = malloc(sizeof(cplx) * nw * nw), *Ukq = malloc(sizeof(cplx) * nw * nw);
    cplx *D = malloc(sizeof(cplx) * nm * nm), *ev = malloc(sizeof(cplx) * nm * nm), *E = malloc(sizeof(cplx) * nm * nm);
    double w2[64], w[64], ekq[64];
#pragma omp for schedule(dynamic)
    for (int iq = 0; iq < nq; iq++) {
      const double *qq = q + 3 * iq;
      double wqi = wq ? wq[iq] : 1.0 / nq;
      oracle_dynmat(m, qq, D);
      if (oracle_eigh(nm, D, w2, ev) < 0) bad++;
      for (int j = 0; j < nm; j++) w[j] = (w2[j] >= 0 ? 1.0 : -1.0) * sqrt(fabs(w2[j]));
      mode_factors(m, w, ev, pr->omega_min, E);
      cplx Cp[64];
      polar_factors(m, qq, E, Cp);
      oracle_g_Re_q(m, qq, gReq);
      for (long i = 0; i < (long)m->nRe * nc; i++) barReq[i] = 0.0;
      for (int ik = 0; ik < nk; ik++) {
        const cplx *U = (cplx *)Uk + (long)ik * nw * nw;
        double kq[3] = {k[3 * ik] + qq[0], k[3 * ik + 1] + qq[1], k[3 * ik + 2] + qq[2]};
        oracle_hk(m, kq, Hkq);
        if (oracle_eigh(nw, Hkq, ekq, Ukq) < 0) bad++;
        g_k_from_Re_q(m, gReq, k + 3 * ik, gk);
        bloch_mode_vertex(nw, nm, gk, U, Ukq, E, gmn, tmp, m->polar ? Cp : NULL);
        /* W_{nu,mn} g_{nu,mn}, and the temperature / Fermi-level partials */
        for (int nu = 0; nu < nm; nu++)
          for (int mm = 0; mm < nw; mm++)
            for (int n = 0; n < nw; n++) {
              long id = (nu * nw + mm) * nw + n;
              Wg[id] = 0.0;
              if (w[nu] < pr->omega_min) continue;
              double c = cot[(long)ik * nw + n];
              double en = epsk[(long)ik * nw + n];
              double nb = oracle_bose(w[nu], pr->T);
              double f = oracle_fermi(ekq[mm], pr->EF, pr->T);
              double dp = oracle_gauss(en - ekq[mm] + w[nu], pr->sigma);
              double dm = oracle_gauss(en - ekq[mm] - w[nu], pr->sigma);
              double W = c * M_PI * wqi * ((nb + f) * dp + (nb + 1.0 - f) * dm);
              Wg[id] = W * gmn[id];
              double g2 = creal(gmn[id]) * creal(gmn[id]) + cimag(gmn[id]) * cimag(gmn[id]);
              double dn_dT = nb * (nb + 1.0) * w[nu] / (kT * pr->T);
              double ff = oracle_fermi_slope(ekq[mm], pr->EF, pr->T);
              double df_dT = ff * (ekq[mm] - pr->EF) / (kT * pr->T);
              double df_dE = ff / kT;
              /* d Im Sigma / dT = sum (dn/dT (d+ + d-) + df/dT (d+ - d-)) |g|^2, d / dE_F with
                 df/dE_F (d+ - d-); d+ - d- in the form without cancellation */
              double dd = oracle_gauss_diff(en - ekq[mm], w[nu], pr->sigma);
              nsum_add(&sT[tid], c * M_PI * wqi * g2 * (dn_dT * (dp + dm) + df_dT * dd));
              nsum_add(&sE[tid], c * M_PI * wqi * g2 * df_dE * dd);
            }
        /* bar_ka[j][i] = 2 sum_nu conj(E[ka][nu]) [Ukq (W g)_nu Uk^dag]_ji */
        for (int ka = 0; ka < nm; ka++)
          for (int j = 0; j < nw; j++)
            for (int i = 0; i < nw; i++) {
              cplx s = 0.0;
              for (int nu = 0; nu < nm; nu++) {
                cplx r = 0.0;
                for (int mm = 0; mm < nw; mm++)
                  for (int n = 0; n < nw; n++)
                    r += Ukq[j * nw + mm] * Wg[(nu * nw + mm) * nw + n] * conj(U[i * nw + n]);
                s += conj(E[ka * nm + nu]) * r;
              }
              bar[(ka * nw + j) * nw + i] = 2.0 * s;
            }
        /* adjoint of the k step: barReq(Re) += wRe conj(e^{2pi i k.Re}) bar */
        for (int a = 0; a < m->nRe; a++) {
          cplx p = conj(phase(k + 3 * ik, m->Re + 3 * a)) * (m->wRe ? m->wRe[a] : 1.0);
          for (int i = 0; i < nc; i++) barReq[(long)a * nc + i] += p * bar[i];
        }
      }
      /* adjoint of the q step: dg(Re,Rp) += wRp conj(e^{2pi i q.Rp}) barReq(Re) */
      for (int b = 0; b < m->nRp; b++) {
        cplx p = conj(phase(qq, m->Rp + 3 * b)) * (m->wRp ? m->wRp[b] : 1.0);
        for (int a = 0; a < m->nRe; a++)
          for (int i = 0; i < nc; i++)
            mydg[((long)a * m->nRp + b) * nc + i] += p * barReq[(long)a * nc + i];
      }
    }
    free(gReq); free(barReq); free(gk); free(tmp); free(gmn); free(Wg); free(bar);
    free(Hkq); free(Ukq); free(D); free(ev); free(E);
  }
  cplx *o = (cplx *)dg;
  for (long i = 0; i < ng; i++) {
    cplx s = 0.0;
    for (int t = 0; t < nthr; t++) s += dgt[(long)t * ng + i];
    o[i] = s;
  }
  nsum aT = {0, 0}, aE = {0, 0};
  for (int t = 0; t < nthr; t++) {
    nsum_add(&aT, sT[t].s); nsum_add(&aT, sT[t].c);
    nsum_add(&aE, sE[t].s); nsum_add(&aE, sE[t].c);
  }
  *dT = nsum_get(&aT);
  *dEF = nsum_get(&aE);
  free(dgt); free(sT); free(sE); free(epsk); free(Uk);
  return bad ? -1 : 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
