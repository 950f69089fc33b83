// Internal declarations of the sm_103a linewidth library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "epw.h"

#define EPW_KB 8.617333262e-5
#define EPW_PI 3.14159265358979323846

// Device status bits (model->dstatus[0]).
#define EPW_DEV_NOT_CONVERGED 1u
#define EPW_DEV_BAD_SHAPE 2u
#define EPW_DEV_TIMEOUT 4u

// ------------------------------------------------------------------ complex
template <typename R>
struct cx {
  R x, y;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mkc(R a, R b) {
  cx<R> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mkc(s * a.x, s * a.y); }
template <typename R>
__host__ __device__ __forceinline__ cx<R> conjc(cx<R> a) { return mkc(a.x, -a.y); }
// conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b) {
  return mkc(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void cfma(cx<R> &acc, cx<R> a, cx<R> b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
template <typename R>
__host__ __device__ __forceinline__ R cabs2(cx<R> a) { return a.x * a.x + a.y * a.y; }

template <typename R, typename S>
__host__ __device__ __forceinline__ cx<R> ccast(cx<S> a) { return mkc((R)a.x, (R)a.y); }

// ------------------------------------------------------------ occupations
// Bose-Einstein n(w) = 1/(e^{w/kT} - 1); T <= 0 gives 0.
__device__ __forceinline__ double bose_d(double w, double T) {
  if (T <= 0.0) return 0.0;
  double x = w / (EPW_KB * T);
  return x > 700.0 ? 0.0 : 1.0 / expm1(x);
}
__device__ __forceinline__ float bose_f(float w, float invkT) {
  if (invkT <= 0.0f) return 0.0f;
  float x = w * invkT;
  return x > 80.0f ? 0.0f : 1.0f / expm1f(x);
}
// Fermi-Dirac f(e) = 1/(e^{(e-EF)/kT} + 1); T <= 0 gives a step with f(EF) = 1/2.
__device__ __forceinline__ double fermi_d(double e, double EF, double T) {
  double d = e - EF;
  if (T <= 0.0) return d < 0.0 ? 1.0 : (d > 0.0 ? 0.0 : 0.5);
  double x = d / (EPW_KB * T);
  if (x > 0.0) {
    double t = exp(-x);
    return t / (1.0 + t);
  }
  return 1.0 / (1.0 + exp(x));
}
__device__ __forceinline__ float fermi_f(float d, float invkT) {
  if (invkT <= 0.0f) return d < 0.0f ? 1.0f : (d > 0.0f ? 0.0f : 0.5f);
  float x = d * invkT;
  float t = __expf(-fabsf(x));
  return x > 0.0f ? t / (1.0f + t) : 1.0f / (1.0f + t);
}

// f (1 - f) = t / (1 + t)^2 with t = e^{-|e - EF|/kT}: no cancellation in the tails
// (forming 1 - f from a rounded f loses everything once f rounds to 1).
__device__ __forceinline__ float fermi_ff_f(float d, float invkT) {
  if (invkT <= 0.0f) return 0.0f;
  const float t = __expf(-fabsf(d * invkT));
  const float u = 1.0f + t;
  return t / (u * u);
}
__device__ __forceinline__ double fermi_ff_d(double d, double T) {
  if (T <= 0.0) return 0.0;
  const double t = exp(-fabs(d / (EPW_KB * T)));
  const double u = 1.0 + t;
  return t / (u * u);
}

// f(ea) - f(eb) without subtracting two rounded occupations: with a, b the
// arguments (e - E_F)/kT, d = b - a and S = |a| + |b|,
//   f(a) - f(b) = 2 sinh(d/2) e^{-S/2} / ((1 + e^{-|a|}) (1 + e^{-|b|})),
// the sinh through expm1 of d or -d so that no exponent is positive.
__device__ __forceinline__ double fermi_diff_d(double ea, double eb, double EF, double T) {
  if (T <= 0.0) return fermi_d(ea, EF, T) - fermi_d(eb, EF, T);
  const double ikt = 1.0 / (EPW_KB * T);
  const double a = (ea - EF) * ikt, b = (eb - EF) * ikt;
  const double d = b - a, S = fabs(a) + fabs(b);
  const double num = d >= 0.0 ? -exp(0.5 * (d - S)) * expm1(-d) : exp(-0.5 * (d + S)) * expm1(d);
  return num / ((1.0 + exp(-fabs(a))) * (1.0 + exp(-fabs(b))));
}
__device__ __forceinline__ float fermi_diff_f(float ea, float eb, double EF, double T) {
  if (T <= 0.0) {
    const float fa = ea < (float)EF ? 1.0f : (ea > (float)EF ? 0.0f : 0.5f);
    const float fb = eb < (float)EF ? 1.0f : (eb > (float)EF ? 0.0f : 0.5f);
    return fa - fb;
  }
  const float ikt = (float)(1.0 / (EPW_KB * T));
  const float a = (float)((double)ea - EF) * ikt, b = (float)((double)eb - EF) * ikt;
  const float d = b - a, S = fabsf(a) + fabsf(b);
  const float num = d >= 0.0f ? -expf(0.5f * (d - S)) * expm1f(-d) : expf(-0.5f * (d + S)) * expm1f(d);
  return num / ((1.0f + expf(-fabsf(a))) * (1.0f + expf(-fabsf(b))));
}

// -------------------------------------------------------- Jacobi eigensolver
// Hermitian N x N (runtime n <= N, compile-time N so that fully unrolled loops
// keep the arrays in registers for small N).  Cyclic sweeps of two-sided
// complex Jacobi rotations: each rotation is a 2x2 unitary
//   G = [[c, s e], [-s conj(e), c]]  (e = a_pq/|a_pq|)
// that zeroes a_pq (a real Jacobi rotation conjugated by the phase of a_pq).
// Stops when the off-diagonal weight falls below tol2 * total weight; sets
// *nonconv when maxsweep sweeps were not enough.  On return the diagonal of A
// holds the eigenvalues (unsorted) and V the eigenvectors (columns).
template <typename R, int N>
__device__ __forceinline__ void jacobi_herm(cx<R> (&A)[N][N], cx<R> (&V)[N][N], int n, R tol2, int maxsweep,
                                            bool &nonconv) {
  constexpr int UR = N <= 4 ? N : 1;
#pragma unroll UR
  for (int i = 0; i < N; i++)
#pragma unroll UR
    for (int j = 0; j < N; j++) V[i][j] = mkc<R>(i == j ? R(1) : R(0), R(0));
  // Hermitian part (only A[i][j], i<j, and the real diagonal are used below)
#pragma unroll UR
  for (int i = 0; i < N; i++) {
    A[i][i].y = R(0);
#pragma unroll UR
    for (int j = i + 1; j < N; j++) {
      cx<R> a = R(0.5) * (A[i][j] + conjc(A[j][i]));
      A[i][j] = a;
      A[j][i] = conjc(a);
    }
  }
  bool done = false;
  for (int sweep = 0; sweep < maxsweep && !done; sweep++) {
    R off = R(0), diag = R(0);
#pragma unroll UR
    for (int i = 0; i < N; i++) {
      if (i < n) diag += A[i][i].x * A[i][i].x;
#pragma unroll UR
      for (int j = i + 1; j < N; j++)
        if (j < n) off += cabs2(A[i][j]);
    }
    if (off <= tol2 * (diag + R(2) * off)) {
      done = true;
      break;
    }
#pragma unroll UR
    for (int p = 0; p < N - 1; p++) {
#pragma unroll UR
      for (int q = p + 1; q < N; q++) {
        if (q >= n) continue;
        cx<R> apq = A[p][q];
        R m2 = cabs2(apq);
        if (m2 == R(0)) continue;
        R mag = sqrt(m2);
        R rinv = R(1) / mag;
        cx<R> e = mkc(apq.x * rinv, apq.y * rinv);
        R theta = (A[q][q].x - A[p][p].x) * (R(0.5) * rinv);
        R t = R(1) / (fabs(theta) + sqrt(fma(theta, theta, R(1))));
        t = theta < R(0) ? -t : t;
        R c = R(1) / sqrt(fma(t, t, R(1)));
        R s = t * c;
        A[p][p].x -= t * mag;
        A[q][q].x += t * mag;
        A[p][q] = mkc(R(0), R(0));
        A[q][p] = mkc(R(0), R(0));
        cx<R> se = s * e;          // s e
        cx<R> sec = s * conjc(e);  // s conj(e)
#pragma unroll UR
        for (int r = 0; r < N; r++) {
          if (r == p || r == q || r >= n) continue;
          cx<R> arp = A[r][p], arq = A[r][q];
          cx<R> nrp = c * arp - sec * arq;
          cx<R> nrq = se * arp + c * arq;
          A[r][p] = nrp;
          A[p][r] = conjc(nrp);
          A[r][q] = nrq;
          A[q][r] = conjc(nrq);
        }
#pragma unroll UR
        for (int r = 0; r < N; r++) {
          if (r >= n) continue;
          cx<R> vrp = V[r][p], vrq = V[r][q];
          V[r][p] = c * vrp - sec * vrq;
          V[r][q] = se * vrp + c * vrq;
        }
      }
    }
  }
  if (!done) {
    // one last convergence check after the final sweep
    R off = R(0), diag = R(0);
#pragma unroll UR
    for (int i = 0; i < N; i++) {
      if (i < n) diag += A[i][i].x * A[i][i].x;
#pragma unroll UR
      for (int j = i + 1; j < N; j++)
        if (j < n) off += cabs2(A[i][j]);
    }
    if (!(off <= tol2 * (diag + R(2) * off))) nonconv = true;
  }
}

// Sort eigenvalues (diagonal of A) ascending into w[], permuting columns of V.
template <typename R, int N>
__device__ __forceinline__ void sort_eig(cx<R> (&A)[N][N], cx<R> (&V)[N][N], R (&w)[N], int n) {
  constexpr int UR = N <= 4 ? N : 1;
#pragma unroll UR
  for (int i = 0; i < N; i++) w[i] = A[i][i].x;
  // insertion network over the first n entries (compile-time loops)
#pragma unroll UR
  for (int i = 1; i < N; i++) {
#pragma unroll UR
    for (int j = i; j > 0; j--) {
      if (j < n && w[j] < w[j - 1]) {
        R t = w[j];
        w[j] = w[j - 1];
        w[j - 1] = t;
#pragma unroll UR
        for (int r = 0; r < N; r++) {
          cx<R> tv = V[r][j];
          V[r][j] = V[r][j - 1];
          V[r][j - 1] = tv;
        }
      }
    }
  }
}

// Gaussian delta, exp(-(x/sigma)^2) / (sigma sqrt(pi)) with norm = 1/(sigma sqrt(pi)).
template <typename R>
__device__ __forceinline__ R gauss_r(R x, R inv_sigma, R norm) {
  R y = x * inv_sigma;
  return norm * exp(-y * y);
}

// delta(x + w) - delta(x - w) for the Gaussian above.  With a = x/sigma, b = w/sigma the
// two exponents differ by 4ab, so the difference is -2 norm exp(-(a^2 + b^2)) sinh(2ab),
// which keeps its relative accuracy for w << sigma (no subtraction of close values); for
// |2ab| > 1 the plain difference is well conditioned and is taken instead.
template <typename R>
__device__ __forceinline__ R gauss_diff_r(R x, R w, R inv_sigma, R norm) {
  const R a = x * inv_sigma, b = w * inv_sigma, y = R(2) * a * b;
  if (fabs(y) > R(1)) return gauss_r<R>(x + w, inv_sigma, norm) - gauss_r<R>(x - w, inv_sigma, norm);
  return R(-2) * norm * exp(-(a * a + b * b)) * sinh(y);
}

// Occupations in working precision (FP64 forms in FP64, FP32 forms with 1/kT).
template <typename R>
__device__ __forceinline__ R occ_bose(R w, double T);
template <>
__device__ __forceinline__ double occ_bose<double>(double w, double T) { return bose_d(w, T); }
template <>
__device__ __forceinline__ float occ_bose<float>(float w, double T) {
  return bose_f(w, T > 0.0 ? (float)(1.0 / (EPW_KB * T)) : 0.0f);
}
template <typename R>
__device__ __forceinline__ R occ_fermi(R e, double EF, double T);
template <>
__device__ __forceinline__ double occ_fermi<double>(double e, double EF, double T) { return fermi_d(e, EF, T); }
template <>
__device__ __forceinline__ float occ_fermi<float>(float e, double EF, double T) {
  return fermi_f((float)((double)e - EF), T > 0.0 ? (float)(1.0 / (EPW_KB * T)) : 0.0f);
}

template <typename R>
struct jacobi_tol;
template <>
struct jacobi_tol<double> {
  static constexpr double tol2 = 1e-30;
  static constexpr int maxsweep = 40;
};
template <>
struct jacobi_tol<float> {
  static constexpr float tol2 = 1e-12f;
  static constexpr int maxsweep = 20;
};

// ------------------------------------------------------------------ model
struct epw_model {
  int device;
  int nw, nat, nm;
  int nRe, nRp, nRph;
  int same_ep, same_eph;  // R sets identical (Re==Rp, Re==Rph)
  int rmax;               // largest |R component| over the three sets
  int *Re, *Rp, *Rph;     // [n][3]
  double *wRe, *wRp;      // [n]
  cx<double> *Hw;         // [nRe][nw][nw], wRe folded
  cx<double> *Phiw;       // [nRph][nm][nm], wRph and 1/sqrt(M M') folded
  float4 *Phidf;          // Phiw in double-float: (Re hi, Re lo, Im hi, Im lo) per entry
  cx<double> *gw;         // [nRe][nRp][nm][nw][nw], wRe wRp folded
  double *mass;           // [nat]
  unsigned int *dstatus;  // device status word
  void *ws;               // workspace arena
  size_t ws_bytes;
  // measurement hook around the dominant kernel
  int timing;
  int nev;
  cudaEvent_t *ev;        // [2 * EPW_MAX_TIMED]
  unsigned char *ev_tag;  // [EPW_MAX_TIMED] tag of each timed launch
  // second stream for the q side of the preparation, and its fork / join events
  cudaStream_t aux;
  cudaEvent_t ev_fork, ev_join, ev_phase;
  // third stream: the k-side bands (H(k) and its eigensolve) beside the k-side vertex GEMM
  cudaStream_t aux2;
  cudaEvent_t ev_fork2, ev_join2;
  // long-range (polar) part of the vertex (epw_set_polar); polar == 0: none
  int polar;
  double pb[9];           // reciprocal vectors b_i (rows), 2 pi (A^{-1})^T
  double peps[9];         // eps_inf
  double *pZ;             // device [nat][3][3]
  double palpha, ppref;
  int pgmax;
};

#define EPW_MAX_TIMED 4096

// Record the start / stop event of a timed launch (no-op unless timing is on).
void epw_timing_begin(epw_model *m, cudaStream_t st);
void epw_timing_begin_tag(epw_model *m, cudaStream_t st, int tag);
void epw_timing_end(epw_model *m, cudaStream_t st);

// Bump allocator over the model's workspace arena.
struct Arena {
  char *base;
  size_t cap, off;
  template <typename T>
  T *take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T *p = (T *)(base ? base + off : nullptr);
    off += n * sizeof(T);
    return p;
  }
};

// Launch accounting (host side).
void epw_count_launch();

// ------------------------------------------------------------- kernels
// Generic SIMT path (epw_generic.cu)
// rmax: the largest |R component| of the set (one-axis factors when small)
void launch_phases(int npt, const double *x, int nR, const int *R, int rmax, cx<double> *out_rowmajor,
                   cx<double> *out_T, cx<float> *out_T32, cudaStream_t st);
void launch_fourier_d(int npt, int nR, const cx<double> *P, const cx<double> *X, int msize, cx<double> *out,
                      cudaStream_t st);
void launch_eigh_d(int nmat, int n, cx<double> *A, double *w, cx<double> *V, unsigned *dstatus, cudaStream_t st);
void launch_phonon_post(int nq, int nm, const double *w2, const cx<double> *ev, const double *mass, double omega_min,
                        double *omegaT, cx<double> *ET64, cx<float> *ET32, double *omega_out, cudaStream_t st);
template <typename R>
void launch_cgemm(int M, int N, int K, const cx<R> *A, int lda, bool transA, bool conjA, const cx<R> *B, int ldb,
                  cx<R> *C, int ldc, bool accumulate, cudaStream_t st);
template <typename R>
void launch_build_B(const epw_model *m, int nk, const cx<double> *Pk, const cx<R> *G1, const cx<double> *Uk,
                    cx<R> *Bg, cx<R> *BH, cudaStream_t st);
void launch_cast_c64_to_c32(size_t n, const cx<double> *in, cx<float> *out, cudaStream_t st);

struct PairArgs {
  int nk, nq, nw, nm, nRe, nRp;
  int k0;                   // first k of this launch (global index)
  const void *PqTe, *PqTp;  // [nR][nq] phases (R precision)
  const void *BH, *Bg;      // [nk][nRe][nw][nw], [nk][nRp][nm][nw][nw] (R precision)
  const void *ET;           // [nm*nm][nq] mode factors (R precision)
  const double *omegaT;     // [nm][nq]
  const double *eps_k;      // [nk][nw]
  const double *wq;         // [nq] or null (1/nq)
  double T, EF, sigma, omega_min;
  // outputs
  double *partial;     // linewidth: [nk][nqb][nw]
  double *eps_kq;      // interp: [nk][nq][nw]
  cx<double> *gout;    // interp: [nk][nq][nm][nw][nw]
  const double *cot;   // backward: [nk][nw]
  void *xbar;          // backward: [nq][nkc][nm][nw][nw] (R precision)
  double *partialT;    // backward: [nkc][nqb]
  double *partialE;    // backward: [nkc][nqb]
  int nkc;             // backward: k in this chunk
  unsigned *dstatus;
  // staged tensor-core form: contraction read from Cq[(kl*cpk + 2c + s)*ldc + q]
  // (kl = k - k0; c over [H(k+q)_ij | (g_a(k,q) U_k)_jn], s = re/im) instead of computed
  const float *Cq;
  size_t ldc;
  int cpk;
  int nk_total;  // phonon side: all k-points of the call (the 1/nk weight when wq (= w_k) is null)
  // long-range vertex: g_nu += i C_nu(q) (U_k+q^dagger U_k), C [nm][nq] (R precision), U_k FP64 [nk][nw][nw]
  const void *Cpol;
  const cx<double> *Uk;
};
// mode: 0 linewidth, 1 interp, 2 backward
template <typename R>
epw_status launch_pair(const PairArgs &a, int mode, cudaStream_t st);
// per-pair kernel on a staged contraction (a.Cq set; FP32)
epw_status launch_pair_staged(const PairArgs &a, int mode, cudaStream_t st);
// phonon side (per-(q, nu) sums over k, nw <= 8, 3nat <= 9): grid (q blocks, nchunk), each chunk
// a.nkc k-points from a.k0 (a.nk of them in total in this launch); a.wq holds w_k here;
// partials [nchunk][nq][2 nm + 1]
template <typename R>
epw_status launch_pair_ph(const PairArgs &a, int nchunk, cudaStream_t st);
void launch_ph_finalize(int nq, int nm, int nchunk, const double *partial, const double *omegaT, double omega_min,
                        const double *dos, double *pi_im, double *lam, double *zeta, cudaStream_t st);
void launch_dos_terms(int nk, int nw, const double *epsk, const double *wk, double EF, double sigma, double *terms,
                      cudaStream_t st);
// Lattice / dielectric inputs of the long-range vertex, by value for the kernel.
struct PolarK {
  double b[9], eps[9];
  double alpha, pref;
  int gmax;
};
// C_nu(q) of the long-range vertex (Eq. (long-range)) into C [nm][nq] from the mode factors E [nm*nm][nq]
template <typename R>
void launch_polar_factors(const epw_model *m, int nq, const double *q, const cx<R> *ET, cx<R> *C, cudaStream_t st);
void launch_eliashberg(int nq, int nm, const double *omega, const double *lam, const double *wq, int ngrid,
                       const double *grid, double sigma_ph, double *a2f, cudaStream_t st);
// complex self-energy on a frequency grid (nw <= 8, 3nat <= 9): per-warp partials
// out[(kl * ceil(nq/32) + warp) * nw + n][nom + 1] (the last point is omega = 0), then the sum
template <typename R>
epw_status launch_pair_se(const PairArgs &a, int nom, const double *omega, double delta, double2 *out,
                          cudaStream_t st);
void launch_se_finalize(int nkc, int k0, int nw, int nqw, int nom, const double2 *part, const double *omega,
                        const double *epsk, double EF, double2 *sig, double *spec, cudaStream_t st);
// warp-per-pair kernel for nw, 3nat up to 18 (modes 0 and 1; a.Cq set: staged
// contraction in the q-major layout Cq[q*ldc + kl*cpk + 2c + s], FP32 only)
template <typename R>
epw_status launch_pair_wide(const PairArgs &a, int mode, cudaStream_t st);
// linewidth (mode 0) of the staged FP32 form for nw <= 18, 3nat <= 18: one warp per pair,
// Householder + implicit QR eigensolve, only the terms within the Gaussian cutoff
epw_status launch_pair_sparse(const PairArgs &a, cudaStream_t st);
void launch_finalize(int nk, int nqb, int nw, const double *partial, double *out, cudaStream_t st);
// m->gw = wRe wRp g (g on the device)
void launch_set_vertex(const epw_model *m, const void *g, int is_c64, cudaStream_t st);
void launch_sum_scalar(int n, const double *partial, double scale, double *out, cudaStream_t st);
// G1bar[k][Rp][a][j][i] = sum_n Bbar[Rp][k][a][j][n] conj(U_{k0+k}[i][n])
template <typename R>
void launch_bg_adjoint_rotate_k0(int nk, int k0, int nRp, int nm, int nw, const cx<R> *Bbar, const cx<double> *Uk,
                                 cx<R> *G1bar, cudaStream_t st);
template <typename R>
void launch_dg_scale(const epw_model *m, const cx<R> *gwbar, double *dg, bool accumulate, cudaStream_t st);
