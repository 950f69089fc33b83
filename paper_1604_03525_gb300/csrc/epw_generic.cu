// Generic SIMT kernels of the linewidth path (FP64 and FP32 forms) and the
// shared preparation steps (phases, k-side bands, phonons, k-side vertex).
//
// Method: EPW (Ponce et al. 2016), Eq. (linewidthel) for the reduction and the
// Wannier interpolation of Sec. "Electron-phonon coupling in polar materials"
// (step iii) with the U rotations of the overlap equation there.
#include <type_traits>
#include <cuda_runtime.h>

#include "epw_internal.cuh"
#include "epw_eig4.cuh"

namespace {

inline int nblocks(size_t n, int bs, int cap = 152 * 32) {
  size_t b = (n + bs - 1) / bs;
  if (b > (size_t)cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// -------------------------------------------------------------------- phases
// e^{2 pi i x.R}: the argument x.R is formed and reduced to [-1/2, 1/2] in
// FP64, then sincospi gives the value.  Index idx = r*npt + i so that the
// transposed outputs [nR][npt] are written coalesced.
__global__ void k_phases(int npt, const double *__restrict__ x, int nR, const int *__restrict__ R,
                         cx<double> *rowmajor, cx<double> *T64, cx<float> *T32) {
  size_t n = (size_t)npt * nR;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % npt);
    int r = (int)(idx / npt);
    double a = x[3 * i] * R[3 * r] + x[3 * i + 1] * R[3 * r + 1] + x[3 * i + 2] * R[3 * r + 2];
    a -= rint(a);
    double s, c;
    sincospi(2.0 * a, &s, &c);
    if (rowmajor) rowmajor[(size_t)i * nR + r] = mkc(c, s);
    if (T64) T64[idx] = mkc(c, s);
    if (T32) T32[idx] = mkc((float)c, (float)s);
  }
}

// The same phases from one-axis factors: e^{2 pi i x.R} = prod_j e^{2 pi i (x_j R_j mod 1)},
// the factors for R_j in [-rmax, rmax] (rmax <= PH_RMAX, the largest |R_j| of the set)
// formed once per point (FP64 argument reduction, sincospi), then two complex
// products per R.  One thread per point.
constexpr int PH_RMAX = 8;
__global__ void k_phases_fact(int npt, const double *__restrict__ x, int nR, const int *__restrict__ R, int rmax,
                              cx<double> *rowmajor, cx<double> *T64, cx<float> *T32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npt) return;
  cx<double> F[3][2 * PH_RMAX + 1];
  for (int j = 0; j < 3; j++) {
    const double xj = x[3 * i + j];
    for (int n = -rmax; n <= rmax; n++) {
      double a = xj * n;
      a -= rint(a);
      double s, c;
      sincospi(2.0 * a, &s, &c);
      F[j][n + PH_RMAX] = mkc(c, s);
    }
  }
  for (int r = 0; r < nR; r++) {
    const cx<double> f0 = F[0][R[3 * r] + PH_RMAX], f1 = F[1][R[3 * r + 1] + PH_RMAX], f2 = F[2][R[3 * r + 2] + PH_RMAX];
    const cx<double> f01 = mkc(f0.x * f1.x - f0.y * f1.y, f0.x * f1.y + f0.y * f1.x);
    const cx<double> p = mkc(f01.x * f2.x - f01.y * f2.y, f01.x * f2.y + f01.y * f2.x);
    if (rowmajor) rowmajor[(size_t)i * nR + r] = p;
    const size_t idx = (size_t)r * npt + i;
    if (T64) T64[idx] = p;
    if (T32) T32[idx] = mkc((float)p.x, (float)p.y);
  }
}

// out[i][e] = sum_r PT[r][i] X[r][e]   (PT transposed phases [nR][npt])
__global__ void k_fourier_d(int npt, int nR, const cx<double> *__restrict__ PT, const cx<double> *__restrict__ X,
                            int msize, cx<double> *out) {
  size_t n = (size_t)npt * msize;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % npt);
    int e = (int)(idx / npt);
    cx<double> acc = mkc(0.0, 0.0);
    for (int r = 0; r < nR; r++) cfma(acc, PT[(size_t)r * npt + i], X[(size_t)r * msize + e]);
    out[(size_t)i * msize + e] = acc;
  }
}

// Batched Hermitian eigensolve, one matrix per thread (FP64, converged to
// full precision).  w ascending; V columns are eigenvectors.
template <int N>
__global__ void k_eigh_d(int nmat, int n, const cx<double> *__restrict__ Ain, double *w, cx<double> *V,
                         unsigned *dstatus) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nmat) return;
  constexpr int UR = N <= 4 ? N : 1;
  cx<double> A[N][N], U[N][N];
  const cx<double> *a = Ain + (size_t)t * n * n;
#pragma unroll UR
  for (int i = 0; i < N; i++)
#pragma unroll UR
    for (int j = 0; j < N; j++) A[i][j] = (i < n && j < n) ? a[i * n + j] : mkc(0.0, 0.0);
  bool nc = false;
  jacobi_herm<double, N>(A, U, n, jacobi_tol<double>::tol2, jacobi_tol<double>::maxsweep, nc);
  double ww[N];
  sort_eig<double, N>(A, U, ww, n);
  if (nc) atomicOr(dstatus, EPW_DEV_NOT_CONVERGED);
#pragma unroll UR
  for (int i = 0; i < N; i++) {
    if (i < n) w[(size_t)t * n + i] = ww[i];
#pragma unroll UR
    for (int j = 0; j < N; j++)
      if (i < n && j < n) V[(size_t)t * n * n + i * n + j] = U[i][j];
  }
}

// omega = sign(w2) sqrt|w2|;  E[ka][nu] = e_{ka,nu} / sqrt(2 M_kappa omega_nu),
// zero when omega_nu < omega_min.  Outputs are transposed ([..][nq]).
__global__ void k_phonon_post(int nq, int nm, const double *__restrict__ w2, const cx<double> *__restrict__ ev,
                              const double *__restrict__ mass, double omega_min, double *omegaT, cx<double> *ET64,
                              cx<float> *ET32, double *omega_out) {
  size_t n = (size_t)nq * nm;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    int q = (int)(idx % nq);
    int nu = (int)(idx / nq);
    double x = w2[(size_t)q * nm + nu];
    double om = x >= 0.0 ? sqrt(x) : -sqrt(-x);
    if (omegaT) omegaT[(size_t)nu * nq + q] = om;
    if (omega_out) omega_out[(size_t)q * nm + nu] = om;
    bool keep = om >= omega_min && om > 0.0;
    for (int ka = 0; ka < nm; ka++) {
      cx<double> e = ev[(size_t)q * nm * nm + ka * nm + nu];
      double f = keep ? 1.0 / sqrt(2.0 * mass[ka / 3] * om) : 0.0;
      cx<double> E = mkc(e.x * f, e.y * f);
      size_t o = ((size_t)ka * nm + nu) * nq + q;
      if (ET64) ET64[o] = E;
      if (ET32) ET32[o] = mkc((float)E.x, (float)E.y);
    }
  }
}

// ---------------------------------------------------------------- complex GEMM
// C[M][N] (+)= op(A)[M][K] B[K][N];  op(A) = A or A^T (A stored [K][M]), optionally conjugated.
template <typename R>
__global__ void __launch_bounds__(256) k_cgemm(int M, int N, int K, const cx<R> *__restrict__ A, int lda, bool transA,
                                               bool conjA, const cx<R> *__restrict__ B, int ldb, cx<R> *C, int ldc,
                                               bool acc) {
  __shared__ cx<R> As[16][65];
  __shared__ cx<R> Bs[16][65];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  cx<R> c[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) c[i][j] = mkc<R>(0, 0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int t = threadIdx.x; t < 1024; t += 256) {
      int kk, mm;
      if (transA) {
        mm = t % 64;
        kk = t / 64;
      } else {
        kk = t % 16;
        mm = t / 16;
      }
      int gm = m0 + mm, gk = k0 + kk;
      cx<R> v = mkc<R>(0, 0);
      if (gm < M && gk < K) v = transA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      if (conjA) v.y = -v.y;
      As[kk][mm] = v;
    }
    for (int t = threadIdx.x; t < 1024; t += 256) {
      int nn = t % 64, kk = t / 64;
      int gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < K) ? B[(size_t)gk * ldb + gn] : mkc<R>(0, 0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; kk++) {
      cx<R> a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) cfma(c[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < M && gn < N) {
        cx<R> *p = C + (size_t)gm * ldc + gn;
        *p = acc ? (*p + c[i][j]) : c[i][j];
      }
    }
}

// Bg[k][Rp][a][j][n] = sum_i G1[k][Rp][a][j][i] U_k[i][n];  BH[k][Re][i][j] = P_k(Re) Hw(Re)_ij
template <typename R>
__global__ void k_build_Bg(int nk, int nRp, int nm, int nw, const cx<R> *__restrict__ G1,
                           const cx<double> *__restrict__ Uk, cx<R> *Bg) {
  size_t n = (size_t)nk * nRp * nm * nw * nw;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    int nn = (int)(idx % nw);
    size_t rest = idx / nw;  // (k, Rp, a, j)
    int k = (int)(rest / ((size_t)nRp * nm * nw));
    const cx<R> *g = G1 + rest * nw;
    const cx<double> *U = Uk + (size_t)k * nw * nw;
    cx<R> acc = mkc<R>(0, 0);
    for (int i = 0; i < nw; i++) cfma(acc, g[i], ccast<R>(U[i * nw + nn]));
    Bg[idx] = acc;
  }
}

template <typename R>
__global__ void k_build_BH(int nk, int nRe, int nw, const cx<double> *__restrict__ Pk, const cx<double> *__restrict__ Hw,
                           cx<R> *BH) {
  size_t nw2 = (size_t)nw * nw;
  size_t n = (size_t)nk * nRe * nw2;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    size_t e = idx % nw2;
    size_t kr = idx / nw2;  // k*nRe + r
    int r = (int)(kr % nRe);
    BH[idx] = ccast<R>(Pk[kr] * Hw[(size_t)r * nw2 + e]);
  }
}

__global__ void k_cast_c64_c32(size_t n, const cx<double> *__restrict__ in, cx<float> *out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = mkc((float)in[i].x, (float)in[i].y);
}

// ------------------------------------------------------------ per-pair kernel
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum v over the 128-thread block in a fixed order; result valid in thread 0.
__device__ __forceinline__ double block_sum128(double v, double *sh /*[4]*/) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) s = ((sh[0] + sh[1]) + sh[2]) + sh[3];
  return s;
}

// 1/x for x > 0: FP32 from rcp.approx with one Newton step (about an ulp), FP64 exact.
template <typename R>
__device__ __forceinline__ R rcp_pos(R x);
template <>
__device__ __forceinline__ float rcp_pos<float>(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r * fmaf(-x, r, 2.0f);
}
template <>
__device__ __forceinline__ double rcp_pos<double>(double x) {
  return 1.0 / x;
}

// f(a) - f(b) for scaled arguments a, b = (e - E_F)/kT (T > 0), given ia = 1/(1 + e^{-|a|})
// and ib = 1/(1 + e^{-|b|}): 2 sinh(d/2) e^{-S/2} ia ib with d = b - a, S = |a| + |b|, the sinh
// through expm1 of d or -d so that no exponent is positive (the identity of fermi_diff_f).
__device__ __forceinline__ float fermi_diff_scaled(float a, float b, float ia, float ib) {
  const float d = b - a, S = fabsf(a) + fabsf(b);
  const float num = d >= 0.0f ? -__expf(0.5f * (d - S)) * expm1f(-d) : __expf(-0.5f * (d + S)) * expm1f(d);
  return num * ia * ib;
}

// The vertex of one pair (k, q) (kl = k - a.k0; qq a valid q):
//   H(k+q)   = sum_Re P_q(Re) BH_k(Re)  (or the staged contraction)  -> Jacobi -> e_m (ascending), U
//   X_a      = sum_Rp P_q(Rp) Bg_k(Rp, a)   (= g_a(k,q) U_k)
//   G_nu     = sum_a E_q[a][nu] U^dagger X_a                 (= g_mn,nu)
// Returns false when the eigensolve did not converge.
template <typename R, int MW, int MM, bool FROMC>
__device__ __forceinline__ bool pair_vertex(const PairArgs &a, int kl, int k, int qq, R (&ekq)[MW], cx<R> (&U)[MW][MW],
                                            cx<R> (&G)[MM][MW][MW]) {
  constexpr int UW = MW <= 4 ? MW : 1;
  constexpr int UM = MM <= 4 ? MM : 1;
  const int nw = a.nw, nm = a.nm, nw2 = nw * nw, nq = a.nq;
  const cx<R> *PqTe = (const cx<R> *)a.PqTe;
  const cx<R> *PqTp = (const cx<R> *)a.PqTp;
  const cx<R> *BH = (const cx<R> *)a.BH + (size_t)k * a.nRe * nw2;
  const cx<R> *Bg = (const cx<R> *)a.Bg + (size_t)k * a.nRp * nm * nw2;
  const cx<R> *ET = (const cx<R> *)a.ET;
  cx<R> A[MW][MW];
#pragma unroll UW
  for (int i = 0; i < MW; i++)
#pragma unroll UW
    for (int j = 0; j < MW; j++) A[i][j] = mkc<R>(0, 0);
  if constexpr (FROMC) {
    // Hermitian part of the staged H(k+q)
    const float *C = a.Cq + (size_t)kl * a.cpk * a.ldc + qq;
#pragma unroll UW
    for (int i = 0; i < MW; i++)
#pragma unroll UW
      for (int j = 0; j < MW; j++)
        if (i < nw && j < nw) {
          const size_t ij = 2 * (size_t)(i * nw + j), ji = 2 * (size_t)(j * nw + i);
          A[i][j] = mkc<R>(R(0.5) * (C[ij * a.ldc] + C[ji * a.ldc]), R(0.5) * (C[(ij + 1) * a.ldc] - C[(ji + 1) * a.ldc]));
        }
  } else {
    for (int r = 0; r < a.nRe; r++) {
      cx<R> p = PqTe[(size_t)r * nq + qq];
      const cx<R> *b = BH + (size_t)r * nw2;
#pragma unroll UW
      for (int i = 0; i < MW; i++)
#pragma unroll UW
        for (int j = 0; j < MW; j++)
          if (i < nw && j < nw) cfma(A[i][j], p, b[i * nw + j]);
    }
  }
  bool nc = false;
  if constexpr (std::is_same<R, float>::value && MW == 4) {
    if (nw == 4) {
      // FP32 4 x 4: Householder reduction to a real tridiagonal matrix, real Jacobi
      // (the same eigensolve as the fused kernel; every lane of the warp calls it)
      Herm<4> Hm;
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = i; j < 4; j++)
          Hm.a[i][j] = i == j ? mkc(A[i][i].x, 0.0f)
                              : mkc(0.5f * (A[i][j].x + A[j][i].x), 0.5f * (A[i][j].y - A[j][i].y));
      nc = !eig_herm4(Hm, U);
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) A[i][j] = i == j ? mkc(Hm.a[i][i].x, 0.0f) : mkc(0.0f, 0.0f);
    } else {
      jacobi_herm<R, MW>(A, U, nw, jacobi_tol<R>::tol2, jacobi_tol<R>::maxsweep, nc);
    }
  } else {
    jacobi_herm<R, MW>(A, U, nw, jacobi_tol<R>::tol2, jacobi_tol<R>::maxsweep, nc);
  }
  sort_eig<R, MW>(A, U, ekq, nw);
#pragma unroll UM
  for (int v = 0; v < MM; v++)
#pragma unroll UW
    for (int i = 0; i < MW; i++)
#pragma unroll UW
      for (int j = 0; j < MW; j++) G[v][i][j] = mkc<R>(0, 0);
  for (int al = 0; al < nm; al++) {
    cx<R> X[MW][MW];
#pragma unroll UW
    for (int i = 0; i < MW; i++)
#pragma unroll UW
      for (int j = 0; j < MW; j++) X[i][j] = mkc<R>(0, 0);
    if constexpr (FROMC) {
      const float *C = a.Cq + ((size_t)kl * a.cpk + 2 * (size_t)nw2 * (1 + al)) * a.ldc + qq;
#pragma unroll UW
      for (int i = 0; i < MW; i++)
#pragma unroll UW
        for (int j = 0; j < MW; j++)
          if (i < nw && j < nw) {
            const size_t ij = 2 * (size_t)(i * nw + j);
            X[i][j] = mkc<R>(C[ij * a.ldc], C[(ij + 1) * a.ldc]);
          }
    } else {
      for (int r = 0; r < a.nRp; r++) {
        cx<R> p = PqTp[(size_t)r * nq + qq];
        const cx<R> *b = Bg + ((size_t)r * nm + al) * nw2;
#pragma unroll UW
        for (int i = 0; i < MW; i++)
#pragma unroll UW
          for (int j = 0; j < MW; j++)
            if (i < nw && j < nw) cfma(X[i][j], p, b[i * nw + j]);
      }
    }
    // Y = U^dagger X, then G_nu += E[al][nu] Y
#pragma unroll UW
    for (int m = 0; m < MW; m++) {
      if (m >= nw) continue;
#pragma unroll UW
      for (int n = 0; n < MW; n++) {
        if (n >= nw) continue;
        cx<R> y = mkc<R>(0, 0);
#pragma unroll UW
        for (int i = 0; i < MW; i++)
          if (i < nw) cfma(y, conjc(U[i][m]), X[i][n]);
#pragma unroll UM
        for (int v = 0; v < MM; v++)
          if (v < nm) cfma(G[v][m][n], ET[((size_t)al * nm + v) * nq + qq], y);
      }
    }
  }
  if (a.Cpol) {
    // long-range part: G_nu += i C_nu(q) [U_k+q^dagger U_k]
    const cx<double> *Uk = a.Uk + (size_t)k * nw2;
    const cx<R> *Cp = (const cx<R> *)a.Cpol;
#pragma unroll UW
    for (int m = 0; m < MW; m++)
#pragma unroll UW
      for (int n = 0; n < MW; n++) {
        if (m >= nw || n >= nw) continue;
        cx<R> o = mkc<R>(0, 0);
#pragma unroll UW
        for (int i = 0; i < MW; i++)
          if (i < nw) cfma(o, conjc(U[i][m]), ccast<R>(Uk[i * nw + n]));
#pragma unroll UM
        for (int v = 0; v < MM; v++) {
          if (v >= nm) continue;
          const cx<R> c = Cp[(size_t)v * nq + qq];
          cfma(G[v][m][n], mkc<R>(-c.y, c.x), o);  // i c o
        }
      }
  }
  return !nc;
}

// One thread per (k, q) pair; a block holds 128 consecutive q of one k.
// mode 0: linewidth terms of Eq. (linewidthel), reduced over the block;
// mode 1: write e_k+q and g_mn,nu;  mode 2: adjoint (see launch_pair).
template <typename R, int MW, int MM, int MODE, bool FROMC = false>
__global__ void __launch_bounds__(128) k_pair(PairArgs a) {
  constexpr int UW = MW <= 4 ? MW : 1;
  constexpr int UM = MM <= 4 ? MM : 1;
  __shared__ double sh[4];
  const int q = blockIdx.x * 128 + threadIdx.x;
  const int kl = blockIdx.y;
  const int k = a.k0 + kl;
  const bool valid = q < a.nq;
  const int qq = valid ? q : 0;
  const int nw = a.nw, nm = a.nm, nw2 = nw * nw, nq = a.nq;
  const cx<R> *ET = (const cx<R> *)a.ET;
  R ekq[MW];
  cx<R> U[MW][MW];
  cx<R> G[MM][MW][MW];
  const bool conv = pair_vertex<R, MW, MM, FROMC>(a, kl, k, qq, ekq, U, G);
  if (!conv && valid) atomicOr(a.dstatus, EPW_DEV_NOT_CONVERGED);

  const double *ek = a.eps_k + (size_t)k * nw;
  const R inv_sigma = (R)(1.0 / a.sigma);
  const R gnorm = (R)(1.0 / (a.sigma * 1.7724538509055160273));
  const double wqi = valid ? (a.wq ? a.wq[q] : 1.0 / nq) : 0.0;

  if (MODE == 0) {
    R acc[MW];
#pragma unroll UW
    for (int n = 0; n < MW; n++) acc[n] = R(0);
#pragma unroll UM
    for (int v = 0; v < MM; v++) {
      if (v >= nm) continue;
      R w = (R)a.omegaT[(size_t)v * nq + qq];
      if (!(w >= (R)a.omega_min) || !(w > R(0))) continue;
      R nb = occ_bose<R>(w, a.T);
#pragma unroll UW
      for (int m = 0; m < MW; m++) {
        if (m >= nw) continue;
        R f = occ_fermi<R>(ekq[m], a.EF, a.T);
        R cp = nb + f, cm = nb + R(1) - f;
#pragma unroll UW
        for (int n = 0; n < MW; n++) {
          if (n >= nw) continue;
          R x = (R)ek[n] - ekq[m];
          R g2 = cabs2(G[v][m][n]);
          acc[n] += g2 * (cp * gauss_r<R>(x + w, inv_sigma, gnorm) + cm * gauss_r<R>(x - w, inv_sigma, gnorm));
        }
      }
    }
    const int nqb = gridDim.x;
#pragma unroll UW
    for (int n = 0; n < MW; n++) {
      if (n >= nw) continue;
      double s = block_sum128((double)acc[n] * wqi, sh);
      if (threadIdx.x == 0) a.partial[((size_t)k * nqb + blockIdx.x) * nw + n] = s;
    }
  } else if (MODE == 1) {
    if (!valid) return;
    if (a.eps_kq) {
#pragma unroll UW
      for (int m = 0; m < MW; m++)
        if (m < nw) a.eps_kq[((size_t)k * nq + q) * nw + m] = (double)ekq[m];
    }
    if (a.gout) {
      cx<double> *o = a.gout + ((size_t)k * nq + q) * nm * nw2;
#pragma unroll UM
      for (int v = 0; v < MM; v++)
#pragma unroll UW
        for (int m = 0; m < MW; m++)
#pragma unroll UW
          for (int n = 0; n < MW; n++)
            if (v < nm && m < nw && n < nw) o[(v * nw + m) * nw + n] = ccast<double>(G[v][m][n]);
    }
  } else {
    // Adjoint of L = sum_{k,n} c_nk Im Sigma_nk.
    //   W_nu,mn = c_nk pi w_q [(n+f) d+ + (n+1-f) d-],  Gbar_nu = 2 W G_nu
    //   Xbar_a  = U sum_nu conj(E[a][nu]) Gbar_nu   (written for the adjoint GEMMs)
    //   dL/dT, dL/dE_F through n(T), f(T, E_F).
    const double *cot = a.cot + (size_t)k * nw;
    double sT = 0.0, sE = 0.0;
    const double kT = EPW_KB * a.T;
#pragma unroll UM
    for (int v = 0; v < MM; v++) {
      if (v >= nm) continue;
      R w = (R)a.omegaT[(size_t)v * nq + qq];
      bool keep = (w >= (R)a.omega_min) && (w > R(0));
      R nb = keep ? occ_bose<R>(w, a.T) : R(0);
      double dn = keep ? (double)nb * ((double)nb + 1.0) * (double)w / (kT * a.T) : 0.0;
#pragma unroll UW
      for (int m = 0; m < MW; m++) {
        if (m >= nw) continue;
        R f = occ_fermi<R>(ekq[m], a.EF, a.T);
        double ff = fermi_ff_d((double)ekq[m] - a.EF, a.T);
        double dfT = ff * ((double)ekq[m] - a.EF) / (kT * a.T);
        double dfE = ff / kT;
#pragma unroll UW
        for (int n = 0; n < MW; n++) {
          if (n >= nw) continue;
          R x = (R)ek[n] - ekq[m];
          R dp = gauss_r<R>(x + w, inv_sigma, gnorm), dm = gauss_r<R>(x - w, inv_sigma, gnorm);
          double c = keep ? cot[n] * EPW_PI * wqi : 0.0;
          R W = (R)(c * ((double)(nb + f) * dp + (double)(nb + R(1) - f) * dm));
          double g2 = (double)cabs2(G[v][m][n]);
          // (dn + dfT) d+ + (dn - dfT) d- = dn (d+ + d-) + dfT (d+ - d-), the difference
          // without cancellation for soft modes
          const double dd = (double)gauss_diff_r<R>(x, w, inv_sigma, gnorm);
          sT += c * g2 * (dn * ((double)dp + (double)dm) + dfT * dd);
          sE += c * g2 * dfE * dd;
          G[v][m][n] = (R(2) * W) * G[v][m][n];
        }
      }
    }
    if (valid) {
      cx<R> *xb = (cx<R> *)a.xbar + ((size_t)q * a.nkc + kl) * nm * nw2;
      for (int al = 0; al < nm; al++) {
        cx<R> Yb[MW][MW];
#pragma unroll UW
        for (int m = 0; m < MW; m++)
#pragma unroll UW
          for (int n = 0; n < MW; n++) {
            cx<R> s = mkc<R>(0, 0);
#pragma unroll UM
            for (int v = 0; v < MM; v++)
              if (v < nm && m < nw && n < nw) cfma(s, conjc(ET[((size_t)al * nm + v) * nq + qq]), G[v][m][n]);
            Yb[m][n] = s;
          }
#pragma unroll UW
        for (int i = 0; i < MW; i++)
#pragma unroll UW
          for (int n = 0; n < MW; n++) {
            if (i >= nw || n >= nw) continue;
            cx<R> s = mkc<R>(0, 0);
#pragma unroll UW
            for (int m = 0; m < MW; m++)
              if (m < nw) cfma(s, U[i][m], Yb[m][n]);
            xb[(size_t)al * nw2 + i * nw + n] = s;
          }
      }
    }
    const int nqb = gridDim.x;
    double tT = block_sum128(sT, sh);
    if (threadIdx.x == 0) a.partialT[(size_t)kl * nqb + blockIdx.x] = tT;
    double tE = block_sum128(sE, sh);
    if (threadIdx.x == 0) a.partialE[(size_t)kl * nqb + blockIdx.x] = tE;
  }
}

// Per-(q, nu) sums over k (phonon self-energy, Eq. (linewidthph) on shell;
// coupling strength, Eq. (lambdaEQ); nesting function, Eq. (nestingfct)):
// one thread per q of a block of 128, looping over the a.nk k-points from
// a.k0 in order; the block's chunk index is blockIdx.y (k = a.k0 + blockIdx.y *
// a.nkc + j).  Writes, per q, the partial sums over its k chunk:
//   out[chunk][q][nu]          sum_k w_k sum_mn |g|^2 (f_nk - f_mk+q) delta(e_nk - e_mk+q - w_qnu)
//   out[chunk][q][nm + nu]     sum_k w_k sum_mn |g|^2 delta(e_nk - E_F) delta(e_mk+q - E_F)
//   out[chunk][q][2 nm]        sum_k w_k sum_mn delta(e_nk - E_F) delta(e_mk+q - E_F)
template <typename R, int MW, int MM, bool FROMC>
__global__ void __launch_bounds__(128) k_pair_ph(PairArgs a) {
  constexpr int UW = MW <= 4 ? MW : 1;
  constexpr int UM = MM <= 4 ? MM : 1;
  const int q = blockIdx.x * 128 + threadIdx.x;
  // lanes past the last q run on q = 0 (the eigensolve exits on a warp vote) and write nothing
  const bool valid = q < a.nq;
  const int qq = valid ? q : 0;
  const int nw = a.nw, nm = a.nm, nq = a.nq;
  const int kc0 = blockIdx.y * a.nkc;
  const int kc1 = min(a.nk, kc0 + a.nkc);
  const R inv_sigma = (R)(1.0 / a.sigma);
  const R gnorm = (R)(1.0 / (a.sigma * 1.7724538509055160273));
  R w[MM];
  bool keep[MM];
#pragma unroll UM
  for (int v = 0; v < MM; v++) {
    w[v] = v < nm ? (R)a.omegaT[(size_t)v * nq + qq] : R(0);
    keep[v] = v < nm && (w[v] >= (R)a.omega_min) && (w[v] > R(0));
  }
  double sp[MM], sl[MM], sz = 0.0;
#pragma unroll UM
  for (int v = 0; v < MM; v++) sp[v] = sl[v] = 0.0;
  const float efF = (float)a.EF, iktF = a.T > 0.0 ? (float)(1.0 / (EPW_KB * a.T)) : 0.0f;
  for (int kl = kc0; kl < kc1; kl++) {
    const int k = a.k0 + kl;
    R ekq[MW];
    cx<R> U[MW][MW];
    cx<R> G[MM][MW][MW];
    const bool conv = pair_vertex<R, MW, MM, FROMC>(a, kl, k, qq, ekq, U, G);
    if (!conv && valid) atomicOr(a.dstatus, EPW_DEV_NOT_CONVERGED);
    const double wk = a.wq ? a.wq[k] : 1.0 / a.nk_total;
    R en[MW], dn[MW], dm[MW];
#pragma unroll UW
    for (int n = 0; n < MW; n++) {
      en[n] = n < nw ? (R)a.eps_k[(size_t)k * nw + n] : R(0);
      dn[n] = gauss_r<R>(en[n] - (R)a.EF, inv_sigma, gnorm);
      dm[n] = gauss_r<R>(ekq[n] - (R)a.EF, inv_sigma, gnorm);
    }
    R z = R(0);
    R fd[MW][MW];  // f_nk - f_mk+q
    // FP32 form: the scaled arguments (e - E_F)/kT and 1/(1 + e^{-|a|}) once per band
    float ga[MW], ia[MW], gb[MW], ib[MW];
    if constexpr (sizeof(R) == sizeof(float)) {
#pragma unroll UW
      for (int n = 0; n < MW; n++) {
        ga[n] = (en[n] - efF) * iktF;
        ia[n] = rcp_pos<float>(1.0f + __expf(-fabsf(ga[n])));
        gb[n] = (ekq[n] - efF) * iktF;
        ib[n] = rcp_pos<float>(1.0f + __expf(-fabsf(gb[n])));
      }
    }
#pragma unroll UW
    for (int m = 0; m < MW; m++)
#pragma unroll UW
      for (int n = 0; n < MW; n++) {
        fd[m][n] = R(0);
        if (m < nw && n < nw) {
          z += dn[n] * dm[m];
          if constexpr (sizeof(R) == sizeof(double))
            fd[m][n] = (R)fermi_diff_d((double)en[n], (double)ekq[m], a.EF, a.T);
          else
            fd[m][n] = a.T > 0.0 ? fermi_diff_scaled(ga[n], gb[m], ia[n], ib[m])
                                 : fermi_diff_f((float)en[n], (float)ekq[m], a.EF, a.T);
        }
      }
    sz += wk * (double)z;
#pragma unroll UM
    for (int v = 0; v < MM; v++) {
      if (!keep[v]) continue;
      R p = R(0), l = R(0);
#pragma unroll UW
      for (int m = 0; m < MW; m++)
#pragma unroll UW
        for (int n = 0; n < MW; n++) {
          if (m >= nw || n >= nw) continue;
          const R g2 = cabs2(G[v][m][n]);
          p += g2 * fd[m][n] * gauss_r<R>(en[n] - ekq[m] - w[v], inv_sigma, gnorm);
          l += g2 * dn[n] * dm[m];
        }
      sp[v] += wk * (double)p;
      sl[v] += wk * (double)l;
    }
  }
  if (!valid) return;
  double *o = a.partial + ((size_t)blockIdx.y * nq + q) * (2 * nm + 1);
  for (int v = 0; v < nm; v++) {
    o[v] = sp[v < MM ? v : 0];
    o[nm + v] = sl[v < MM ? v : 0];
  }
  o[2 * nm] = sz;
}

// Sum of the per-chunk partials in chunk order; Pi'' = 2 pi sum_p, lambda = sum_l / (N(E_F) w)
// for kept modes (0 otherwise), zeta = sum_z.  dos: N(E_F) on the device.
__global__ void k_ph_finalize(int nq, int nm, int nchunk, const double *__restrict__ partial,
                              const double *__restrict__ omegaT, double omega_min, const double *__restrict__ dos,
                              double *pi_im, double *lam, double *zeta) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int st = 2 * nm + 1;
  for (int j = 0; j < st; j++) {
    double s = 0.0, c = 0.0;  // Neumaier over chunks
    for (int ch = 0; ch < nchunk; ch++) {
      const double x = partial[((size_t)ch * nq + q) * st + j];
      const double t = s + x;
      c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
      s = t;
    }
    s += c;
    if (j < nm) {
      const double w = omegaT[(size_t)j * nq + q];
      const bool keep = w >= omega_min && w > 0.0;
      if (pi_im) pi_im[(size_t)q * nm + j] = keep ? 2.0 * EPW_PI * s : 0.0;
    } else if (j < 2 * nm) {
      const int v = j - nm;
      const double w = omegaT[(size_t)v * nq + q];
      const bool keep = w >= omega_min && w > 0.0 && dos[0] > 0.0;
      if (lam) lam[(size_t)q * nm + v] = keep ? s / (dos[0] * w) : 0.0;
    } else if (zeta) {
      zeta[q] = s;
    }
  }
}

// Per-k terms of N(E_F) = sum_k w_k sum_n delta(e_nk - E_F).
__global__ void k_dos_terms(int nk, int nw, const double *__restrict__ epsk, const double *__restrict__ wk,
                            double EF, double sigma, double *terms) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  const double inv = 1.0 / sigma, norm = 1.0 / (sigma * 1.7724538509055160273);
  double s = 0.0;
  for (int n = 0; n < nw; n++) s += gauss_r<double>(epsk[(size_t)k * nw + n] - EF, inv, norm);
  terms[k] = (wk ? wk[k] : 1.0 / nk) * s;
}

// Complex self-energy of Eq. (elselfenergy) on a frequency grid (omega from E_F, i delta
// broadening): one thread per (k, q) pair, a block holds 128 consecutive q of one k.  For
// each band n and grid point i (the grid, then omega = 0 for the shift of Eq. (realpartselfenergy)),
// the thread sums over (m, nu), each warp sums its 32 q (shuffles), and lane 0 writes
//   out[(kl * nqw + q / 32) * nw + n][i]   (complex, re/im),  nqw = ceil(nq / 32).
template <typename R, int MW, int MM, bool FROMC>
__global__ void __launch_bounds__(128) k_pair_se(PairArgs a, int nom, const double *__restrict__ omega,
                                                 double delta, double2 *out) {
  constexpr int UW = MW <= 4 ? MW : 1;
  constexpr int UM = MM <= 4 ? MM : 1;
  const int q = blockIdx.x * 128 + threadIdx.x;
  const int kl = blockIdx.y, k = a.k0 + kl;
  const bool valid = q < a.nq;
  const int qq = valid ? q : 0;
  const int nw = a.nw, nm = a.nm, nq = a.nq;
  R ekq[MW];
  cx<R> U[MW][MW];
  cx<R> G[MM][MW][MW];
  const bool conv = pair_vertex<R, MW, MM, FROMC>(a, kl, k, qq, ekq, U, G);
  if (!conv && valid) atomicOr(a.dstatus, EPW_DEV_NOT_CONVERGED);
  const R wqi = valid ? (R)(a.wq ? a.wq[q] : 1.0 / nq) : R(0);
  R w[MM], cp[MM][MW], cm[MM][MW];
#pragma unroll UM
  for (int v = 0; v < MM; v++) {
    w[v] = v < nm ? (R)a.omegaT[(size_t)v * nq + qq] : R(0);
    const bool keep = v < nm && (w[v] >= (R)a.omega_min) && (w[v] > R(0));
    const R nb = keep ? occ_bose<R>(w[v], a.T) : R(0);
#pragma unroll UW
    for (int m = 0; m < MW; m++) {
      const R f = m < nw ? occ_fermi<R>(ekq[m], a.EF, a.T) : R(0);
      cp[v][m] = keep ? wqi * (nb + f) : R(0);
      cm[v][m] = keep ? wqi * (nb + R(1) - f) : R(0);
    }
  }
  const R dl = (R)delta, d2 = dl * dl;
  const int nqw = (nq + 31) / 32;
  const int lane = threadIdx.x & 31;
  // |g_mn,nu|^2 once; the Lorentzian factors depend on (omega_i, nu, m) only and
  // serve every band n
  R g2[MM][MW][MW];
#pragma unroll UM
  for (int v = 0; v < MM; v++)
#pragma unroll UW
    for (int m = 0; m < MW; m++)
#pragma unroll UW
      for (int n = 0; n < MW; n++) g2[v][m][n] = (v < nm && m < nw && n < nw) ? cabs2(G[v][m][n]) : R(0);
  for (int i = 0; i <= nom; i++) {
    const R om = i < nom ? (R)omega[i] : R(0);
    R sr[MW], si[MW];
#pragma unroll UW
    for (int n = 0; n < MW; n++) sr[n] = si[n] = R(0);
#pragma unroll UM
    for (int v = 0; v < MM; v++) {
      if (v >= nm) continue;
#pragma unroll UW
      for (int m = 0; m < MW; m++) {
        if (m >= nw) continue;
        const R x = om - (ekq[m] - (R)a.EF);
        const R xp = x + w[v], xm = x - w[v];
        // 1/(x + i delta) = (x - i delta) / (x^2 + delta^2)
        const R ap = cp[v][m] * rcp_pos<R>(xp * xp + d2), am = cm[v][m] * rcp_pos<R>(xm * xm + d2);
        const R tr = ap * xp + am * xm, ti = ap + am;
#pragma unroll UW
        for (int n = 0; n < MW; n++) {
          sr[n] += g2[v][m][n] * tr;
          si[n] += g2[v][m][n] * ti;
        }
      }
    }
#pragma unroll UW
    for (int n = 0; n < MW; n++) {
      if (n >= nw) continue;
      // warp sum in the working precision (FP32 forms: 32 terms, a few ulp; the FP64
      // pipe is a small fraction of FP32 here), then FP64 for the cross-warp sum
      R dr = sr[n], di = -dl * si[n];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dr += __shfl_down_sync(0xffffffffu, dr, o);
        di += __shfl_down_sync(0xffffffffu, di, o);
      }
      if (lane == 0 && q - lane < nq)
        out[(((size_t)kl * nqw + (q >> 5)) * nw + n) * (nom + 1) + i] = make_double2((double)dr, (double)di);
    }
  }
}

// Sum over the per-warp partials (fixed order, compensated) into Sigma_nk(omega_i) and, with
// spec, the spectral function of Eq. (spectral_funct) (Sigma'' = -Im Sigma, real part shifted
// by its value at omega = 0): one block per (k, n), one thread per grid point (the q-warp rows
// of a (k, n) are read along omega, contiguously), then the spectral function from the sums.
__global__ void k_se_finalize(int nkc, int k0, int nw, int nqw, int nom, const double2 *__restrict__ part,
                              const double *__restrict__ omega, const double *__restrict__ epsk, double EF,
                              double2 *sig, double *spec) {
  __shared__ double re0s;
  const int kl = blockIdx.x / nw, n = blockIdx.x % nw, k = k0 + kl;
  const size_t stride = (size_t)nw * (nom + 1);
  const double2 *base = part + ((size_t)kl * nqw * nw + n) * (nom + 1);
  for (int i = threadIdx.x; i <= nom; i += blockDim.x) {
    double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;
    for (int j = 0; j < nqw; j++) {
      const double2 x = base[(size_t)j * stride + i];
      double u = sr + x.x;
      cr += fabs(sr) >= fabs(x.x) ? (sr - u) + x.x : (x.x - u) + sr;
      sr = u;
      u = si + x.y;
      ci += fabs(si) >= fabs(x.y) ? (si - u) + x.y : (x.y - u) + si;
      si = u;
    }
    const double2 t = make_double2(sr + cr, si + ci);
    if (i < nom)
      sig[((size_t)k * nw + n) * nom + i] = t;
    else
      re0s = t.x;
  }
  __syncthreads();
  if (!spec) return;
  const double re0 = re0s;
  const double e = epsk[(size_t)k * nw + n] - EF;
  for (int i = threadIdx.x; i < nom; i += blockDim.x) {
    const size_t o = ((size_t)k * nw + n) * nom + i;
    const double2 t = sig[o];
    const double s2 = -t.y;
    const double den = omega[i] - e - (t.x - re0);
    spec[o] = fabs(s2) / (EPW_PI * (den * den + s2 * s2));
  }
}

// C_nu(q) = pref sum_{kappa,a} E[kappa a][nu] F_{kappa a}(q), F = sum_{G, q+G != 0} damp(q+G)
// ((q+G).Z*_kappa)_a / ((q+G).eps.(q+G)), damp(x) = exp(-x.eps.x / (4 alpha)), G = sum n_i b_i,
// |n_i| <= gmax (Eq. (long-range) with the readings of its prefactor and convergence factor).
// One thread per q; F accumulated in FP64.
template <typename R>
__global__ void k_polar_factors(int nq, int nm, int nat, const double *__restrict__ q, PolarK pk,
                                const double *__restrict__ Z, const cx<R> *__restrict__ ET, cx<R> *C) {
  const int iq = blockIdx.x * blockDim.x + threadIdx.x;
  if (iq >= nq) return;
  double F[18];
  for (int i = 0; i < 18; i++) F[i] = 0.0;
  const double q0 = q[3 * iq], q1 = q[3 * iq + 1], q2 = q[3 * iq + 2];
  const int G = pk.gmax;
  for (int n1 = -G; n1 <= G; n1++)
    for (int n2 = -G; n2 <= G; n2++)
      for (int n3 = -G; n3 <= G; n3++) {
        double x[3];
        for (int c = 0; c < 3; c++)
          x[c] = (q0 + n1) * pk.b[c] + (q1 + n2) * pk.b[3 + c] + (q2 + n3) * pk.b[6 + c];
        if (x[0] * x[0] + x[1] * x[1] + x[2] * x[2] == 0.0) continue;
        double xex = 0.0;
        for (int c = 0; c < 3; c++)
          for (int d = 0; d < 3; d++) xex += x[c] * pk.eps[c * 3 + d] * x[d];
        const double w = exp(-xex / (4.0 * pk.alpha)) / xex;
        for (int kap = 0; kap < nat; kap++)
          for (int a = 0; a < 3; a++) {
            const double *Zk = Z + kap * 9;
            F[kap * 3 + a] += w * (x[0] * Zk[a] + x[1] * Zk[3 + a] + x[2] * Zk[6 + a]);
          }
      }
  for (int v = 0; v < nm; v++) {
    double cr = 0.0, ci = 0.0;
    for (int ka = 0; ka < nm; ka++) {
      const cx<R> e = ET[((size_t)ka * nm + v) * nq + iq];
      cr += (double)e.x * F[ka];
      ci += (double)e.y * F[ka];
    }
    C[(size_t)v * nq + iq] = mkc<R>((R)(pk.pref * cr), (R)(pk.pref * ci));
  }
}

// alpha^2 F on a grid (Eq. (isotropiceliash)): one block per grid point, each
// thread a fixed stride of the (q, nu) terms (compensated), then a fixed tree.
__global__ void k_eliashberg(int nq, int nm, const double *__restrict__ omega, const double *__restrict__ lam,
                             const double *__restrict__ wq, const double *__restrict__ grid, double sigma_ph,
                             double *a2f) {
  __shared__ double ss[256];
  const double x0 = grid[blockIdx.x];
  const double inv = 1.0 / sigma_ph, norm = 1.0 / (sigma_ph * 1.7724538509055160273);
  double s = 0.0, c = 0.0;
  const size_t n = (size_t)nq * nm;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int iq = (int)(i / nm);
    const double w = omega[i];
    const double x = 0.5 * (wq ? wq[iq] : 1.0 / nq) * w * lam[i] * gauss_r<double>(x0 - w, inv, norm);
    const double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  ss[threadIdx.x] = s + c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) ss[threadIdx.x] += ss[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) a2f[blockIdx.x] = ss[0];
}

// gw[Re][Rp][...] = wRe wRp g   (g complex128 or, with is_c64, complex64)
__global__ void k_set_vertex(int nRe, int nRp, size_t per, const void *__restrict__ g, int is_c64,
                             const double *__restrict__ wRe, const double *__restrict__ wRp, cx<double> *gw) {
  size_t n = (size_t)nRe * nRp * per;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    size_t rr = idx / per;
    int a = (int)(rr / nRp), b = (int)(rr % nRp);
    double s = wRe[a] * wRp[b];
    double re, im;
    if (is_c64) {
      re = ((const float *)g)[2 * idx];
      im = ((const float *)g)[2 * idx + 1];
    } else {
      re = ((const double *)g)[2 * idx];
      im = ((const double *)g)[2 * idx + 1];
    }
    gw[idx] = mkc(s * re, s * im);
  }
}

__device__ __forceinline__ void neumaier_add(double &s, double &c, double x) {
  const double u = s + x;
  c += fabs(s) >= fabs(x) ? (s - u) + x : (x - u) + s;
  s = u;
}

// out[k][n] = pi * sum_qb partial[k][qb][n], compensated (Neumaier).  One warp
// per (k, n): lane l sums qb = l, l+32, ... in order, then the 32 partial sums
// are combined by a fixed shuffle tree, so the result does not depend on timing.
__global__ void k_finalize(int nk, int nqb, int nw, const double *__restrict__ partial, double *out) {
  const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= nk * nw) return;
  const int k = w / nw, n = w % nw;
  double s = 0.0, c = 0.0;
  for (int b = lane; b < nqb; b += 32) neumaier_add(s, c, partial[((size_t)k * nqb + b) * nw + n]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double s2 = __shfl_down_sync(0xffffffffu, s, o);
    const double c2 = __shfl_down_sync(0xffffffffu, c, o);
    neumaier_add(s, c, s2);
    c += c2;
  }
  if (lane == 0) out[w] = EPW_PI * (s + c);
}

// The same sums with one block of four warps per k when nw divides 32: the
// partial row of k is read contiguously, warp w taking the w-th quarter; lane l
// owns band n = l % nw, lanes with the same n are combined by a fixed shuffle tree
// (offsets 16 .. nw) and the four warps' sums in warp order.
__global__ void __launch_bounds__(128) k_finalize_k(int nk, int nqb, int nw, const double *__restrict__ partial,
                                                    double *out) {
  __shared__ double sh_s[4][32], sh_c[4][32];
  const int k = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double *row = partial + (size_t)k * nqb * nw;
  const int n = nqb * nw;
  const int per = ((n + 127) / 128) * 32;  // elements per warp, a multiple of 32
  const int j0 = warp * per, j1 = min(n, j0 + per);
  double s = 0.0, c = 0.0;
  int j = j0 + lane;
  for (; j + 96 < j1; j += 128) {
    const double x0 = row[j], x1 = row[j + 32], x2 = row[j + 64], x3 = row[j + 96];
    neumaier_add(s, c, x0);
    neumaier_add(s, c, x1);
    neumaier_add(s, c, x2);
    neumaier_add(s, c, x3);
  }
  for (; j < j1; j += 32) neumaier_add(s, c, row[j]);
  for (int o = 16; o >= nw; o >>= 1) {
    const double s2 = __shfl_down_sync(0xffffffffu, s, o);
    const double c2 = __shfl_down_sync(0xffffffffu, c, o);
    neumaier_add(s, c, s2);
    c += c2;
  }
  sh_s[warp][lane] = s;
  sh_c[warp][lane] = c;
  __syncthreads();
  if (warp == 0 && lane < nw) {
    double S = 0.0, C = 0.0;
    for (int w = 0; w < 4; w++) {
      neumaier_add(S, C, sh_s[w][lane]);
      C += sh_c[w][lane];
    }
    out[(size_t)k * nw + lane] = EPW_PI * (S + C);
  }
}

// out[0] (+)= scale * sum_i partial[i], one block, fixed order, compensated.
__global__ void k_sum_scalar(int n, const double *__restrict__ partial, double scale, double *out) {
  __shared__ double ss[256], cc[256];
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    double x = partial[i];
    double u = s + x;
    c += fabs(s) >= fabs(x) ? (s - u) + x : (x - u) + s;
    s = u;
  }
  ss[threadIdx.x] = s;
  cc[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, C = 0.0;
    for (int i = 0; i < 256; i++) {
      double x = ss[i];
      double u = S + x;
      C += fabs(S) >= fabs(x) ? (S - u) + x : (x - u) + S;
      S = u;
      C += cc[i];
    }
    out[0] += scale * (S + C);
  }
}

// G1bar[k][Rp][a][j][i] = sum_n Bbar[Rp][k][a][j][n] conj(U_k[i][n])
template <typename R>
__global__ void k_bg_adjoint_rotate(int nk, int k0, int nRp, int nm, int nw, const cx<R> *__restrict__ Bbar,
                                    const cx<double> *__restrict__ Uk, cx<R> *G1bar) {
  size_t per = (size_t)nm * nw * nw;
  size_t n = (size_t)nk * nRp * per;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(idx % nw);
    size_t rest = idx / nw;  // (k, Rp, a, j)
    int aj = (int)(rest % ((size_t)nm * nw));
    size_t kr = rest / ((size_t)nm * nw);
    int Rp = (int)(kr % nRp);
    int k = (int)(kr / nRp);
    const cx<R> *b = Bbar + ((size_t)Rp * nk + k) * per + (size_t)aj * nw;
    const cx<double> *U = Uk + (size_t)(k0 + k) * nw * nw;
    cx<R> acc = mkc<R>(0, 0);
    for (int nn = 0; nn < nw; nn++) cfma(acc, b[nn], conjc(ccast<R>(U[i * nw + nn])));
    G1bar[idx] = acc;
  }
}

// dg[Re][Rp][...] (+)= wRe wRp gwbar
template <typename R>
__global__ void k_dg_scale(int nRe, int nRp, size_t per, const double *__restrict__ wRe,
                           const double *__restrict__ wRp, const cx<R> *__restrict__ gwbar, double *dg, bool acc) {
  size_t n = (size_t)nRe * nRp * per;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    size_t rr = idx / per;
    int a = (int)(rr / nRp), b = (int)(rr % nRp);
    double s = wRe[a] * wRp[b];
    double re = s * (double)gwbar[idx].x, im = s * (double)gwbar[idx].y;
    if (acc) {
      dg[2 * idx] += re;
      dg[2 * idx + 1] += im;
    } else {
      dg[2 * idx] = re;
      dg[2 * idx + 1] = im;
    }
  }
}

}  // namespace

// ------------------------------------------------------------------ launchers
void launch_phases(int npt, const double *x, int nR, const int *R, int rmax, cx<double> *rm, cx<double> *T64,
                   cx<float> *T32, cudaStream_t st) {
  size_t n = (size_t)npt * nR;
  if (!n) return;
  if (rmax <= PH_RMAX && nR >= 2 * (2 * PH_RMAX + 1))
    k_phases_fact<<<(npt + 127) / 128, 128, 0, st>>>(npt, x, nR, R, rmax < 0 ? 0 : rmax, rm, T64, T32);
  else
    k_phases<<<nblocks(n, 256), 256, 0, st>>>(npt, x, nR, R, rm, T64, T32);
  epw_count_launch();
}

void launch_fourier_d(int npt, int nR, const cx<double> *PT, const cx<double> *X, int msize, cx<double> *out,
                      cudaStream_t st) {
  size_t n = (size_t)npt * msize;
  if (!n) return;
  k_fourier_d<<<nblocks(n, 256), 256, 0, st>>>(npt, nR, PT, X, msize, out);
  epw_count_launch();
}

void launch_eigh_d(int nmat, int n, cx<double> *A, double *w, cx<double> *V, unsigned *dstatus, cudaStream_t st) {
  if (!nmat) return;
  // one warp per block: the FP64 pipe is per SM, so small batches spread over more SMs
  int b = (nmat + 31) / 32;
  if (n <= 3)
    k_eigh_d<3><<<b, 32, 0, st>>>(nmat, n, A, w, V, dstatus);
  else if (n <= 4)
    k_eigh_d<4><<<b, 32, 0, st>>>(nmat, n, A, w, V, dstatus);
  else if (n <= 9)
    k_eigh_d<9><<<(nmat + 63) / 64, 64, 0, st>>>(nmat, n, A, w, V, dstatus);
  else
    k_eigh_d<18><<<(nmat + 63) / 64, 64, 0, st>>>(nmat, n, A, w, V, dstatus);
  epw_count_launch();
}

void launch_phonon_post(int nq, int nm, const double *w2, const cx<double> *ev, const double *mass, double omega_min,
                        double *omegaT, cx<double> *ET64, cx<float> *ET32, double *omega_out, cudaStream_t st) {
  size_t n = (size_t)nq * nm;
  if (!n) return;
  k_phonon_post<<<nblocks(n, 256), 256, 0, st>>>(nq, nm, w2, ev, mass, omega_min, omegaT, ET64, ET32, omega_out);
  epw_count_launch();
}

template <typename R>
void launch_cgemm(int M, int N, int K, const cx<R> *A, int lda, bool transA, bool conjA, const cx<R> *B, int ldb,
                  cx<R> *C, int ldc, bool accumulate, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_cgemm<R><<<grid, 256, 0, st>>>(M, N, K, A, lda, transA, conjA, B, ldb, C, ldc, accumulate);
  epw_count_launch();
}
template void launch_cgemm<double>(int, int, int, const cx<double> *, int, bool, bool, const cx<double> *, int,
                                   cx<double> *, int, bool, cudaStream_t);
template void launch_cgemm<float>(int, int, int, const cx<float> *, int, bool, bool, const cx<float> *, int,
                                  cx<float> *, int, bool, cudaStream_t);

template <typename R>
void launch_build_B(const epw_model *m, int nk, const cx<double> *Pk, const cx<R> *G1, const cx<double> *Uk,
                    cx<R> *Bg, cx<R> *BH, cudaStream_t st) {
  size_t nbg = (size_t)nk * m->nRp * m->nm * m->nw * m->nw;
  if (nbg && Bg) {
    k_build_Bg<R><<<nblocks(nbg, 256), 256, 0, st>>>(nk, m->nRp, m->nm, m->nw, G1, Uk, Bg);
    epw_count_launch();
  }
  size_t nbh = (size_t)nk * m->nRe * m->nw * m->nw;
  if (nbh && BH) {
    k_build_BH<R><<<nblocks(nbh, 256), 256, 0, st>>>(nk, m->nRe, m->nw, Pk, m->Hw, BH);
    epw_count_launch();
  }
}
template void launch_build_B<double>(const epw_model *, int, const cx<double> *, const cx<double> *,
                                     const cx<double> *, cx<double> *, cx<double> *, cudaStream_t);
template void launch_build_B<float>(const epw_model *, int, const cx<double> *, const cx<float> *,
                                    const cx<double> *, cx<float> *, cx<float> *, cudaStream_t);

void launch_cast_c64_to_c32(size_t n, const cx<double> *in, cx<float> *out, cudaStream_t st) {
  if (!n) return;
  k_cast_c64_c32<<<nblocks(n, 256), 256, 0, st>>>(n, in, out);
  epw_count_launch();
}

template <typename R, int MW, int MM>
static void pair_dispatch_mode(const PairArgs &a, int mode, dim3 grid, cudaStream_t st) {
  if (mode == 0)
    k_pair<R, MW, MM, 0><<<grid, 128, 0, st>>>(a);
  else if (mode == 1)
    k_pair<R, MW, MM, 1><<<grid, 128, 0, st>>>(a);
  else
    k_pair<R, MW, MM, 2><<<grid, 128, 0, st>>>(a);
  epw_count_launch();
}

template <typename R>
epw_status launch_pair(const PairArgs &a, int mode, cudaStream_t st) {
  int nkl = (mode == 2) ? a.nkc : a.nk;
  if (nkl <= 0 || a.nq <= 0) return EPW_OK;
  dim3 grid((a.nq + 127) / 128, nkl);
  if (a.nw <= 1 && a.nm <= 3)
    pair_dispatch_mode<R, 1, 3>(a, mode, grid, st);
  else if (a.nw <= 4 && a.nm <= 3)
    pair_dispatch_mode<R, 4, 3>(a, mode, grid, st);
  else if (a.nw <= 8 && a.nm <= 9)
    pair_dispatch_mode<R, 8, 9>(a, mode, grid, st);
  else
    return launch_pair_wide<R>(a, mode, st);
  return EPW_OK;
}
template epw_status launch_pair<double>(const PairArgs &, int, cudaStream_t);
template epw_status launch_pair<float>(const PairArgs &, int, cudaStream_t);

epw_status launch_pair_staged(const PairArgs &a, int mode, cudaStream_t st) {
  int nkl = (mode == 2) ? a.nkc : a.nk;
  if (nkl <= 0 || a.nq <= 0) return EPW_OK;
  if (!a.Cq) return EPW_ERR_UNSUPPORTED;
  if (a.nw > 8 || a.nm > 9) {
    // linewidth: only the terms within the Gaussian cutoff (EPW_STAGED_PAIR=dense: every term,
    // cyclic Jacobi per warp)
    const char *f = getenv("EPW_STAGED_PAIR");
    if (mode == 0 && !(f && !strcmp(f, "dense"))) return launch_pair_sparse(a, st);
    return launch_pair_wide<float>(a, mode, st);
  }
  dim3 grid((a.nq + 127) / 128, nkl);
  if (mode == 0)
    k_pair<float, 8, 9, 0, true><<<grid, 128, 0, st>>>(a);
  else if (mode == 1)
    k_pair<float, 8, 9, 1, true><<<grid, 128, 0, st>>>(a);
  else
    k_pair<float, 8, 9, 2, true><<<grid, 128, 0, st>>>(a);
  epw_count_launch();
  return EPW_OK;
}

template <typename R, bool FROMC>
static epw_status ph_dispatch(const PairArgs &a, dim3 grid, cudaStream_t st) {
  if (a.nw <= 1 && a.nm <= 3)
    k_pair_ph<R, 1, 3, FROMC><<<grid, 128, 0, st>>>(a);
  else if (a.nw <= 4 && a.nm <= 3)
    k_pair_ph<R, 4, 3, FROMC><<<grid, 128, 0, st>>>(a);
  else if (a.nw <= 8 && a.nm <= 9)
    k_pair_ph<R, 8, 9, FROMC><<<grid, 128, 0, st>>>(a);
  else
    return EPW_ERR_UNSUPPORTED;
  epw_count_launch();
  return EPW_OK;
}

template <typename R>
epw_status launch_pair_ph(const PairArgs &a, int nchunk, cudaStream_t st) {
  if (a.nk <= 0 || a.nq <= 0) return EPW_OK;
  dim3 grid((a.nq + 127) / 128, nchunk);
  if (a.Cq) {
    if constexpr (sizeof(R) == sizeof(float)) return ph_dispatch<float, true>(a, grid, st);
    return EPW_ERR_UNSUPPORTED;
  }
  return ph_dispatch<R, false>(a, grid, st);
}
template epw_status launch_pair_ph<double>(const PairArgs &, int, cudaStream_t);
template epw_status launch_pair_ph<float>(const PairArgs &, int, cudaStream_t);

void launch_ph_finalize(int nq, int nm, int nchunk, const double *partial, const double *omegaT, double omega_min,
                        const double *dos, double *pi_im, double *lam, double *zeta, cudaStream_t st) {
  if (nq <= 0) return;
  k_ph_finalize<<<(nq + 127) / 128, 128, 0, st>>>(nq, nm, nchunk, partial, omegaT, omega_min, dos, pi_im, lam, zeta);
  epw_count_launch();
}

void launch_dos_terms(int nk, int nw, const double *epsk, const double *wk, double EF, double sigma, double *terms,
                      cudaStream_t st) {
  if (nk <= 0) return;
  k_dos_terms<<<(nk + 127) / 128, 128, 0, st>>>(nk, nw, epsk, wk, EF, sigma, terms);
  epw_count_launch();
}

template <typename R, bool FROMC>
static epw_status se_dispatch(const PairArgs &a, dim3 grid, int nom, const double *omega, double delta, double2 *out,
                              cudaStream_t st) {
  if (a.nw <= 1 && a.nm <= 3)
    k_pair_se<R, 1, 3, FROMC><<<grid, 128, 0, st>>>(a, nom, omega, delta, out);
  else if (a.nw <= 4 && a.nm <= 3)
    k_pair_se<R, 4, 3, FROMC><<<grid, 128, 0, st>>>(a, nom, omega, delta, out);
  else if (a.nw <= 8 && a.nm <= 9)
    k_pair_se<R, 8, 9, FROMC><<<grid, 128, 0, st>>>(a, nom, omega, delta, out);
  else
    return EPW_ERR_UNSUPPORTED;
  epw_count_launch();
  return EPW_OK;
}

template <typename R>
epw_status launch_pair_se(const PairArgs &a, int nom, const double *omega, double delta, double2 *out,
                          cudaStream_t st) {
  if (a.nk <= 0 || a.nq <= 0) return EPW_OK;
  dim3 grid((a.nq + 127) / 128, a.nk);
  if (a.Cq) {
    if constexpr (sizeof(R) == sizeof(float)) return se_dispatch<float, true>(a, grid, nom, omega, delta, out, st);
    return EPW_ERR_UNSUPPORTED;
  }
  return se_dispatch<R, false>(a, grid, nom, omega, delta, out, st);
}
template epw_status launch_pair_se<double>(const PairArgs &, int, const double *, double, double2 *, cudaStream_t);
template epw_status launch_pair_se<float>(const PairArgs &, int, const double *, double, double2 *, cudaStream_t);

void launch_se_finalize(int nkc, int k0, int nw, int nqw, int nom, const double2 *part, const double *omega,
                        const double *epsk, double EF, double2 *sig, double *spec, cudaStream_t st) {
  const int n = nkc * nw;
  if (n <= 0) return;
  const int bs = nom + 1 <= 64 ? 64 : nom + 1 <= 128 ? 128 : 256;
  k_se_finalize<<<n, bs, 0, st>>>(nkc, k0, nw, nqw, nom, part, omega, epsk, EF, sig, spec);
  epw_count_launch();
}

template <typename R>
void launch_polar_factors(const epw_model *m, int nq, const double *q, const cx<R> *ET, cx<R> *C, cudaStream_t st) {
  if (nq <= 0 || !m->polar) return;
  PolarK pk;
  for (int i = 0; i < 9; i++) {
    pk.b[i] = m->pb[i];
    pk.eps[i] = m->peps[i];
  }
  pk.alpha = m->palpha;
  pk.pref = m->ppref;
  pk.gmax = m->pgmax;
  k_polar_factors<R><<<(nq + 127) / 128, 128, 0, st>>>(nq, m->nm, m->nat, q, pk, m->pZ, ET, C);
  epw_count_launch();
}
template void launch_polar_factors<double>(const epw_model *, int, const double *, const cx<double> *, cx<double> *,
                                           cudaStream_t);
template void launch_polar_factors<float>(const epw_model *, int, const double *, const cx<float> *, cx<float> *,
                                          cudaStream_t);

void launch_eliashberg(int nq, int nm, const double *omega, const double *lam, const double *wq, int ngrid,
                       const double *grid, double sigma_ph, double *a2f, cudaStream_t st) {
  if (ngrid <= 0) return;
  k_eliashberg<<<ngrid, 256, 0, st>>>(nq, nm, omega, lam, wq, grid, sigma_ph, a2f);
  epw_count_launch();
}

void launch_set_vertex(const epw_model *m, const void *g, int is_c64, cudaStream_t st) {
  size_t per = (size_t)m->nm * m->nw * m->nw;
  size_t n = (size_t)m->nRe * m->nRp * per;
  if (!n) return;
  k_set_vertex<<<nblocks(n, 256), 256, 0, st>>>(m->nRe, m->nRp, per, g, is_c64, m->wRe, m->wRp, m->gw);
  epw_count_launch();
}

void launch_finalize(int nk, int nqb, int nw, const double *partial, double *out, cudaStream_t st) {
  int n = nk * nw;  // one warp each
  if (!n) return;
  if (32 % nw == 0)
    k_finalize_k<<<nk, 128, 0, st>>>(nk, nqb, nw, partial, out);
  else
    k_finalize<<<(n + 3) / 4, 128, 0, st>>>(nk, nqb, nw, partial, out);
  epw_count_launch();
}

void launch_sum_scalar(int n, const double *partial, double scale, double *out, cudaStream_t st) {
  k_sum_scalar<<<1, 256, 0, st>>>(n, partial, scale, out);
  epw_count_launch();
}

template <typename R>
void launch_bg_adjoint_rotate_k0(int nk, int k0, int nRp, int nm, int nw, const cx<R> *Bbar, const cx<double> *Uk,
                                 cx<R> *G1bar, cudaStream_t st) {
  size_t n = (size_t)nk * nRp * nm * nw * nw;
  if (!n) return;
  k_bg_adjoint_rotate<R><<<nblocks(n, 256), 256, 0, st>>>(nk, k0, nRp, nm, nw, Bbar, Uk, G1bar);
  epw_count_launch();
}
template void launch_bg_adjoint_rotate_k0<double>(int, int, int, int, int, const cx<double> *, const cx<double> *,
                                                  cx<double> *, cudaStream_t);
template void launch_bg_adjoint_rotate_k0<float>(int, int, int, int, int, const cx<float> *, const cx<double> *,
                                                 cx<float> *, cudaStream_t);

template <typename R>
void launch_dg_scale(const epw_model *m, const cx<R> *gwbar, double *dg, bool accumulate, cudaStream_t st) {
  size_t per = (size_t)m->nm * m->nw * m->nw;
  size_t n = (size_t)m->nRe * m->nRp * per;
  if (!n) return;
  k_dg_scale<R><<<nblocks(n, 256), 256, 0, st>>>(m->nRe, m->nRp, per, m->wRe, m->wRp, gwbar, dg, accumulate);
  epw_count_launch();
}
template void launch_dg_scale<double>(const epw_model *, const cx<double> *, double *, bool, cudaStream_t);
template void launch_dg_scale<float>(const epw_model *, const cx<float> *, double *, bool, cudaStream_t);
