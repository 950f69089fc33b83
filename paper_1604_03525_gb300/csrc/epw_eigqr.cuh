// FP32 Hermitian eigensolver of one small matrix per thread (3 <= N <= 8), for
// the per-pair eigensolve of H(k+q) in the wide-shape tensor-core path:
//   1. Householder reduction A = Q T_c Q^dagger, Q = P_0 ... P_{N-3},
//      P_k = I - tau_k v_k v_k^dagger acting on indices k+1..N-1 (reflectors kept);
//   2. a diagonal phase D (phi_0 = 1, phi_{i+1} = phi_i t_i/|t_i|) makes the
//      subdiagonal t_i of T_c real: T = D^dagger T_c D;
//   3. implicit symmetric QR steps with Wilkinson shifts on T (Golub & Van Loan,
//      Sec. 8.3), deflating from the bottom, the Givens rotations accumulated into
//      the real matrix V (T = V Lambda V^T);
//   4. eigenvector m of A on demand: u_m = Q D V e_m.
// Control flow is warp-uniform: the QR loop exits when every lane of the warp has
// converged and each Givens position of a sweep is skipped when no lane of the
// warp needs it, so every lane of the warp must make the calls.
#pragma once
#include "epw_eig4.cuh"
#include "epw_tcgen05.cuh"

namespace {

template <int N>
struct HhQR {
  static_assert(N >= 3 && N <= 8, "3 <= N <= 8");
  static constexpr int NP = (N + 1) / 2;
  float d[N];             // diagonal of T; the eigenvalues (unsorted) after tri_qr
  float e[N - 1];         // subdiagonal of T
  float2 V[NP][N];        // V, rows in pairs: V[r][c] = (V_{2r,c}, V_{2r+1,c}); row N is 0 for odd N
  cx<float> v[N - 2][N - 1];  // reflector k: v[k][i - k - 1], i = k+1..N-1
  float tau[N - 2];
  cx<float> phi[N];
};

// Householder reduction of the Hermitian H (upper triangle and real diagonal used).
template <int N>
__device__ __forceinline__ void hh_tridiag(Herm<N> &H, HhQR<N> &S) {
  cx<float> t[N - 1];  // complex subdiagonal of T_c: t_i = T_c[i+1][i]
#pragma unroll
  for (int k = 0; k < N - 2; k++) {
    // column k below the diagonal: x_i = A[i][k] = conj(A[k][i]), i = k+1..N-1
    float srest = 0.0f;
#pragma unroll
    for (int i = k + 2; i < N; i++) srest += cabs2(H.a[k][i]);
    const Hh h = householder(conjc(H.a[k][k + 1]), srest);
    constexpr int L = N - 1;
    cx<float> v[L], p[L], w[L];
    v[0] = h.v0;
#pragma unroll
    for (int i = k + 2; i < N; i++) v[i - k - 1] = conjc(H.a[k][i]);
    // p = tau B v on the trailing block B = A[k+1.., k+1..]; K = tau/2 Re(v^dagger p)
    float vp = 0.0f;
#pragma unroll
    for (int i = k + 1; i < N; i++) {
      cx<float> s = mkc(0.0f, 0.0f);
#pragma unroll
      for (int j = k + 1; j < N; j++) {
        const cx<float> bij = i == j ? mkc(H.a[i][i].x, 0.0f) : H.get(i, j);
        cfma(s, bij, v[j - k - 1]);
      }
      const int ii = i - k - 1;
      p[ii] = mkc(h.tau * s.x, h.tau * s.y);
      vp = fmaf(v[ii].x, p[ii].x, fmaf(v[ii].y, p[ii].y, vp));
    }
    const float K = 0.5f * h.tau * vp;
#pragma unroll
    for (int i = 0; i < N - k - 1; i++) w[i] = mkc(p[i].x - K * v[i].x, p[i].y - K * v[i].y);
    // B <- P B P = B - v w^dagger - w v^dagger (upper triangle, real diagonal)
#pragma unroll
    for (int i = k + 1; i < N; i++)
#pragma unroll
      for (int j = i; j < N; j++) {
        const int ii = i - k - 1, jj = j - k - 1;
        const cx<float> x1 = cmul_conjb(v[ii], w[jj]), x2 = cmul_conjb(w[ii], v[jj]);
        if (i == j)
          H.a[i][i].x -= x1.x + x2.x;
        else
          H.a[i][j] = mkc(H.a[i][j].x - x1.x - x2.x, H.a[i][j].y - x1.y - x2.y);
      }
    S.tau[k] = h.tau;
#pragma unroll
    for (int i = 0; i < N - k - 1; i++) S.v[k][i] = v[i];
    t[k] = h.beta;
  }
  t[N - 2] = conjc(H.a[N - 2][N - 1]);
#pragma unroll
  for (int i = 0; i < N; i++) S.d[i] = H.a[i][i].x;
  S.phi[0] = mkc(1.0f, 0.0f);
#pragma unroll
  for (int i = 0; i < N - 1; i++) {
    const float m2 = cabs2(t[i]);
    const float rm = rsqrt_nr(fmaxf(m2, 1e-37f));
    const cx<float> ph = m2 > 0.0f ? mkc(t[i].x * rm, t[i].y * rm) : mkc(1.0f, 0.0f);
    S.phi[i + 1] = mkc(S.phi[i].x * ph.x - S.phi[i].y * ph.y, S.phi[i].x * ph.y + S.phi[i].y * ph.x);
    S.e[i] = m2 * rm;
  }
}

// Implicit QR steps on (d, e) with Wilkinson shifts, rotations into V (set to I
// here).  A subdiagonal entry below tol = 2^-22 max(|d|, |e|) is set to zero;
// the active block is the bottom unreduced one [l, h].  Returns false when
// maxit steps were not enough.
template <int N>
__device__ __forceinline__ bool tri_qr(HhQR<N> &S) {
  constexpr int NP = HhQR<N>::NP;
  constexpr int MAXIT = 6 * N;
#pragma unroll
  for (int r = 0; r < NP; r++)
#pragma unroll
    for (int c = 0; c < N; c++) S.V[r][c] = make_float2(2 * r == c ? 1.0f : 0.0f, 2 * r + 1 == c ? 1.0f : 0.0f);
  float scale = 0.0f;
#pragma unroll
  for (int i = 0; i < N; i++) scale = fmaxf(scale, fabsf(S.d[i]));
#pragma unroll
  for (int i = 0; i < N - 1; i++) scale = fmaxf(scale, fabsf(S.e[i]));
  const float tol = 2.384185791015625e-07f * scale;
  bool conv = false;
  for (int it = 0; it <= MAXIT; it++) {
    int h = 0;
#pragma unroll
    for (int i = 0; i < N - 1; i++) {
      if (fabsf(S.e[i]) <= tol) S.e[i] = 0.0f;
      if (S.e[i] != 0.0f) h = i + 1;
    }
    conv = h == 0;
    if (__all_sync(0xffffffffu, conv) || it == MAXIT) break;
    int l = 0;
#pragma unroll
    for (int i = 0; i < N - 1; i++)
      if (i < h && S.e[i] == 0.0f) l = i + 1;
    // Wilkinson shift from the trailing 2 x 2 block [[a, b], [b, c]] of [l, h]
    // (entries picked by 0/1 weights: a plain select at a runtime index becomes an
    // indexed access that moves the arrays to local memory)
    float a = 0.0f, c = 0.0f, b = 0.0f, x = 0.0f, z = 0.0f;
#pragma unroll
    for (int i = 0; i < N - 1; i++) {
      const float w = i == h - 1 ? 1.0f : 0.0f;
      a = fmaf(w, S.d[i], a);
      c = fmaf(w, S.d[i + 1], c);
      b = fmaf(w, S.e[i], b);
    }
    const float del = 0.5f * (a - c);
    const float rr = sqrtf(fmaf(del, del, b * b));
    const float den = del >= 0.0f ? del + rr : del - rr;
    const float mu = den != 0.0f ? c - b * (b / den) : c;
#pragma unroll
    for (int i = 0; i < N - 1; i++) {
      const float w = i == l ? 1.0f : 0.0f;
      x = fmaf(w, S.d[i] - mu, x);
      z = fmaf(w, S.e[i], z);
    }
    // bulge chase over the Givens positions k = l..h-1 (T <- G^T T G, G = [[c, s], [-s, c]])
#pragma unroll
    for (int k = 0; k < N - 1; k++) {
      const bool act = !conv && k >= l && k < h;
      if (__any_sync(0xffffffffu, act)) {
        const float r2 = fmaf(x, x, z * z);
        const float ri = rsqrt_nr(fmaxf(r2, 1e-37f));
        const bool rot = act && r2 > 0.0f;
        const float cg = rot ? x * ri : 1.0f, sg = rot ? -z * ri : 0.0f;
        if (k > 0) {
          if (rot && k > l) S.e[k - 1] = r2 * ri;
        }
        const float ak = S.d[k], bk = S.d[k + 1], ok = S.e[k];
        const float cc = cg * cg, ss = sg * sg, cs = cg * sg;
        S.d[k] = fmaf(cc, ak, fmaf(-2.0f * cs, ok, ss * bk));
        S.d[k + 1] = fmaf(ss, ak, fmaf(2.0f * cs, ok, cc * bk));
        S.e[k] = fmaf(cs, ak - bk, (cc - ss) * ok);
        if (k + 1 < N - 1) {
          const float en = S.e[k + 1];
          if (rot && k + 1 < h) {
            z = -sg * en;
            S.e[k + 1] = cg * en;
            x = S.e[k];
          }
        }
        const float2 c2 = bc2(cg), s2 = bc2(sg), ns2 = bc2(-sg);
#pragma unroll
        for (int r = 0; r < NP; r++) {
          const float2 vk = S.V[r][k], vk1 = S.V[r][k + 1];
          S.V[r][k] = ffma2(ns2, vk1, fmul2(c2, vk));
          S.V[r][k + 1] = ffma2(s2, vk, fmul2(c2, vk1));
        }
      }
    }
  }
  return conv;
}

// Eigenvector m of A: u = Q D V e_m (reflectors applied last to first).  m is a
// runtime index: column m of V is picked with 0/1 weights, so that the code is
// one loop body (instruction cache) and V stays in registers.
template <int N>
__device__ __forceinline__ void hh_vector(const HhQR<N> &S, int m, cx<float> (&u)[N]) {
  float y[N];
#pragma unroll
  for (int i = 0; i < N; i++) y[i] = 0.0f;
#pragma unroll
  for (int c = 0; c < N; c++) {
    const float w = c == m ? 1.0f : 0.0f;
#pragma unroll
    for (int i = 0; i < N; i++) y[i] = fmaf(w, (i & 1) ? S.V[i >> 1][c].y : S.V[i >> 1][c].x, y[i]);
  }
#pragma unroll
  for (int i = 0; i < N; i++) u[i] = mkc(S.phi[i].x * y[i], S.phi[i].y * y[i]);
#pragma unroll
  for (int k = N - 3; k >= 0; k--) {
    cx<float> s = mkc(0.0f, 0.0f);
#pragma unroll
    for (int i = k + 1; i < N; i++) {
      const cx<float> vi = S.v[k][i - k - 1];
      s = mkc(fmaf(vi.x, u[i].x, fmaf(vi.y, u[i].y, s.x)), fmaf(vi.x, u[i].y, fmaf(-vi.y, u[i].x, s.y)));
    }
    s = mkc(S.tau[k] * s.x, S.tau[k] * s.y);
#pragma unroll
    for (int i = k + 1; i < N; i++) {
      const cx<float> vi = S.v[k][i - k - 1];
      u[i] = mkc(u[i].x - fmaf(vi.x, s.x, -vi.y * s.y), u[i].y - fmaf(vi.x, s.y, vi.y * s.x));
    }
  }
}

// d[m] at a runtime index, by 0/1 weights
template <int N>
__device__ __forceinline__ float pick(const float (&d)[N], int m) {
  float r = 0.0f;
#pragma unroll
  for (int i = 0; i < N; i++) r = fmaf(i == m ? 1.0f : 0.0f, d[i], r);
  return r;
}

}  // namespace
