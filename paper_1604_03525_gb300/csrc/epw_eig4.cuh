// FP32 Hermitian eigensolvers of small matrices in registers, one matrix per
// thread: complex cyclic Jacobi for N < 4 and, for N = 4, two Householder
// reflectors to a real tridiagonal matrix followed by real Jacobi sweeps.  The
// sweeps exit when every lane of the warp has converged (a warp vote), so every
// lane of the warp must make the call.
#pragma once
#include "epw_internal.cuh"

namespace {

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------- FP32 Jacobi (epilogue)
// Hermitian N x N in registers, upper triangle stored (A[i][j], i < j; the
// diagonal's real part).  One rotation of the (p,q) plane, parameters without
// a division by |a_pq| (branch-free, so a zero a_pq gives the identity):
//   d = a_qq - a_pp,  den = |d| + sqrt(d^2 + 4|a_pq|^2),  t = 2|a_pq| sgn(d) / den,
//   c = 1/sqrt(1+t^2),  s e = 2 sgn(d) c a_pq / den,  a_pp -= t|a_pq|,  a_qq += t|a_pq|.
template <int N>
struct Herm {
  cx<float> a[N][N];  // only i < j used, plus a[i][i].x
  __device__ __forceinline__ cx<float> get(int i, int j) const { return i < j ? a[i][j] : conjc(a[j][i]); }
  __device__ __forceinline__ void set(int i, int j, cx<float> v) {
    if (i < j)
      a[i][j] = v;
    else
      a[j][i] = conjc(v);
  }
};

struct Rot {
  float c, tb;
  cx<float> se;
};

template <int N>
__device__ __forceinline__ Rot rot_params(const Herm<N> &H, int p, int q) {
  const cx<float> apq = H.a[p][q];
  const float d = H.a[q][q].x - H.a[p][p].x;
  const float m2 = fmaf(apq.x, apq.x, apq.y * apq.y);
  const float x = fmaf(d, d, 4.0f * m2);
  // hardware approximations refined by one Newton step each (to ~1 ulp), so
  // that the rotation stays unitary and consistent with the diagonal update
  const float xs = fmaxf(x, 1e-37f);
  float ri = rsqrt_approx(xs);
  ri = ri * fmaf(-0.5f * xs * ri, ri, 1.5f);
  const float sq = x * ri;
  const float den = fmaxf(fabsf(d) + sq, 1e-30f);
  float rden = rcp_approx(den);
  rden = rden * fmaf(-den, rden, 2.0f);
  const float sg = d >= 0.0f ? 2.0f : -2.0f;
  const float tmag = 2.0f * m2 * rden;  // |t| |a_pq|
  const float t2 = tmag * (2.0f * rden);
  Rot r;
  const float u = 1.0f + t2;
  float c = rsqrt_approx(u);
  r.c = c * fmaf(-0.5f * u * c, c, 1.5f);
  r.tb = 0.5f * sg * tmag;
  const float kap = sg * rden * r.c;
  r.se = mkc(kap * apq.x, kap * apq.y);
  return r;
}

template <int N>
__device__ __forceinline__ void rot_apply(Herm<N> &H, cx<float> (&V)[N][N], int p, int q, const Rot &r) {
  H.a[p][p].x -= r.tb;
  H.a[q][q].x += r.tb;
  H.a[p][q] = mkc(0.0f, 0.0f);
  const cx<float> sec = conjc(r.se);
#pragma unroll
  for (int k = 0; k < N; k++) {
    if (k == p || k == q) continue;
    const cx<float> akp = H.get(k, p), akq = H.get(k, q);
    cx<float> nkp = mkc(r.c * akp.x, r.c * akp.y);
    cx<float> nkq = mkc(r.c * akq.x, r.c * akq.y);
    cfma(nkp, mkc(-sec.x, -sec.y), akq);
    cfma(nkq, r.se, akp);
    H.set(k, p, nkp);
    H.set(k, q, nkq);
  }
#pragma unroll
  for (int k = 0; k < N; k++) {
    const cx<float> vp = V[k][p], vq = V[k][q];
    cx<float> np = mkc(r.c * vp.x, r.c * vp.y);
    cx<float> nq = mkc(r.c * vq.x, r.c * vq.y);
    cfma(np, mkc(-sec.x, -sec.y), vq);
    cfma(nq, r.se, vp);
    V[k][p] = np;
    V[k][q] = nq;
  }
}

template <int N>
__device__ __forceinline__ float offdiag_frac(const Herm<N> &H) {
  float off = 0.0f, dg = 0.0f;
#pragma unroll
  for (int i = 0; i < N; i++) {
    dg = fmaf(H.a[i][i].x, H.a[i][i].x, dg);
#pragma unroll
    for (int j = i + 1; j < N; j++) off += cabs2(H.a[i][j]);
  }
  return off / fmaxf(dg + 2.0f * off, 1e-37f);
}

// ---------------------------------------------- 4 x 4: tridiagonal, then real
// Two Householder reflectors reduce the Hermitian A to a tridiagonal matrix
// with complex off-diagonals t_i, and a diagonal phase D (phi_0 = 1,
// phi_i = phi_{i-1} t_i / |t_i|) makes them real: A = Z T Z^dagger with
// Z = P1 P2 D unitary and T real symmetric.  Jacobi then runs on T with real
// rotations, accumulated into Z: a real rotation costs about a third of a
// complex one on the matrix and two thirds on the eigenvectors.
struct RotR {
  float c, s, tb;
};

// Rotation of the (p,q) plane of a real symmetric matrix zeroing a_pq, from the
// half-angle formulas: d = a_qq - a_pp, r = sqrt(d^2 + 4 a_pq^2), cos 2t = |d|/r
// (1 when r = 0), c^2 = (1 + cos 2t)/2, s = sgn(d) a_pq/(r c) (= sin 2t/(2c)), and
// the diagonal moves by t a_pq = sgn(d) a_pq^2/(r c^2): a_pp -= t a_pq, a_qq += t a_pq.
// (The same rotation as t = 2 a_pq sgn(d)/(|d| + r), c = 1/sqrt(1+t^2), s = t c,
// with two reciprocal square roots and no division.)
__device__ __forceinline__ RotR rotr_params(float app, float aqq, float apq) {
  const float d = aqq - app;
  const float x = fmaf(d, d, 4.0f * apq * apq);
  const float xs = fmaxf(x, 1e-37f);
  float ri = rsqrt_approx(xs);
  ri = ri * fmaf(-0.5f * xs * ri, ri, 1.5f);  // 1/r
  const float cos2 = x > 0.0f ? fabsf(d) * ri : 1.0f;
  const float u = fmaf(0.5f, cos2, 0.5f);      // c^2, in [1/2, 1]
  float ru = rsqrt_approx(u);
  ru = ru * fmaf(-0.5f * u * ru, ru, 1.5f);    // 1/c
  const float sa = (d >= 0.0f ? apq : -apq) * ri;  // sin 2t / 2
  RotR r;
  r.c = u * ru;
  r.s = sa * ru;
  r.tb = sa * apq * (ru * ru);
  return r;
}

// S: upper triangle of the real symmetric matrix (S[i][j], i < j) and its diagonal.
template <int P, int Q>
__device__ __forceinline__ void rotr_apply(float (&S)[4][4], cx<float> (&V)[4][4], const RotR &r) {
  S[P][P] -= r.tb;
  S[Q][Q] += r.tb;
  S[P][Q] = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (k == P || k == Q) continue;
    float &skp = k < P ? S[k][P] : S[P][k];
    float &skq = k < Q ? S[k][Q] : S[Q][k];
    const float a = skp, b = skq;
    skp = r.c * a - r.s * b;
    skq = fmaf(r.s, a, r.c * b);
  }
  // eigenvector columns: (re, im) of each entry as one packed pair
  const float2 c2 = make_float2(r.c, r.c), s2 = make_float2(r.s, r.s), ns2 = make_float2(-r.s, -r.s);
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const float2 vp = make_float2(V[k][P].x, V[k][P].y), vq = make_float2(V[k][Q].x, V[k][Q].y);
    const float2 np = __ffma2_rn(ns2, vq, __fmul2_rn(c2, vp)), nq = __ffma2_rn(s2, vp, __fmul2_rn(c2, vq));
    V[k][P] = mkc(np.x, np.y);
    V[k][Q] = mkc(nq.x, nq.y);
  }
}

// Householder vector of x = (x_0, rest) with |rest|^2 = srest: v = (phi (|x_0| + |x|), rest),
// P = I - tau v v^dagger maps x to (-phi |x|, 0...), phi = x_0 / |x_0| (1 when x_0 = 0).
// With rest = 0 no reflection is needed: tau = 0 and the entry stays x_0.
struct Hh {
  cx<float> v0, beta;
  float tau;
};
// 1/sqrt(x) and 1/x from the hardware approximations with one Newton step (~1 ulp)
__device__ __forceinline__ float rsqrt_nr(float x) {
  float r = rsqrt_approx(x);
  return r * fmaf(-0.5f * x * r, r, 1.5f);
}
__device__ __forceinline__ float rcp_nr(float x) {
  float r = rcp_approx(x);
  return r * fmaf(-x, r, 2.0f);
}

// Fermi-Dirac occupation as fermi_f, with the reciprocal from rcp.approx and one
// Newton step instead of an IEEE division.
__device__ __forceinline__ float fermi_fast(float d, float invkT) {
  if (invkT <= 0.0f) return d < 0.0f ? 1.0f : (d > 0.0f ? 0.0f : 0.5f);
  const float x = d * invkT;
  const float t = __expf(-fabsf(x));
  const float r = rcp_nr(1.0f + t);
  return x > 0.0f ? t * r : r;
}

__device__ __forceinline__ Hh householder(cx<float> x0, float srest) {
  const float n0sq = cabs2(x0);
  const float tot = n0sq + srest;
  const float rn0 = rsqrt_nr(fmaxf(n0sq, 1e-37f));
  const float n0 = n0sq * rn0;
  const float al = tot * rsqrt_nr(fmaxf(tot, 1e-37f));
  const cx<float> ph = n0sq > 0.0f ? mkc(x0.x * rn0, x0.y * rn0) : mkc(1.0f, 0.0f);
  Hh h;
  const bool refl = srest > 0.0f;
  h.tau = refl ? rcp_nr(al * (al + n0)) : 0.0f;
  h.v0 = mkc(ph.x * (n0 + al), ph.y * (n0 + al));
  h.beta = refl ? mkc(-ph.x * al, -ph.y * al) : x0;
  return h;
}

__device__ __forceinline__ cx<float> cmul_conjb(cx<float> a, cx<float> b) {  // a conj(b)
  return mkc(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

__device__ __forceinline__ bool eig_herm4(Herm<4> &H, cx<float> (&V)[4][4]) {
  // reflector 1 on rows/columns 1..3: zero A[2][0], A[3][0]
  const cx<float> x1 = conjc(H.a[0][1]), x2 = conjc(H.a[0][2]), x3 = conjc(H.a[0][3]);
  const Hh h1 = householder(x1, cabs2(x2) + cabs2(x3));
  const cx<float> v[3] = {h1.v0, x2, x3};
  cx<float> B[3][3];  // A[1..3][1..3], full
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) B[i][j] = i == j ? mkc(H.a[1 + i][1 + i].x, 0.0f) : H.get(1 + i, 1 + j);
  {
    cx<float> p[3];
    float vp = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      cx<float> s = mkc(0.0f, 0.0f);
#pragma unroll
      for (int j = 0; j < 3; j++) cfma(s, B[i][j], v[j]);
      p[i] = mkc(h1.tau * s.x, h1.tau * s.y);
      vp = fmaf(v[i].x, p[i].x, fmaf(v[i].y, p[i].y, vp));  // Re(conj(v) p)
    }
    const float K = 0.5f * h1.tau * vp;
    cx<float> w[3];
#pragma unroll
    for (int i = 0; i < 3; i++) w[i] = mkc(p[i].x - K * v[i].x, p[i].y - K * v[i].y);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = i; j < 3; j++) {
        const cx<float> a = cmul_conjb(v[i], w[j]), b = cmul_conjb(w[i], v[j]);
        B[i][j] = mkc(B[i][j].x - a.x - b.x, i == j ? 0.0f : B[i][j].y - a.y - b.y);
      }
  }
  // reflector 2 on rows/columns 2..3: zero A[3][1]
  const cx<float> y1 = conjc(B[0][1]), y2 = conjc(B[0][2]);
  const Hh h2 = householder(y1, cabs2(y2));
  const cx<float> u[2] = {h2.v0, y2};
  cx<float> C00 = mkc(B[1][1].x, 0.0f), C01 = B[1][2], C11 = mkc(B[2][2].x, 0.0f);
  {
    const cx<float> C10 = conjc(C01);
    cx<float> p0 = mkc(0.0f, 0.0f), p1 = mkc(0.0f, 0.0f);
    cfma(p0, C00, u[0]);
    cfma(p0, C01, u[1]);
    cfma(p1, C10, u[0]);
    cfma(p1, C11, u[1]);
    p0 = mkc(h2.tau * p0.x, h2.tau * p0.y);
    p1 = mkc(h2.tau * p1.x, h2.tau * p1.y);
    const float vp = u[0].x * p0.x + u[0].y * p0.y + u[1].x * p1.x + u[1].y * p1.y;
    const float K = 0.5f * h2.tau * vp;
    const cx<float> w0 = mkc(p0.x - K * u[0].x, p0.y - K * u[0].y), w1 = mkc(p1.x - K * u[1].x, p1.y - K * u[1].y);
    C00.x -= 2.0f * (u[0].x * w0.x + u[0].y * w0.y);
    C11.x -= 2.0f * (u[1].x * w1.x + u[1].y * w1.y);
    const cx<float> a = cmul_conjb(u[0], w1), b = cmul_conjb(w0, u[1]);
    C01 = mkc(C01.x - a.x - b.x, C01.y - a.y - b.y);
  }
  // T: diagonal d, complex subdiagonal t1, t2, t3
  const cx<float> t1 = h1.beta, t2 = h2.beta, t3 = conjc(C01);
  float S[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) S[i][j] = 0.0f;
  S[0][0] = H.a[0][0].x;
  S[1][1] = B[0][0].x;
  S[2][2] = C00.x;
  S[3][3] = C11.x;
  // phases: phi_i = phi_{i-1} t_i / |t_i|, real subdiagonal |t_i|
  cx<float> phi[4];
  phi[0] = mkc(1.0f, 0.0f);
  {
    const cx<float> t[3] = {t1, t2, t3};
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const float m2 = cabs2(t[i]);
      const float rm = rsqrt_nr(fmaxf(m2, 1e-37f));
      const float m = m2 * rm;
      const cx<float> e = m2 > 0.0f ? mkc(t[i].x * rm, t[i].y * rm) : mkc(1.0f, 0.0f);
      phi[i + 1] = mkc(phi[i].x * e.x - phi[i].y * e.y, phi[i].x * e.y + phi[i].y * e.x);
      S[i][i + 1] = m;
    }
  }
  // Z = P1 P2 D:  P1 = I - tau1 v v^dagger on 1..3, P2 = I - tau2 u u^dagger on 2..3
  cx<float> P1[3][3];
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const cx<float> a = cmul_conjb(v[i], v[j]);
      P1[i][j] = mkc((i == j ? 1.0f : 0.0f) - h1.tau * a.x, -h1.tau * a.y);
    }
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int c = 0; c < 4; c++) V[r][c] = mkc(r == 0 && c == 0 ? 1.0f : 0.0f, 0.0f);
#pragma unroll
  for (int i = 0; i < 3; i++) {
    // column 1 of Q is P1's first column; columns 2, 3 are P1[:,1..2] P2
    const cx<float> q1 = P1[i][0];
    cx<float> s = mkc(0.0f, 0.0f);
    cfma(s, P1[i][1], u[0]);
    cfma(s, P1[i][2], u[1]);
    s = mkc(h2.tau * s.x, h2.tau * s.y);  // tau2 (P1 u)_i
    const cx<float> q2 = mkc(P1[i][1].x - (s.x * u[0].x + s.y * u[0].y), P1[i][1].y - (s.y * u[0].x - s.x * u[0].y));
    const cx<float> q3 = mkc(P1[i][2].x - (s.x * u[1].x + s.y * u[1].y), P1[i][2].y - (s.y * u[1].x - s.x * u[1].y));
    const cx<float> q[3] = {q1, q2, q3};
#pragma unroll
    for (int c = 0; c < 3; c++)
      V[1 + i][1 + c] = mkc(q[c].x * phi[c + 1].x - q[c].y * phi[c + 1].y, q[c].x * phi[c + 1].y + q[c].y * phi[c + 1].x);
  }
  // real Jacobi on S, parallel ordering, warp-uniform exit
  constexpr float TOL2 = 1e-10f;
  constexpr int MAXSWEEP = 12;
  bool conv = false;
  for (int sweep = 0; sweep <= MAXSWEEP; sweep++) {
    float off = 0.0f, dg = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      dg = fmaf(S[i][i], S[i][i], dg);
#pragma unroll
      for (int j = i + 1; j < 4; j++) off = fmaf(S[i][j], S[i][j], off);
    }
    conv = off <= TOL2 * fmaxf(dg + 2.0f * off, 1e-37f);
    if (__all_sync(0xffffffffu, conv) || sweep == MAXSWEEP) break;
    const RotR r01 = rotr_params(S[0][0], S[1][1], S[0][1]), r23 = rotr_params(S[2][2], S[3][3], S[2][3]);
    rotr_apply<0, 1>(S, V, r01);
    rotr_apply<2, 3>(S, V, r23);
    const RotR r02 = rotr_params(S[0][0], S[2][2], S[0][2]), r13 = rotr_params(S[1][1], S[3][3], S[1][3]);
    rotr_apply<0, 2>(S, V, r02);
    rotr_apply<1, 3>(S, V, r13);
    const RotR r03 = rotr_params(S[0][0], S[3][3], S[0][3]), r12 = rotr_params(S[1][1], S[2][2], S[1][2]);
    rotr_apply<0, 3>(S, V, r03);
    rotr_apply<1, 2>(S, V, r12);
  }
#pragma unroll
  for (int i = 0; i < 4; i++) H.a[i][i].x = S[i][i];
  return conv;
}

// Sweeps until every lane of the warp has converged (warp-uniform exit).
// N = 4: tridiagonal reduction, then real Jacobi (above); N < 4: complex
// cyclic Jacobi sweeps until every lane of the warp has converged.
template <int N>
__device__ __forceinline__ bool jacobi_fast(Herm<N> &H, cx<float> (&V)[N][N]) {
  if constexpr (N == 4) {
    return eig_herm4(H, V);
  } else {
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
      for (int j = 0; j < N; j++) V[i][j] = mkc(i == j ? 1.0f : 0.0f, 0.0f);
    if constexpr (N == 1) return true;
    constexpr float TOL2 = 1e-10f;
    constexpr int MAXSWEEP = 12;
    for (int sweep = 0; sweep < MAXSWEEP; sweep++) {
      const bool conv = offdiag_frac(H) <= TOL2;
      if (__all_sync(0xffffffffu, conv)) return true;
#pragma unroll
      for (int p = 0; p < N - 1; p++)
#pragma unroll
        for (int q = p + 1; q < N; q++) {
          const Rot r = rot_params(H, p, q);
          rot_apply(H, V, p, q, r);
        }
    }
    return offdiag_frac(H) <= TOL2;
  }
}

}  // namespace
