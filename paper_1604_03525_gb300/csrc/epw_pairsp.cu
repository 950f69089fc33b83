// Per-pair linewidth terms for the staged shapes beyond the register-tile kernel
// (nw up to 18 Wannier functions, up to 18 modes), FP32, from the staged tensor-core
// contraction [H(k+q) | X_a = g_a(k,q) U_k] (q-major rows).  One warp per (k, q) pair:
//   1. Householder reduction of the Hermitian H(k+q) = Q T_c Q^dagger, lanes over rows
//      (p = tau B v and the rank-2 update B - v w^dagger - w v^dagger in parallel),
//      the reflectors kept in shared memory; a diagonal phase D makes T = D^dagger T_c D
//      real (as in the per-thread solver of the wide fused kernel);
//   2. implicit symmetric QR steps with Wilkinson shifts on T (Golub & Van Loan, Sec.
//      8.3): every lane runs the same scalar recurrence, lane r applies each Givens
//      rotation to row r of V (T = V Lambda V^T);
//   3. the eigenvectors some band n at k can reach, u_m = Q D V e_m, lane m forming u_m;
//   4. only the (m, n) terms of Eq. (linewidthel) whose Gaussians are not below the
//      cutoff (|e_nk - e_mk+q| <= max kept w_q,nu + X sigma, X = sqrt(130 ln 2): every
//      skipped Gaussian is below 1e-39 of its peak), one term per lane:
//        t_a = u_m^dagger X_a[:, n],  g_nu = sum_a E_q[a][nu] t_a,
//      then |g_nu|^2 times the occupation-weighted Gaussians, summed over nu.
// A block of 4 warps covers 128 consecutive q of one k, each warp 32 of them in order;
// each band's sum over m is formed in ascending m and over q in ascending q, so the
// per-(k, q-tile) partial sums are deterministic.
#include "epw_internal.cuh"

namespace {

constexpr int SP_WARPS = 4;
constexpr int SP_MMAX = 18;  // modes
constexpr float SP_CUT = 9.4921453036541f;  // sqrt(130 ln 2)

__device__ __forceinline__ float sp_wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// 1/sqrt(x) from the hardware approximation with one Newton step
__device__ __forceinline__ float sp_rsqrt(float x) {
  const float r = rsqrtf(x);
  return r * fmaf(-0.5f * x * r, r, 1.5f);
}
__device__ __forceinline__ float sp_wmax(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Shared memory of one warp (W: largest nw of the instantiation).
template <int W>
struct SpWarp {
  cx<float> A[W * W];     // H(k+q) during the reduction; then V^T (floats); then X_a
  cx<float> Ref[W * W];   // reflector k at Ref[k W + i], i = k+1..n-1; then the term sums
  cx<float> U[W * W];     // eigenvector m at U[i W + m]
  cx<float> E[SP_MMAX * SP_MMAX];  // mode factors of this q, E[a][nu]
  cx<float> w[W];         // Householder: p - K v
  cx<float> phi[W];       // diagonal phases
  float tau[W];
  float om[SP_MMAX], nb[SP_MMAX];  // kept frequencies and Bose factors of this q
  float em[W], ek[W];              // eigenvalues at k+q (unsorted), band energies at k
  unsigned char tm[W * W], tn[W * W];  // the term list (m, n)
};

// Householder vector of x = (x_0, rest), |rest|^2 = srest: v = (phi (|x_0| + |x|), rest),
// P = I - tau v v^dagger maps x to (-phi |x|, 0, ...); tau = 0 (no reflection) when rest = 0.
__device__ __forceinline__ void sp_householder(cx<float> x0, float srest, cx<float> &v0, cx<float> &beta,
                                               float &tau) {
  const float n0sq = cabs2(x0);
  const float tot = n0sq + srest;
  const float n0 = sqrtf(n0sq), al = sqrtf(tot);
  const cx<float> ph = n0sq > 0.0f ? mkc(x0.x / n0, x0.y / n0) : mkc(1.0f, 0.0f);
  const bool refl = srest > 0.0f;
  tau = refl ? 1.0f / (al * (al + n0)) : 0.0f;
  v0 = mkc(ph.x * (n0 + al), ph.y * (n0 + al));
  beta = refl ? mkc(-ph.x * al, -ph.y * al) : x0;
}


template <int W>
__global__ void __launch_bounds__(SP_WARPS * 32) k_pair_sparse(PairArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double nsum[SP_WARPS][W];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  SpWarp<W> &S = reinterpret_cast<SpWarp<W> *>(smraw)[warp];
  const int n = a.nw, nm = a.nm, nq = a.nq, nn2 = n * n;
  const int kl = blockIdx.y, k = a.k0 + kl;
  const float inv_sigma = (float)(1.0 / a.sigma);
  const float gnorm = (float)(1.0 / (a.sigma * 1.7724538509055160273));
  const float cut = SP_CUT * (float)a.sigma;
  const cx<float> *ET = (const cx<float> *)a.ET;
  if (lane < n) S.ek[lane] = (float)a.eps_k[(size_t)k * n + lane];
  double accn = 0.0;  // lane n: this warp's sum for band n
  for (int it_q = 0; it_q < 32; it_q++) {
    const int q = blockIdx.x * (SP_WARPS * 32) + warp * 32 + it_q;
    if (q >= nq) break;
    const float *C = a.Cq + (size_t)q * a.ldc + (size_t)kl * a.cpk;
    // H(k+q): Hermitian part of the contraction
    for (int e = lane; e < nn2; e += 32) {
      const int r = e / n, c = e - r * n;
      const float xr = C[2 * e], xi = C[2 * e + 1], yr = C[2 * (c * n + r)], yi = C[2 * (c * n + r) + 1];
      S.A[r * W + c] = mkc(0.5f * (xr + yr), r == c ? 0.0f : 0.5f * (xi - yi));
    }
    // modes of this q: kept frequencies, Bose factors, the cutoff, the mode factors
    float wl = -1.0f;
    bool keep = false;
    if (lane < nm) {
      const float w = (float)a.omegaT[(size_t)lane * nq + q];
      keep = (w >= (float)a.omega_min) && (w > 0.0f);
      S.om[lane] = w;
      S.nb[lane] = keep ? occ_bose<float>(w, a.T) : 0.0f;
      wl = keep ? w : -1.0f;
    }
    const unsigned keepmask = __ballot_sync(0xffffffffu, keep);
    const float wmax = sp_wmax(wl);
    const float thr = wmax >= 0.0f ? wmax + cut : -1.0f;
    for (int e = lane; e < nm * nm; e += 32) S.E[e] = ET[(size_t)e * nq + q];
    __syncwarp();

    // 1. Householder reduction, lanes over rows i = kk+1..n-1 of the trailing block
#pragma unroll 1
    for (int kk = 0; kk < n - 2; kk++) {
      const int i = lane;
      const bool own = i > kk && i < n;
      const cx<float> x = own ? S.A[i * W + kk] : mkc(0.0f, 0.0f);
      const float sr = sp_wsum(own && i > kk + 1 ? cabs2(x) : 0.0f);
      cx<float> v0, beta;
      float tau;
      sp_householder(S.A[(kk + 1) * W + kk], sr, v0, beta, tau);
      const cx<float> vi = i == kk + 1 ? v0 : x;
      if (own) S.Ref[kk * W + i] = vi;
      if (lane == 0) {
        S.tau[kk] = tau;
        S.w[kk] = beta;  // T_c[kk+1][kk] (entries of w below kk+1 are not used again)
      }
      __syncwarp();
      cx<float> p = mkc(0.0f, 0.0f);
      if (own) {
        for (int j = kk + 1; j < n; j++) cfma(p, S.A[i * W + j], S.Ref[kk * W + j]);
        p = mkc(tau * p.x, tau * p.y);
      }
      const float K = 0.5f * tau * sp_wsum(own ? vi.x * p.x + vi.y * p.y : 0.0f);
      const cx<float> wi = mkc(p.x - K * vi.x, p.y - K * vi.y);
      if (own) S.w[i] = wi;
      __syncwarp();
      if (own) {
        // row i of B - v w^dagger - w v^dagger (the diagonal kept real)
        for (int j = kk + 1; j < n; j++) {
          const cx<float> vj = S.Ref[kk * W + j], wj = S.w[j];
          cx<float> b = S.A[i * W + j];
          b.x -= fmaf(vi.x, wj.x, vi.y * wj.y) + fmaf(wi.x, vj.x, wi.y * vj.y);
          b.y = j == i ? 0.0f : b.y - (fmaf(vi.y, wj.x, -vi.x * wj.y) + fmaf(wi.y, vj.x, -wi.x * vj.y));
          S.A[i * W + j] = b;
        }
      }
      __syncwarp();
    }
    if (lane == 0 && n >= 2) S.w[n - 2] = S.A[(n - 1) * W + n - 2];
    __syncwarp();
    // T = D^dagger T_c D: diagonal d, subdiagonal e = |t|, phases phi (every lane the same)
    float d[W], e[W];
    {
      cx<float> ph = mkc(1.0f, 0.0f);
      if (lane == 0) S.phi[0] = ph;
#pragma unroll
      for (int r = 0; r < W; r++) {
        d[r] = r < n ? S.A[r * W + r].x : 0.0f;
        e[r] = 0.0f;
        if (r < n - 1) {
          const cx<float> t = S.w[r];
          const float m2 = cabs2(t);
          const float mag = sqrtf(m2);
          const cx<float> u = m2 > 0.0f ? mkc(t.x / mag, t.y / mag) : mkc(1.0f, 0.0f);
          ph = mkc(ph.x * u.x - ph.y * u.y, ph.x * u.y + ph.y * u.x);
          e[r] = mag;
          if (lane == 0) S.phi[r + 1] = ph;
        }
      }
    }
    // 2. implicit QR steps with Wilkinson shifts on (d, e); lane r keeps row r of V.  A
    // subdiagonal entry below 2^-22 max(|d|, |e|) is set to zero; the active block is the
    // bottom unreduced one [l, h].
    float vr[W];
#pragma unroll
    for (int c = 0; c < W; c++) vr[c] = c == lane ? 1.0f : 0.0f;
    bool conv = true;
    {
      float scale = 0.0f;
#pragma unroll
      for (int r = 0; r < W; r++) scale = fmaxf(scale, fmaxf(fabsf(d[r]), fabsf(e[r])));
      const float tol = 2.384185791015625e-07f * scale;
      const int maxit = 8 * n;
#pragma unroll 1
      for (int it = 0;; it++) {
        int h = 0;
#pragma unroll
        for (int r = 0; r < W - 1; r++) {
          if (fabsf(e[r]) <= tol) e[r] = 0.0f;
          if (e[r] != 0.0f) h = r + 1;
        }
        if (h == 0) break;
        if (it == maxit) {
          conv = false;
          break;
        }
        int l = 0;
#pragma unroll
        for (int r = 0; r < W - 1; r++)
          if (r < h && e[r] == 0.0f) l = r + 1;
        // Wilkinson shift from the trailing 2 x 2 block [[p, b], [b, s]] of [l, h]
        float pa = 0.0f, sc = 0.0f, b = 0.0f, x = 0.0f, z = 0.0f;
#pragma unroll
        for (int r = 0; r < W - 1; r++) {
          if (r == h - 1) {
            pa = d[r];
            sc = d[r + 1];
            b = e[r];
          }
          if (r == l) {
            x = d[r];
            z = e[r];
          }
        }
        const float del = 0.5f * (pa - sc);
        const float rr = sqrtf(fmaf(del, del, b * b));
        const float den = del >= 0.0f ? del + rr : del - rr;
        const float mu = den != 0.0f ? sc - b * (b / den) : sc;
        x -= mu;
        // bulge chase over the Givens positions l..h-1 (T <- G^T T G, G = [[c, s], [-s, c]])
#pragma unroll
        for (int r = 0; r < W - 1; r++) {
          if (r >= l && r < h) {
            const float r2 = fmaf(x, x, z * z);
            const bool rot = r2 > 0.0f;
            const float ri = rot ? sp_rsqrt(r2) : 0.0f;
            const float cg = rot ? x * ri : 1.0f, sg = rot ? -z * ri : 0.0f;
            if (r > 0 && rot && r > l) e[r - 1] = r2 * ri;
            const float ak = d[r], bk = d[r + 1], ok = e[r];
            const float cc = cg * cg, ss = sg * sg, cs = cg * sg;
            d[r] = fmaf(cc, ak, fmaf(-2.0f * cs, ok, ss * bk));
            d[r + 1] = fmaf(ss, ak, fmaf(2.0f * cs, ok, cc * bk));
            e[r] = fmaf(cs, ak - bk, (cc - ss) * ok);
            if (rot && r + 1 < h) {
              const float en = e[r + 1];
              z = -sg * en;
              e[r + 1] = cg * en;
              x = e[r];
            }
            const float v0 = vr[r], v1 = vr[r + 1];
            vr[r] = fmaf(-sg, v1, cg * v0);
            vr[r + 1] = fmaf(sg, v0, cg * v1);
          }
        }
      }
    }
    if (!conv && lane == 0) atomicOr(a.dstatus, EPW_DEV_NOT_CONVERGED);
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < W; r++)
        if (r < n) S.em[r] = d[r];
    }
    // reachable (m, n): lane n's bands m, as a bit mask; the term list in lane order
    unsigned mask = 0;
    if (lane < n && thr >= 0.0f) {
      const float ekn = S.ek[lane];
#pragma unroll
      for (int m = 0; m < W; m++)
        if (m < n && fabsf(ekn - d[m]) <= thr) mask |= 1u << m;
    }
    const unsigned need = __reduce_or_sync(0xffffffffu, mask);
    int off = __popc(mask);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, off, o);
      if (lane >= o) off += y;
    }
    const int nterm = __shfl_sync(0xffffffffu, off, 31);
    off -= __popc(mask);
    // V^T into the A region (H is no longer needed), for the eigenvector columns
    __syncwarp();
    float *Vt = reinterpret_cast<float *>(S.A);
    if (lane < n) {
#pragma unroll
      for (int c = 0; c < W; c++)
        if (c < n) Vt[lane * W + c] = vr[c];
    }
    {
      unsigned mm = mask;
      int j = off;
      while (mm) {
        const int m = __ffs(mm) - 1;
        mm &= mm - 1;
        S.tm[j] = (unsigned char)m;
        S.tn[j] = (unsigned char)lane;
        j++;
      }
    }
    __syncwarp();
    // 3. eigenvector m (lane m, when some band reaches it): u = Q D V e_m, the reflectors
    // applied last to first
    if (lane < n && ((need >> lane) & 1u)) {
      cx<float> u[W];
#pragma unroll
      for (int r = 0; r < W; r++) {
        const float y = r < n ? Vt[r * W + lane] : 0.0f;
        const cx<float> ph = r < n ? S.phi[r] : mkc(0.0f, 0.0f);
        u[r] = mkc(ph.x * y, ph.y * y);
      }
#pragma unroll
      for (int kk = W - 3; kk >= 0; kk--) {
        if (kk <= n - 3) {
          cx<float> sv = mkc(0.0f, 0.0f);
#pragma unroll
          for (int r = kk + 1; r < W; r++)
            if (r < n) {
              const cx<float> vv = S.Ref[kk * W + r];
              sv = mkc(fmaf(vv.x, u[r].x, fmaf(vv.y, u[r].y, sv.x)), fmaf(vv.x, u[r].y, fmaf(-vv.y, u[r].x, sv.y)));
            }
          const float tk = S.tau[kk];
          sv = mkc(tk * sv.x, tk * sv.y);
#pragma unroll
          for (int r = kk + 1; r < W; r++)
            if (r < n) {
              const cx<float> vv = S.Ref[kk * W + r];
              u[r] = mkc(u[r].x - fmaf(vv.x, sv.x, -vv.y * sv.y), u[r].y - fmaf(vv.x, sv.y, vv.y * sv.x));
            }
        }
      }
#pragma unroll
      for (int r = 0; r < W; r++)
        if (r < n) S.U[r * W + lane] = u[r];
    }
    __syncwarp();
    // 4. the reachable terms, one per lane: t_a = u_m^dagger X_a[:, n], g_nu = sum_a E[a][nu] t_a
    float *red = reinterpret_cast<float *>(S.Ref);  // term sums [m W + n] (reflectors done)
    for (int e2 = lane; e2 < W * W; e2 += 32) red[e2] = 0.0f;
    __syncwarp();
    for (int r0 = 0; r0 < nterm; r0 += 32) {
      const int j = r0 + lane;
      const bool act = j < nterm;
      const int m = act ? S.tm[j] : 0, nb_ = act ? S.tn[j] : 0;
      cx<float> um[W];
#pragma unroll
      for (int r = 0; r < W; r++) um[r] = (act && r < n) ? S.U[r * W + m] : mkc(0.0f, 0.0f);
      cx<float> g[SP_MMAX];
#pragma unroll
      for (int v = 0; v < SP_MMAX; v++) g[v] = mkc(0.0f, 0.0f);
#pragma unroll 1
      for (int al = 0; al < nm; al++) {
        // X_a of this pair into the A region (coalesced), then the lanes' columns
        __syncwarp();
        const float *Xa = C + 2 * (size_t)nn2 * (1 + al);
        for (int e2 = lane; e2 < nn2; e2 += 32) {
          const int r = e2 / n, c = e2 - r * n;
          S.A[r * W + c] = mkc(Xa[2 * e2], Xa[2 * e2 + 1]);
        }
        __syncwarp();
        cx<float> t = mkc(0.0f, 0.0f);
#pragma unroll
        for (int r = 0; r < W; r++)
          if (r < n) {
            const cx<float> xv = S.A[r * W + nb_];
            t = mkc(fmaf(um[r].x, xv.x, fmaf(um[r].y, xv.y, t.x)), fmaf(um[r].x, xv.y, fmaf(-um[r].y, xv.x, t.y)));
          }
        const cx<float> *Ea = S.E + al * nm;
#pragma unroll
        for (int v = 0; v < SP_MMAX; v++)
          if (v < nm) cfma(g[v], Ea[v], t);
      }
      if (a.Cpol) {
        // long-range part: g_nu += i C_nu(q) (u_m^dagger U_k)_n
        const cx<double> *Uk = a.Uk + (size_t)k * nn2;
        const cx<float> *Cp = (const cx<float> *)a.Cpol;
        cx<float> tp = mkc(0.0f, 0.0f);
#pragma unroll
        for (int r = 0; r < W; r++)
          if (r < n) {
            const cx<float> w = act ? ccast<float>(Uk[r * n + nb_]) : mkc(0.0f, 0.0f);
            tp = mkc(fmaf(um[r].x, w.x, fmaf(um[r].y, w.y, tp.x)), fmaf(um[r].x, w.y, fmaf(-um[r].y, w.x, tp.y)));
          }
#pragma unroll
        for (int v = 0; v < SP_MMAX; v++)
          if (v < nm) {
            const cx<float> c = Cp[(size_t)v * nq + q];
            cfma(g[v], mkc(-c.y, c.x), tp);
          }
      }
      if (act) {
        const float emm = S.em[m];
        const float x = S.ek[nb_] - emm;
        const float f = occ_fermi<float>(emm, a.EF, a.T);
        float acc = 0.0f;
#pragma unroll
        for (int v = 0; v < SP_MMAX; v++)
          if (v < nm && ((keepmask >> v) & 1u)) {
            const float w = S.om[v], nbv = S.nb[v];
            acc += cabs2(g[v]) * ((nbv + f) * gauss_r<float>(x + w, inv_sigma, gnorm) +
                                  (nbv + 1.0f - f) * gauss_r<float>(x - w, inv_sigma, gnorm));
          }
        red[m * W + nb_] = acc;
      }
    }
    __syncwarp();
    // per band n: the sum over m (ascending), times w_q
    if (lane < n) {
      double sm = 0.0;
      for (int m = 0; m < n; m++) sm += (double)red[m * W + lane];
      const double wqi = a.wq ? a.wq[q] : 1.0 / nq;
      accn += sm * wqi;
    }
    __syncwarp();
  }
  if (lane < W) nsum[warp][lane] = lane < n ? accn : 0.0;
  __syncthreads();
  if (threadIdx.x < n) {
    const int nb_ = threadIdx.x;
    const double s = ((nsum[0][nb_] + nsum[1][nb_]) + nsum[2][nb_]) + nsum[3][nb_];
    a.partial[((size_t)k * gridDim.x + blockIdx.x) * n + nb_] = s;
  }
}

}  // namespace

// Linewidth terms (mode 0) for the staged FP32 form of the wide shapes: one warp per pair.
epw_status launch_pair_sparse(const PairArgs &a, cudaStream_t st) {
  if (a.nk <= 0 || a.nq <= 0) return EPW_OK;
  if (!a.Cq || a.nw > 18 || a.nm > SP_MMAX) return EPW_ERR_UNSUPPORTED;
  dim3 grid((a.nq + SP_WARPS * 32 - 1) / (SP_WARPS * 32), a.nk);
  auto go = [&](auto kern, size_t smem) -> epw_status {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return EPW_ERR_CUDA;
    kern<<<grid, SP_WARPS * 32, smem, st>>>(a);
    epw_count_launch();
    return cudaGetLastError() == cudaSuccess ? EPW_OK : EPW_ERR_CUDA;
  };
  // register arrays (QR rows, eigenvectors) sized for the smallest width that holds nw
  if (a.nw <= 8) return go(k_pair_sparse<8>, SP_WARPS * sizeof(SpWarp<8>));
  if (a.nw <= 12) return go(k_pair_sparse<12>, SP_WARPS * sizeof(SpWarp<12>));
  return go(k_pair_sparse<18>, SP_WARPS * sizeof(SpWarp<18>));
}
