// Per-pair work for wide shapes (nw up to 18 Wannier functions, up to 18
// modes): the same steps as the register-tile per-pair kernel (Eq.
// (linewidthel) with the overlap rotation of the interpolation), with one warp
// per (k,q) pair and the matrices in shared memory:
//   H(k+q)  -> warp-cooperative cyclic Jacobi -> e_m, U          (A, U in smem)
//   G'_nu   = sum_a E_q[a][nu] X_a,   X_a = g_a(k,q) U_k        (lanes own entries)
//   g_nu    = U^dagger G'_nu                                    (G'_nu staged in smem)
// Modes are taken in blocks of NB so that the lanes' accumulators stay in
// registers; the contraction X_a is recomputed (or re-read from the staged
// tensor-core result) once per block.  A block of 4 warps covers 128
// consecutive q of one k, each warp 32 of them in order, so the per-(k, q-tile)
// partial sums are formed in a fixed order.
#include "epw_internal.cuh"

namespace {

constexpr int WMAX = 18;                         // largest nw and 3nat
constexpr int TMAX = (WMAX * WMAX + 31) / 32;    // matrix entries per lane
constexpr int WARPS = 4;

template <typename R>
struct WideNB;
template <>
struct WideNB<float> {
  static constexpr int v = 6;
};
template <>
struct WideNB<double> {
  static constexpr int v = 3;
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Rotation of the (p,q) plane that zeroes a_pq (same parametrisation as the
// register-tile solver): d = a_qq - a_pp, t = 2|a_pq| sgn(d) / (|d| + sqrt(d^2 + 4|a_pq|^2)),
// c = 1/sqrt(1+t^2), se = c t a_pq/|a_pq|; a_pp -= t|a_pq|, a_qq += t|a_pq|.
template <typename R>
__device__ __forceinline__ void jrot(R app, R aqq, cx<R> apq, R &c, cx<R> &se, R &tb) {
  const R a2 = apq.x * apq.x + apq.y * apq.y;
  const R d = aqq - app;
  const R sg = d >= R(0) ? R(1) : R(-1);
  const R den = fabs(d) + sqrt(d * d + R(4) * a2);
  const R am = sqrt(a2);
  const R t = R(2) * am * sg / den;
  c = R(1) / sqrt(R(1) + t * t);
  const R kap = sg * R(2) * c / den;
  se = mkc<R>(kap * apq.x, kap * apq.y);
  tb = t * am;
}

// Hermitian A (nw x nw, row-major, smem) -> diagonal (eigenvalues on it), U the
// eigenvector columns.  Every lane takes the same branch (values read from smem).
template <typename R>
__device__ bool warp_jacobi(cx<R> *A, cx<R> *U, int nw, int lane) {
  const int nw2 = nw * nw;
  for (int e = lane; e < nw2; e += 32) U[e] = mkc<R>(e / nw == e % nw ? R(1) : R(0), R(0));
  __syncwarp();
  for (int sweep = 0; sweep <= jacobi_tol<R>::maxsweep; sweep++) {
    double off = 0.0, dg = 0.0;
    for (int e = lane; e < nw2; e += 32) {
      const int i = e / nw, j = e % nw;
      if (i < j) off += (double)cabs2(A[e]);
      if (i == j) dg += (double)A[e].x * (double)A[e].x;
    }
    off = wsum(off);
    dg = wsum(dg);
    if (off <= (double)jacobi_tol<R>::tol2 * (dg + 2.0 * off)) return true;
    if (sweep == jacobi_tol<R>::maxsweep) break;
    for (int p = 0; p < nw - 1; p++)
      for (int q = p + 1; q < nw; q++) {
        const cx<R> apq = A[p * nw + q];
        if (apq.x == R(0) && apq.y == R(0)) continue;
        const R app = A[p * nw + p].x, aqq = A[q * nw + q].x;
        R c, tb;
        cx<R> se;
        jrot<R>(app, aqq, apq, c, se, tb);
        const cx<R> sec = conjc(se);
        cx<R> akp = mkc<R>(0, 0), akq = mkc<R>(0, 0), ukp = mkc<R>(0, 0), ukq = mkc<R>(0, 0);
        const int k = lane;
        if (k < nw) {
          akp = A[k * nw + p];
          akq = A[k * nw + q];
          ukp = U[k * nw + p];
          ukq = U[k * nw + q];
        }
        __syncwarp();
        if (k < nw) {
          if (k != p && k != q) {
            cx<R> nkp = mkc<R>(c * akp.x, c * akp.y), nkq = mkc<R>(c * akq.x, c * akq.y);
            cfma(nkp, mkc<R>(-sec.x, -sec.y), akq);
            cfma(nkq, se, akp);
            A[k * nw + p] = nkp;
            A[p * nw + k] = conjc(nkp);
            A[k * nw + q] = nkq;
            A[q * nw + k] = conjc(nkq);
          }
          cx<R> np = mkc<R>(c * ukp.x, c * ukp.y), nq = mkc<R>(c * ukq.x, c * ukq.y);
          cfma(np, mkc<R>(-sec.x, -sec.y), ukq);
          cfma(nq, se, ukp);
          U[k * nw + p] = np;
          U[k * nw + q] = nq;
        }
        if (lane == 0) {
          A[p * nw + p] = mkc<R>(app - tb, R(0));
          A[q * nw + q] = mkc<R>(aqq + tb, R(0));
          A[p * nw + q] = mkc<R>(R(0), R(0));
          A[q * nw + p] = mkc<R>(R(0), R(0));
        }
        __syncwarp();
      }
  }
  return false;
}

// Entry e of the contraction block `blk` (0: H(k+q), 1 + a: X_a) of pair (kl, q).
template <typename R, bool FROMC>
__device__ __forceinline__ cx<R> contraction(const PairArgs &a, int kl, int k, int q, int blk, int e) {
  const int nw2 = a.nw * a.nw;
  if constexpr (FROMC) {
    const float *C = a.Cq + (size_t)q * a.ldc + (size_t)kl * a.cpk + 2 * ((size_t)blk * nw2 + e);
    return mkc<R>((R)C[0], (R)C[1]);
  } else {
    cx<R> s = mkc<R>(0, 0);
    if (blk == 0) {
      const cx<R> *P = (const cx<R> *)a.PqTe;
      const cx<R> *B = (const cx<R> *)a.BH + (size_t)k * a.nRe * nw2 + e;
      for (int r = 0; r < a.nRe; r++) cfma(s, P[(size_t)r * a.nq + q], B[(size_t)r * nw2]);
    } else {
      const cx<R> *P = (const cx<R> *)a.PqTp;
      const cx<R> *B = (const cx<R> *)a.Bg + ((size_t)k * a.nRp * a.nm + (blk - 1)) * nw2 + e;
      for (int r = 0; r < a.nRp; r++) cfma(s, P[(size_t)r * a.nq + q], B[(size_t)r * a.nm * nw2]);
    }
    return s;
  }
}

template <typename R, int MODE, bool FROMC>
__global__ void __launch_bounds__(WARPS * 32) k_pair_wide(PairArgs a) {
  constexpr int NB = WideNB<R>::v;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double nsum[WARPS][WMAX];
  __shared__ int rks[WARPS][WMAX];  // MODE 1: ascending position of eigenvalue m
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = a.nw, nm = a.nm, nw2 = nw * nw, nq = a.nq;
  const int kl = blockIdx.y, k = a.k0 + kl;
  cx<R> *A = (cx<R> *)smraw + (size_t)warp * 3 * nw2;
  cx<R> *U = A + nw2, *Gs = U + nw2;
  R *fm = (R *)((cx<R> *)smraw + (size_t)WARPS * 3 * nw2) + warp * 2 * WMAX;
  R *em = fm + WMAX;
  const double *ek = a.eps_k + (size_t)k * nw;
  const R inv_sigma = (R)(1.0 / a.sigma);
  const R gnorm = (R)(1.0 / (a.sigma * 1.7724538509055160273));
  double accn = 0.0;  // lane n: this warp's sum for band n
  for (int i = 0; i < 32; i++) {
    const int q = blockIdx.x * (WARPS * 32) + warp * 32 + i;
    if (q >= nq) break;
    // H(k+q): Hermitian part of the contraction
    for (int e = lane; e < nw2; e += 32) Gs[e] = contraction<R, FROMC>(a, kl, k, q, 0, e);
    __syncwarp();
    for (int e = lane; e < nw2; e += 32) {
      const int r = e / nw, c = e % nw;
      const cx<R> x = Gs[e], y = Gs[c * nw + r];
      A[e] = mkc<R>(R(0.5) * (x.x + y.x), r == c ? R(0) : R(0.5) * (x.y - y.y));
    }
    __syncwarp();
    const bool conv = warp_jacobi<R>(A, U, nw, lane);
    if (!conv && lane == 0) atomicOr(a.dstatus, EPW_DEV_NOT_CONVERGED);
    if (lane < nw) {
      const R e = A[lane * nw + lane].x;
      em[lane] = e;
      fm[lane] = occ_fermi<R>(e, a.EF, a.T);
    }
    __syncwarp();
    if (MODE == 1) {
      if (lane < nw) {
        const R e = em[lane];
        int rank = 0;
        for (int j = 0; j < nw; j++) rank += (em[j] < e || (em[j] == e && j < lane)) ? 1 : 0;
        rks[warp][lane] = rank;
        if (a.eps_kq) a.eps_kq[((size_t)k * nq + q) * nw + rank] = (double)e;
      }
      __syncwarp();
    }
    R acc[TMAX];
#pragma unroll
    for (int t = 0; t < TMAX; t++) acc[t] = R(0);
    for (int v0 = 0; v0 < nm; v0 += NB) {
      const int nb = min(NB, nm - v0);
      cx<R> Gp[NB][TMAX];
#pragma unroll
      for (int b = 0; b < NB; b++)
#pragma unroll
        for (int t = 0; t < TMAX; t++) Gp[b][t] = mkc<R>(0, 0);
      for (int al = 0; al < nm; al++) {
        cx<R> E[NB];
        const cx<R> *ET = (const cx<R> *)a.ET;
#pragma unroll
        for (int b = 0; b < NB; b++) E[b] = b < nb ? ET[((size_t)al * nm + v0 + b) * nq + q] : mkc<R>(0, 0);
#pragma unroll
        for (int t = 0; t < TMAX; t++) {
          const int e = lane + 32 * t;
          if (e < nw2) {
            const cx<R> x = contraction<R, FROMC>(a, kl, k, q, 1 + al, e);
#pragma unroll
            for (int b = 0; b < NB; b++) cfma(Gp[b][t], E[b], x);
          }
        }
      }
      if (a.Cpol) {
        // long-range part in the Wannier gauge: G'_nu += i C_nu(q) U_k
        const cx<R> *Cp = (const cx<R> *)a.Cpol;
        const cx<double> *Uk = a.Uk + (size_t)k * nw2;
#pragma unroll
        for (int b = 0; b < NB; b++) {
          if (b >= nb) break;
          const cx<R> c = Cp[(size_t)(v0 + b) * nq + q];
#pragma unroll
          for (int t = 0; t < TMAX; t++) {
            const int e = lane + 32 * t;
            if (e < nw2) cfma(Gp[b][t], mkc<R>(-c.y, c.x), ccast<R>(Uk[e]));
          }
        }
      }
#pragma unroll
      for (int b = 0; b < NB; b++) {
        if (b >= nb) break;
        const int v = v0 + b;
#pragma unroll
        for (int t = 0; t < TMAX; t++) {
          const int e = lane + 32 * t;
          if (e < nw2) Gs[e] = Gp[b][t];
        }
        __syncwarp();
        const R w = (R)a.omegaT[(size_t)v * nq + q];
        const bool keep = (w >= (R)a.omega_min) && (w > R(0));
        const R nbose = keep ? occ_bose<R>(w, a.T) : R(0);
#pragma unroll
        for (int t = 0; t < TMAX; t++) {
          const int e = lane + 32 * t;
          if (e >= nw2) continue;
          const int m = e / nw, n = e % nw;
          cx<R> y = mkc<R>(0, 0);
          for (int r = 0; r < nw; r++) cfma(y, conjc(U[r * nw + m]), Gs[r * nw + n]);
          if constexpr (MODE == 1) {
            if (a.gout) a.gout[(((size_t)k * nq + q) * nm + v) * nw2 + (size_t)rks[warp][m] * nw + n] = ccast<double>(y);
          } else {
            if (keep) {
              const R x = (R)ek[n] - em[m];
              const R f = fm[m];
              acc[t] += cabs2(y) * ((nbose + f) * gauss_r<R>(x + w, inv_sigma, gnorm) +
                                    (nbose + R(1) - f) * gauss_r<R>(x - w, inv_sigma, gnorm));
            }
          }
        }
        __syncwarp();
      }
    }
    if constexpr (MODE == 0) {
      // per-entry sums -> per band n (sum over m), times w_q
      R *red = (R *)Gs;
#pragma unroll
      for (int t = 0; t < TMAX; t++) {
        const int e = lane + 32 * t;
        if (e < nw2) red[e] = acc[t];
      }
      __syncwarp();
      if (lane < nw) {
        double s = 0.0;
        for (int m = 0; m < nw; m++) s += (double)red[m * nw + lane];
        const double wqi = a.wq ? a.wq[q] : 1.0 / nq;
        accn += s * wqi;
      }
      __syncwarp();
    }
  }
  if constexpr (MODE == 0) {
    if (lane < WMAX) nsum[warp][lane] = lane < nw ? accn : 0.0;
    __syncthreads();
    if (threadIdx.x < nw) {
      const int n = threadIdx.x;
      const double s = ((nsum[0][n] + nsum[1][n]) + nsum[2][n]) + nsum[3][n];
      a.partial[((size_t)k * gridDim.x + blockIdx.x) * nw + n] = s;
    }
  }
}

}  // namespace

template <typename R>
epw_status launch_pair_wide(const PairArgs &a, int mode, cudaStream_t st) {
  const int nkl = a.nk;
  if (nkl <= 0 || a.nq <= 0) return EPW_OK;
  if (a.nw > WMAX || a.nm > WMAX || mode == 2) return EPW_ERR_UNSUPPORTED;
  const bool fromc = a.Cq != nullptr;
  if (fromc && sizeof(R) != sizeof(float)) return EPW_ERR_UNSUPPORTED;
  const size_t smem = (size_t)WARPS * 3 * a.nw * a.nw * sizeof(cx<R>) + (size_t)WARPS * 2 * WMAX * sizeof(R);
  dim3 grid((a.nq + WARPS * 32 - 1) / (WARPS * 32), nkl);
  auto go = [&](auto kern) -> epw_status {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return EPW_ERR_CUDA;
    kern<<<grid, WARPS * 32, smem, st>>>(a);
    epw_count_launch();
    return cudaGetLastError() == cudaSuccess ? EPW_OK : EPW_ERR_CUDA;
  };
  if constexpr (sizeof(R) == sizeof(float)) {
    if (fromc) return mode == 0 ? go(k_pair_wide<float, 0, true>) : go(k_pair_wide<float, 1, true>);
  }
  return mode == 0 ? go(k_pair_wide<R, 0, false>) : go(k_pair_wide<R, 1, false>);
}
template epw_status launch_pair_wide<double>(const PairArgs &, int, cudaStream_t);
template epw_status launch_pair_wide<float>(const PairArgs &, int, cudaStream_t);
