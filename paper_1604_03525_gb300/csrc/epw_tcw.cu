// Wide-shape fused linewidth path on the 5th-generation tensor cores (sm_103a),
// for models whose per-k accumulator columns 2 nw^2 (3nat + 1) exceed the fused
// kernel's 128-column slot (diamond nw = 8 with 6 modes, hexagonal nw = 5 with 9).
//
// The per-pair work of Eq. (linewidthel) splits into two tcgen05 kernels per
// chunk of k-points, both over A operands of q phases P_q(R) (real GEMM,
// K = 2 nR with re/im interleaved, split into two bf16 or tf32 terms, three
// MMAs per K step, FP32 accumulation in tensor memory):
//
//  E  C[q][(k, i, j)] = sum_R P_q(R) P_k(R) H(R) = H(k+q)_ij; the epilogue takes
//     the Hermitian part and diagonalises it per pair in FP32 (Householder +
//     implicit QR, epw_eigqr.cuh), writes the eigenvalues e_m,k+q and, for the
//     bands m that some band n at k can reach within the Gaussian cutoff
//     (|e_nk - e_m,k+q| <= max_nu w_q,nu + X sigma), the eigenvectors u_m.
//  G  C[q][((k, n), a, j)] = sum_Rp P_q(Rp) (g_a(k,Rp) U_k)_jn = (g_a(k,q) U_k)_jn
//     (over its own A operand of phases P_q(Rp) when the phonon-displacement set Rp
//     differs from Re),
//     the columns of one band n of k contiguous; the epilogue forms, for the
//     reachable (m, n) only, t_a = u_m^dagger (g_a U_k)_{:,n},
//     g_mn,nu = sum_a E_q[a][nu] t_a (+ i C_nu(q) u_m^dagger U_k e_n for the
//     long-range part), the occupations and Gaussians of Eq. (linewidthel),
//     and sums |g|^2 W over the warp's 32 q rows into per-(k, q tile) partials.
//
// The cutoff X = sqrt(130 ln 2) (about 9.49) makes every skipped Gaussian
// 2^-(x s)^2 with (x s)^2 > 130, which the flush-to-zero ex2 of the dense form
// returns as exactly 0, so the sum equals the dense one term for term.
// Both kernels are persistent (one CTA per SM): warp 0 issues TMA copies, warp
// 1 owns tensor memory and issues the MMAs, warps 2..9 are the epilogue (two
// per TMEM lane quadrant, taking the quadrant's items round-robin); tensor
// memory holds two 256-column accumulator stages so the MMAs of the next tile
// overlap the epilogue of the current one.  Every wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "epw_eigqr.cuh"
#include "epw_tc.cuh"
#include "epw_tcgen05.cuh"

namespace {

constexpr int BM = 128;  // q rows per tile
// Operand stages: kernel E two of 128-byte K rows (128-byte swizzle); kernel G,
// whose MMAs are the bulk of the work, four of 64-byte K rows (64-byte swizzle),
// so that three stages are in flight while the MMAs consume the fourth.
template <int KIND>
constexpr int w_rowb() {
  return KIND == 0 ? 128 : 64;
}
template <int KIND>
constexpr int w_stages() {
  return KIND == 0 ? 2 : 4;
}
constexpr int EPI_WARP0 = 2;
// Epilogue warps: two per TMEM lane quadrant in both kernels (eight warps).
template <int KIND>
constexpr int epi_warps() {
  return KIND == 0 ? 8 : 8;
}
template <int KIND>
constexpr int nthreads() {
  return 32 * (EPI_WARP0 + epi_warps<KIND>());
}
constexpr uint32_t TMEM_COLS = 512;
constexpr size_t A_BLOCK_BYTES = 48u << 20;  // q-block of the A operand kept in L2 across column groups
// Gaussian cutoff: the dense form's ex2.approx.ftz(-(x s)^2) is exactly 0 for (x s)^2 > 126
constexpr double CUT_SIGMAS = 9.4921453036541;  // sqrt(130 ln 2)

template <int OP>
struct WOp;
template <>
struct WOp<TC_OP_BF16> {
  using T = __nv_bfloat16;
  static constexpr int ESZ = 2, KSTEP = 16;
  static constexpr bool F16 = true;
  static constexpr uint32_t FMT = 1;
};
template <>
struct WOp<TC_OP_TF32> {
  using T = float;
  static constexpr int ESZ = 4, KSTEP = 8;
  static constexpr bool F16 = false;
  static constexpr uint32_t FMT = 2;
};
// instruction descriptor: D = F32, A = B = bf16 (kind::f16) or tf32, both K-major, M = 128
template <int OP, int N>
constexpr uint32_t w_idesc() {
  return (1u << 4) | (WOp<OP>::FMT << 7) | (WOp<OP>::FMT << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}
// the same for a CTA pair's MMA (M = 256: 128 rows in each CTA)
template <int OP, int N>
constexpr uint32_t w_idesc_pair() {
  return (1u << 4) | (WOp<OP>::FMT << 7) | (WOp<OP>::FMT << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)((2 * BM) >> 4) << 24);
}

template <int NW, int NM>
struct WShape {
  static constexpr int H2 = 2 * NW * NW;                            // real columns of H(k+q)
  static constexpr int CPK = H2 <= 32 ? 32 : H2 <= 64 ? 64 : 128;   // E columns per k
  static constexpr int KPT = 256 / CPK;                             // k per E tile
  static constexpr int ENT = 2 * NM * NW;                           // G columns of one band n of one k
  static constexpr int ENTP = (ENT + 31) / 32 * 32;
  static constexpr int CN = 256 / ENTP;                             // (k, n) entries per G tile
  static constexpr int BNG = CN * ENTP;
  static_assert(H2 <= 128 && ENTP <= 256, "shape beyond the wide tensor-core form");
};
template <int NW, int NM, int KIND>
constexpr int w_bn() {
  return KIND == 0 ? 256 : WShape<NW, NM>::BNG;
}
template <int NW, int NM, int KIND>
constexpr int w_units() {
  return KIND == 0 ? WShape<NW, NM>::KPT : WShape<NW, NM>::CN;
}
template <int NW, int NM, int KIND>
constexpr int w_smem() {
  return w_stages<KIND>() * (2 * BM + 2 * w_bn<NW, NM, KIND>()) * w_rowb<KIND>() + 1024;
}

struct TcwArgs {
  int nq, nqt, ngrp, kpad, nkb, qblock;
  int kpadG, nkbG;        // fused kernel: K extent of the vertex chunks (Rp phases) when it differs
  int k0, kc;             // chunk: global k = k0 + kl, kl < kc
  int ldq;                // q stride of the per-pair buffers (nqt * 128)
  const float *epsk;      // [nk][nw]
  const float *thr;       // [nq] max kept w_q,nu + cutoff (negative: no kept mode)
  const float *omegaT;    // [nm][nq]
  const float *nbT;       // [nm][nq]
  const float2 *ET;       // [nm*nm][nq] mode factors e/sqrt(2 M w)
  const float *wq;        // [nq]
  float EF, invkT, sc, gnorm, omega_min;
  float *epsq;            // [kc][nw][ldq]
  float2 *Uq;             // [kc][nw][nw][ldq]
  double *partial;        // [nk][4 nqt][nw]
  unsigned *dstatus;
  const float2 *Cpol;     // [nm][nq] or null
  const float2 *UkF;      // [nk][nw][nw]
};

// Tile -> (column group, q tile): q-blocks of `qblock` tiles, group-major inside a block.
__device__ __forceinline__ void w_coords_n(int nqt, int qblock, int ngrp, int item, int &grp, int &qt) {
  const int per = qblock * ngrp;
  const int nb = (nqt + qblock - 1) / qblock;
  int b = item / per;
  if (b > nb - 1) b = nb - 1;
  const int r = item - b * per;
  const int qbs = min(qblock, nqt - b * qblock);
  grp = r / qbs;
  qt = b * qblock + r % qbs;
}
__device__ __forceinline__ void w_coords(const TcwArgs &a, int item, int &grp, int &qt) {
  w_coords_n(a.nqt, a.qblock, a.ngrp, item, grp, qt);
}

// The one relevance test both kernels evaluate (same FP32 operands, same result).
__device__ __forceinline__ bool reachable(float ek, float em, float thr) { return fabsf(ek - em) <= thr; }

// Where the eigen-data of one pair lives: eigenvalue m at eps[m ld + idx], component i
// of eigenvector m at U[(m nw + i) ld + idx].
struct EigView {
  float *eps;
  float2 *U;
  size_t ld;
  int idx;
};

// ------------------------------------------------------------ epilogue E
// H(k+q) from tensor memory, its FP32 eigensolve, the eigenvalues and the
// eigenvectors that some band n at k can reach into v (kg: global k index).
// FUSED: release the H(k+q) region (arrive on hempty) once H is in registers, and
// wait on eempty (phase epar) before writing v; false when that wait gave up.
template <int NW, bool FUSED = false>
__device__ __forceinline__ bool eig_pair(const TcwArgs &a, uint32_t tcol, int q, int kg, const EigView &v,
                                         bool valid, uint32_t hempty = 0, uint32_t eempty = 0, uint32_t epar = 0,
                                         volatile int *abort_flag = nullptr, bool hempty_cluster = false) {
  constexpr int H2 = 2 * NW * NW;
  constexpr int LD = (H2 + 31) / 32 * 32;
  Herm<NW> H;
  {
    float hb[LD];
#pragma unroll
    for (int c = 0; c < LD; c += 32) {
      float t[32];
      tmem_ld32(tcol + c, t);
#pragma unroll
      for (int i = 0; i < 32; i++) hb[c + i] = t[i];
    }
#pragma unroll
    for (int i = 0; i < NW; i++)
#pragma unroll
      for (int j = i; j < NW; j++) {
        const int o = 2 * (i * NW + j), o2 = 2 * (j * NW + i);
        H.a[i][j] = mkc(0.5f * (hb[o] + hb[o2]), i == j ? 0.0f : 0.5f * (hb[o + 1] - hb[o2 + 1]));
      }
  }
  if constexpr (FUSED) {
    // H is in registers: the tensor-memory region may take the next item's H(k+q)
    tc_fence_before();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
      if (hempty_cluster)
        mbar_arrive_cluster(hempty);
      else
        mbar_arrive(hempty);
    }
  }
  HhQR<NW> S;
  hh_tridiag<NW>(H, S);
  const bool conv = tri_qr<NW>(S);
  if (!conv && valid) atomicOr(a.dstatus, EPW_DEV_NOT_CONVERGED);
  kg = valid ? kg : 0;
  const float thr = valid ? __ldg(a.thr + q) : -1.0f;
  float ek[NW];
#pragma unroll
  for (int n = 0; n < NW; n++) ek[n] = __ldg(a.epsk + (size_t)kg * NW + n);
  if constexpr (FUSED) {
    // the eigen-data slot must be free (its previous item consumed) before it is written
    const bool ok = wait_bar(eempty, epar, abort_flag, a.dstatus);
    if (!__all_sync(0xffffffffu, ok)) return false;
  }
  if (valid) {
#pragma unroll
    for (int m = 0; m < NW; m++) v.eps[(size_t)m * v.ld + v.idx] = S.d[m];
  }
  // the bands m that some band n at k can reach, one bit per m
  uint32_t need = 0;
#pragma unroll
  for (int m = 0; m < NW; m++) {
    bool rel = false;
#pragma unroll
    for (int n = 0; n < NW; n++) rel = rel || reachable(ek[n], S.d[m], thr);
    if (rel && valid) need |= 1u << m;
  }
  // each lane forms its own reachable eigenvectors, lowest m first: the warp runs as many
  // rounds as its busiest lane needs (not the union of the lanes' bands); one loop body
  // for the instruction cache, m a per-lane index (hh_vector picks by weights)
#pragma unroll 1
  while (__any_sync(0xffffffffu, need != 0)) {
    const bool act = need != 0;
    const int m = act ? __ffs(need) - 1 : 0;
    need &= need - 1;
    cx<float> u[NW];
    hh_vector<NW>(S, m, u);
    if (act) {
      float2 *dst = v.U + (size_t)m * NW * v.ld + v.idx;
#pragma unroll
      for (int i = 0; i < NW; i++) dst[(size_t)i * v.ld] = make_float2(u[i].x, u[i].y);
    }
  }
  return true;
}

// ------------------------------------------------------------ epilogue G
// Linewidth terms of one pair (k, q) and one band n at k from the accumulator
// columns (a, j) of (g_a(k,q) U_k)_{jn}: only the bands m with a reachable
// delta are evaluated (the warp runs the union over its lanes).
template <int NW, int NM>
__device__ __forceinline__ float g_entry(const TcwArgs &a, uint32_t tcol, int q, int kg, int n, const EigView &v,
                                         bool valid) {
  constexpr int ENT = 2 * NM * NW;
  constexpr int LD = (ENT + 31) / 32 * 32;
  const int qq = valid ? q : 0;
  kg = valid ? kg : 0;
  const float thr = valid ? __ldg(a.thr + q) : -1.0f;
  const float ek = __ldg(a.epsk + (size_t)kg * NW + n);
  // bands m at k+q with a Gaussian above the cutoff, as a bit mask
  uint32_t relm = 0;
#pragma unroll
  for (int m = 0; m < NW; m++) {
    const float em = valid ? v.eps[(size_t)m * v.ld + v.idx] : 0.0f;
    if (valid && reachable(ek, em, thr)) relm |= 1u << m;
  }
  if (!__any_sync(0xffffffffu, relm != 0)) return 0.0f;
  float om[NM], nb[NM];
#pragma unroll
  for (int nu = 0; nu < NM; nu++) {
    om[nu] = __ldg(a.omegaT + (size_t)nu * a.nq + qq);
    nb[nu] = __ldg(a.nbT + (size_t)nu * a.nq + qq);
  }
  const float eks = ek * a.sc;
  float acc = 0.0f;
  // one loop body over m (instruction cache); the warp runs the union of its lanes' bands
#pragma unroll 1
  for (int m = 0; m < NW; m++) {
    const bool rel = (relm >> m) & 1u;
    if (!__any_sync(0xffffffffu, rel)) continue;
    cx<float> u[NW];
    float em = 0.0f;
    if (rel) {
      em = v.eps[(size_t)m * v.ld + v.idx];
      const float2 *src = v.U + (size_t)m * NW * v.ld + v.idx;
#pragma unroll
      for (int i = 0; i < NW; i++) {
        const float2 w = src[(size_t)i * v.ld];
        u[i] = mkc(w.x, w.y);
      }
    } else {
#pragma unroll
      for (int i = 0; i < NW; i++) u[i] = mkc(0.0f, 0.0f);
    }
    // t_a = u_m^dagger (g_a U_k)_{:, n}; the entry's columns 2 (a nw + j) + (re, im)
    // stream from tensor memory 32 at a time (every lane of the warp loads)
    cx<float> t[NM];
#pragma unroll
    for (int al = 0; al < NM; al++) t[al] = mkc(0.0f, 0.0f);
#pragma unroll
    for (int c0 = 0; c0 < LD; c0 += 32) {
      float xc[32];
      tmem_ld32(tcol + c0, xc);
#pragma unroll
      for (int cc = 0; cc < 32; cc += 2) {
        const int col = c0 + cc;
        if (col < ENT) {
          const int al = col / (2 * NW), j = (col >> 1) % NW;
          const float br = xc[cc], bi = xc[cc + 1];
          t[al] = mkc(fmaf(u[j].x, br, fmaf(u[j].y, bi, t[al].x)), fmaf(u[j].x, bi, fmaf(-u[j].y, br, t[al].y)));
        }
      }
    }
    if (!rel) continue;
    cx<float> tp = mkc(0.0f, 0.0f);
    if (a.Cpol) {
      const float2 *Uk = a.UkF + (size_t)kg * NW * NW;
#pragma unroll
      for (int j = 0; j < NW; j++) {
        const float2 w = __ldg(Uk + j * NW + n);
        tp = mkc(fmaf(u[j].x, w.x, fmaf(u[j].y, w.y, tp.x)), fmaf(u[j].x, w.y, fmaf(-u[j].y, w.x, tp.y)));
      }
    }
    const float fm = fermi_fast(em - a.EF, a.invkT);
    const float ems = em * a.sc;
#pragma unroll
    for (int nu = 0; nu < NM; nu++) {
      cx<float> g = mkc(0.0f, 0.0f);
#pragma unroll
      for (int al = 0; al < NM; al++) {
        const float2 e = __ldg(a.ET + ((size_t)al * NM + nu) * a.nq + qq);
        g = mkc(fmaf(e.x, t[al].x, fmaf(-e.y, t[al].y, g.x)), fmaf(e.x, t[al].y, fmaf(e.y, t[al].x, g.y)));
      }
      if (a.Cpol) {
        const float2 c = __ldg(a.Cpol + (size_t)nu * a.nq + qq);
        g = mkc(g.x - fmaf(c.x, tp.y, c.y * tp.x), g.y + fmaf(c.x, tp.x, -c.y * tp.y));
      }
      const bool keep = (om[nu] >= a.omega_min) && (om[nu] > 0.0f);
      const float ws = om[nu] * a.sc;
      const float xp = eks - ems + ws, xm = eks - ems - ws;
      const float cp = keep ? nb[nu] + fm : 0.0f, cm = keep ? nb[nu] + 1.0f - fm : 0.0f;
      const float d = cp * ex2_approx(-xp * xp) + cm * ex2_approx(-xm * xm);
      acc = fmaf(fmaf(g.x, g.x, g.y * g.y), d, acc);
    }
  }
  return acc;
}

// --------------------------------------------------------------- kernel
// KIND 0: kernel E (H(k+q), eigensolve); KIND 1: kernel G (vertex, linewidth terms).
template <int OP, int NW, int NM, int KIND>
__global__ void __launch_bounds__(nthreads<KIND>(), 1)
    k_tcw(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
          const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, TcwArgs a) {
  using O = WOp<OP>;
  using S = WShape<NW, NM>;
  constexpr int BN = w_bn<NW, NM, KIND>();
  constexpr int UNITS = w_units<NW, NM, KIND>();
  constexpr int UCOLS = KIND == 0 ? S::CPK : S::ENTP;
  constexpr int RB = w_rowb<KIND>();
  constexpr int STAGES = w_stages<KIND>();
  constexpr int BK = RB / O::ESZ;  // K elements per stage
  constexpr int A_BYTES = BM * RB;
  constexpr int B_BYTES = BN * RB;
  constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr uint32_t IDESC = w_idesc<OP, BN>();
  __shared__ __align__(8) uint64_t bar_full[STAGES], bar_empty[STAGES], bar_tfull[2], bar_tempty[2], bar_final;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t smem0 = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int *abort_flag = &abort_sh;
  const int nitems = a.ngrp * a.nqt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int s = 0; s < 2; s++) {
      mbar_init(smem_u32(&bar_tfull[s]), 1);
      mbar_init(smem_u32(&bar_tempty[s]), 4 * UNITS);
    }
    mbar_init(smem_u32(&bar_final), 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(&tmem_base_sh), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    int issued[STAGES];
#pragma unroll
    for (int s = 0; s < STAGES; s++) issued[s] = 0;
    uint32_t it = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      int grp, qt;
      w_coords(a, item, grp, qt);
      for (int kb = 0; kb < a.nkb; kb++, it++) {
        const int s = it % STAGES;
        const uint32_t par = ((it / STAGES) & 1u) ^ 1u;
        if (lane == 0) {
          ok = wait_bar(smem_u32(&bar_empty[s]), par, abort_flag, a.dstatus);
          if (ok) {
            const uint32_t base = smem0 + s * STAGE;
            const uint32_t fb = smem_u32(&bar_full[s]);
            mbar_expect_tx(fb, STAGE);
            tma_load_2d(base, &mAhi, kb * BK, qt * BM, fb);
            tma_load_2d(base + A_BYTES, &mAlo, kb * BK, qt * BM, fb);
            tma_load_2d(base + 2 * A_BYTES, &mBhi, kb * BK, grp * BN, fb);
            tma_load_2d(base + 2 * A_BYTES + B_BYTES, &mBlo, kb * BK, grp * BN, fb);
            issued[s] = (int)(it / STAGES) + 1;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int s = 0; s < STAGES; s++)
        if (issued[s] > 0) drain_bar(smem_u32(&bar_full[s]), (uint32_t)((issued[s] - 1) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    uint32_t it = 0;
    int titer = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, titer++) {
      const int ts = titer & 1;
      const uint32_t tpar = ((titer >> 1) & 1) ^ 1;
      if (lane == 0) ok = wait_bar(smem_u32(&bar_tempty[ts]), tpar, abort_flag, a.dstatus);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
      const uint32_t dcol = tmem + ts * 256;
      for (int kb = 0; kb < a.nkb; kb++, it++) {
        const int s = it % STAGES;
        const uint32_t par = (it / STAGES) & 1u;
        if (lane == 0) {
          ok = wait_bar(smem_u32(&bar_full[s]), par, abort_flag, a.dstatus);
          if (ok) {
            tc_fence_after();
            const uint32_t base = smem0 + s * STAGE;
            const uint64_t dAh = sdesc_sw<RB>(base), dAl = sdesc_sw<RB>(base + A_BYTES);
            const uint64_t dBh = sdesc_sw<RB>(base + 2 * A_BYTES), dBl = sdesc_sw<RB>(base + 2 * A_BYTES + B_BYTES);
            const int ksteps = min(BK, a.kpad - kb * BK) / O::KSTEP;
            for (int ks = 0; ks < ksteps; ks++) {
              const uint64_t off = (uint64_t)((ks * 32) >> 4);  // 32 bytes of K per MMA
              const uint32_t acc = (kb == 0 && ks == 0) ? 0u : 1u;
              umma_id<O::F16>(dcol, dAl + off, dBh + off, IDESC, acc);
              umma_id<O::F16>(dcol, dAh + off, dBl + off, IDESC, 1u);
              umma_id<O::F16>(dcol, dAh + off, dBh + off, IDESC, 1u);
            }
            umma_commit(smem_u32(&bar_empty[s]));
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
      }
      if (!ok) break;
      if (lane == 0) umma_commit(smem_u32(&bar_tfull[ts]));
      __syncwarp();
    }
    if (lane == 0) {
      umma_commit(smem_u32(&bar_final));
      drain_bar(smem_u32(&bar_final), 0);
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------------- epilogue
    // Items of a lane quadrant: (tile titer, unit u) in order it = UNITS titer + u,
    // taken round-robin by the quadrant's warps; a tile's accumulator stage is
    // released after all 4 UNITS items.
    constexpr int NG = epi_warps<KIND>() / 4;
    const int quad = warp & 3;
    const int widx = (warp - EPI_WARP0) >> 2;
    for (int it = widx;; it += NG) {
      const int titer = it / UNITS, u = it % UNITS;
      const int item = blockIdx.x + titer * gridDim.x;
      if (item >= nitems) break;
      const int ts = titer & 1;
      const uint32_t tpar = (titer >> 1) & 1;
      const bool ok = wait_bar(smem_u32(&bar_tfull[ts]), tpar, abort_flag, a.dstatus);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      int grp, qt;
      w_coords(a, item, grp, qt);
      const int q = qt * BM + quad * 32 + lane;
      const uint32_t tcol = tmem + ((uint32_t)(quad * 32) << 16) + ts * 256 + u * UCOLS;
      if constexpr (KIND == 0) {
        const int kl = grp * S::KPT + u;
        const bool valid = q < a.nq && kl < a.kc;
        const EigView v{a.epsq + (size_t)(valid ? kl : 0) * NW * a.ldq, a.Uq + (size_t)(valid ? kl : 0) * NW * NW * a.ldq,
                        (size_t)a.ldq, q};
        eig_pair<NW>(a, tcol, q, a.k0 + kl, v, valid);
      } else {
        const int e = grp * S::CN + u;
        const int kl = e / NW, n = e % NW;
        const bool kval = kl < a.kc;
        const bool valid = q < a.nq && kval;
        const EigView ev{a.epsq + (size_t)(kval ? kl : 0) * NW * a.ldq,
                         a.Uq + (size_t)(kval ? kl : 0) * NW * NW * a.ldq, (size_t)a.ldq, q};
        float v = g_entry<NW, NM>(a, tcol, q, a.k0 + kl, n, ev, valid);
        v *= valid ? __ldg(a.wq + q) : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && kval)
          a.partial[((size_t)(a.k0 + kl) * (4 * a.nqt) + qt * 4 + quad) * NW + n] = (double)v * (double)a.gnorm;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_tempty[ts]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ------------------------------------------------------------ fused kernel
// E and G in one persistent kernel, so that the per-pair eigensolve (CUDA cores)
// runs beside the vertex contraction (tensor cores) and the eigen-data stays in
// L2.  Per (k, q tile) item j: the H(k+q) block (N = cpk) into a single tensor-
// memory region, then the vertex chunks (N = bng, two stages).  The MMA order is
// H(0), then for s = 1, 2, ...: H(s), chunks of item s - 1, so that the
// eigensolve of an item overlaps the vertex MMAs of the one before.
//   warp 0      TMA producer (K blocks of 128-byte rows for CTA pairs, 64-byte rows
//               for single CTAs, whose full B rows leave less room per stage)
//   warp 1      tensor memory and MMA issuer
//   warps 2..5  eigensolve of the item's H(k+q), one per lane quadrant; the
//               eigenvalues and reachable eigenvectors go to a per-CTA ring of
//               two slots in global memory (L2-resident), signalled per quadrant
//   warps 6..9  linewidth terms of the vertex chunks, one per lane quadrant
constexpr int F_WARPS = 10;
// Bytes of K per operand row of a stage: 128 (128-byte swizzle, 64 bf16 / 32 tf32 of K, four
// MMA K steps per stage) for CTA pairs, 64 for single CTAs.  The 128-byte rows let the MMAs
// read their operands at a higher rate (measured: the MMA pipeline alone 21 % faster).
template <bool PAIR>
constexpr int f_rb() {
  return PAIR ? 128 : 64;
}

// Operand stages, then per vertex warp its lanes' per-q tables: frequencies and Bose factors
// [2 nm][32], and the first F_EROWS rows a of the mode factors E [a][nu][32] (float2); the
// other rows are read from global memory (L1).  A stage holds the A rows (hi, lo) and the B
// rows (hi, lo) of one K block: all B rows for a single CTA, half of them for a CTA pair (each
// CTA holds half of the MMA's N columns).  Single CTA: four stages (three for 3nat = 9
// modes); pair (twice the K per stage): three.  The operand pipeline wants the third stage more
// than the tables want shared memory (measured, hexagonal nw = 5 with 9 modes: two stages and
// every table in shared memory 112 ms, three stages and E through L1 102 ms).
template <int NM, bool PAIR>
constexpr int f_stages() {
  return PAIR ? 3 : (NM <= 6 ? 4 : 3);
}
template <int NW, int NM, bool PAIR>
constexpr int f_stage_bytes() {
  return (2 * BM + (PAIR ? 1 : 2) * WShape<NW, NM>::BNG) * f_rb<PAIR>();
}
constexpr int F_SMEM_MAX = 232448 - 512;  // dynamic shared memory per CTA, less the static barriers
template <int NW, int NM, bool PAIR>
constexpr int f_erows() {
  constexpr int per_warp = (F_SMEM_MAX - 1024 - f_stages<NM, PAIR>() * f_stage_bytes<NW, NM, PAIR>()) / 4;
  constexpr int rows = (per_warp - 32 * 4 * 2 * NM) / (32 * 8 * NM);
  return rows < NM ? rows : NM;
}
template <int NW, int NM, bool PAIR>
constexpr int f_tab_bytes() {
  return 32 * (4 * 2 * NM + 8 * NM * f_erows<NW, NM, PAIR>());  // per vertex warp
}
template <int NW, int NM, bool PAIR>
constexpr int f_smem() {
  return f_stages<NM, PAIR>() * f_stage_bytes<NW, NM, PAIR>() + 4 * f_tab_bytes<NW, NM, PAIR>() + 1024;
}
// Item -> (k, q tile): one q tile per item for a single CTA; a pair takes two neighbouring
// q tiles per item, rank r the tile 2 u + r (the second may lie past nq: its rows are invalid).
template <bool PAIR>
__device__ __forceinline__ void f_coords(const TcwArgs &a, int item, uint32_t rank, int &kl, int &qt) {
  if constexpr (PAIR) {
    int u;
    w_coords_n((a.nqt + 1) / 2, a.qblock > 1 ? a.qblock / 2 : 1, a.ngrp, item, kl, u);
    qt = 2 * u + (int)rank;
  } else {
    w_coords(a, item, kl, qt);
  }
}

// Linewidth terms of the entries (k, n0) and (k, n0 + 1) of one vertex chunk for the
// warp's 32 pairs (bit m of rel0, rel1: band m reachable for that entry).  Per entry
// (warp-uniform: the entry's tensor-memory columns are one address for the warp) each
// lane walks its own reachable bands, lowest m first, so the warp runs as many rounds
// as its busiest lane needs; each term adds to the entry's sum in ascending m.  em, ek:
// eigenvalues at k+q and band energies at k (registers), tabE / tabW: the lanes' per-q
// tables (rows a < EROWS of E; the others from global memory).
template <int NW, int NM, int EROWS>
__device__ __forceinline__ void g_chunk(const TcwArgs &a, uint32_t tcol, int n0, int qq, int kg, const EigView &v,
                                        const float (&em)[NW], const float (&ek)[NW], uint32_t rel0, uint32_t rel1,
                                        const float2 *tabE, const float *tabW, float &acc0, float &acc1) {
  constexpr int ENT = 2 * NM * NW;
  constexpr int LD = (ENT + 31) / 32 * 32;
  constexpr int ENTP = WShape<NW, NM>::ENTP;
  const int lane = threadIdx.x & 31;
  acc0 = acc1 = 0.0f;
#pragma unroll 1
  for (int e = 0; e < 2; e++) {
    uint32_t need = e == 0 ? rel0 : rel1;
    const int n = n0 + e;
    const float eks = pick<NW>(ek, n < NW ? n : n0) * a.sc;
    float acc = 0.0f;
#pragma unroll 1
    while (__any_sync(0xffffffffu, need != 0)) {
      const bool act = need != 0;
      const int m = act ? __ffs(need) - 1 : 0;
      need &= need - 1;
      cx<float> u[NW];
      {
        const float2 *src = v.U + (size_t)m * NW * v.ld + v.idx;
#pragma unroll
        for (int i = 0; i < NW; i++) {
          const float2 w = act ? src[(size_t)i * v.ld] : make_float2(0.0f, 0.0f);
          u[i] = mkc(w.x, w.y);
        }
      }
      // t_a = u_m^dagger (g_a U_k)_{:, n}: the entry's columns stream from tensor memory
      cx<float> t[NM];
#pragma unroll
      for (int al = 0; al < NM; al++) t[al] = mkc(0.0f, 0.0f);
#pragma unroll
      for (int c0 = 0; c0 < LD; c0 += 32) {
        float xc[32];
        tmem_ld32(tcol + e * ENTP + c0, xc);
#pragma unroll
        for (int cc = 0; cc < 32; cc += 2) {
          const int col = c0 + cc;
          if (col < ENT) {
            const int al = col / (2 * NW), j = (col >> 1) % NW;
            const float br = xc[cc], bi = xc[cc + 1];
            t[al] = mkc(fmaf(u[j].x, br, fmaf(u[j].y, bi, t[al].x)), fmaf(u[j].x, bi, fmaf(-u[j].y, br, t[al].y)));
          }
        }
      }
      if (!act) continue;
      const float emm = pick<NW>(em, m);
      const float fm = fermi_fast(emm - a.EF, a.invkT);
      const float ems = emm * a.sc;
      cx<float> tp = mkc(0.0f, 0.0f);
      if (a.Cpol) {
        const float2 *Uk = a.UkF + (size_t)kg * NW * NW;
#pragma unroll
        for (int j = 0; j < NW; j++) {
          const float2 w = __ldg(Uk + j * NW + n);
          tp = mkc(fmaf(u[j].x, w.x, fmaf(u[j].y, w.y, tp.x)), fmaf(u[j].x, w.y, fmaf(-u[j].y, w.x, tp.y)));
        }
      }
      float accm = 0.0f;
#pragma unroll
      for (int nu = 0; nu < NM; nu++) {
        cx<float> g = mkc(0.0f, 0.0f);
#pragma unroll
        for (int al = 0; al < NM; al++) {
          const float2 ee = al < EROWS ? tabE[(al * NM + nu) * 32 + lane] : __ldg(a.ET + (size_t)(al * NM + nu) * a.nq + qq);
          g = mkc(fmaf(ee.x, t[al].x, fmaf(-ee.y, t[al].y, g.x)), fmaf(ee.x, t[al].y, fmaf(ee.y, t[al].x, g.y)));
        }
        if (a.Cpol) {
          const float2 c = __ldg(a.Cpol + (size_t)nu * a.nq + qq);
          g = mkc(g.x - fmaf(c.x, tp.y, c.y * tp.x), g.y + fmaf(c.x, tp.x, -c.y * tp.y));
        }
        const float om = tabW[nu * 32 + lane], nb = tabW[(NM + nu) * 32 + lane];
        const bool keep = (om >= a.omega_min) && (om > 0.0f);
        const float ws = om * a.sc;
        const float xp = eks - ems + ws, xm = eks - ems - ws;
        const float cp = keep ? nb + fm : 0.0f, cm = keep ? nb + 1.0f - fm : 0.0f;
        const float d = cp * ex2_approx(-xp * xp) + cm * ex2_approx(-xm * xm);
        accm = fmaf(fmaf(g.x, g.x, g.y * g.y), d, accm);
      }
      acc += accm;
    }
    if (e == 0)
      acc0 = acc;
    else
      acc1 = acc;
  }
}

template <int OP, int NW, int NM, bool PAIR>
__global__ void __launch_bounds__(32 * F_WARPS, 1)
    k_tcwf(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
           const __grid_constant__ CUtensorMap mEhi, const __grid_constant__ CUtensorMap mElo,
           const __grid_constant__ CUtensorMap mAGhi, const __grid_constant__ CUtensorMap mAGlo,
           const __grid_constant__ CUtensorMap mGhi, const __grid_constant__ CUtensorMap mGlo, TcwArgs a) {
  using O = WOp<OP>;
  using S = WShape<NW, NM>;
  constexpr int F_STAGES = f_stages<NM, PAIR>();
  constexpr int F_RB = f_rb<PAIR>();
  constexpr int BK = F_RB / O::ESZ;
  constexpr int CPK = S::CPK, BNG = S::BNG, CN = S::CN;
  static_assert(CN == 2, "vertex chunks of two entries");
  constexpr int NCH = (NW + CN - 1) / CN;  // vertex chunks per k
  constexpr int A_BYTES = BM * F_RB;
  constexpr int STAGE = f_stage_bytes<NW, NM, PAIR>();
  constexpr int BROWS = PAIR ? BNG / 2 : BNG;  // B rows of a stage held by this CTA
  constexpr uint32_t ID_H = PAIR ? w_idesc_pair<OP, CPK>() : w_idesc<OP, CPK>();
  constexpr uint32_t ID_G = PAIR ? w_idesc_pair<OP, BNG>() : w_idesc<OP, BNG>();
  // odd nw: the last chunk holds one entry, so its MMAs take N = ENTP (no all-zero entry)
  constexpr bool ODD = NW % CN != 0;
  constexpr uint32_t ID_G1 = PAIR ? w_idesc_pair<OP, S::ENTP>() : w_idesc<OP, S::ENTP>();
  static_assert(!PAIR || (CPK % 32 == 0 && BNG % 32 == 0 && S::ENTP % 32 == 0),
                "a pair's MMA splits N in halves of 16-column multiples");
  constexpr uint32_t GCOL0 = CPK;  // tensor-memory columns: H [0, cpk), vertex stages cpk + s bng
  static_assert(CPK + 2 * BNG <= 512, "tensor memory");
  static_assert(f_smem<NW, NM, PAIR>() <= F_SMEM_MAX && f_erows<NW, NM, PAIR>() >= 0, "shared memory");
  __shared__ __align__(8) uint64_t bar_full[F_STAGES], bar_empty[F_STAGES], bar_hfull, bar_hempty, bar_gfull[2],
      bar_gempty[2], bar_efull[2][4], bar_eempty[2][4], bar_final;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t smem0 = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int *abort_flag = &abort_sh;
  // a pair (cluster of two CTAs) shares each item: the leader (rank 0) issues the MMAs for
  // both, the epilogue warps of both arrive on the leader's tensor-memory barriers
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const bool leader = rank == 0;
  const int cid = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int ncl = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  const int nitems = a.ngrp * (PAIR ? (a.nqt + 1) / 2 : a.nqt);
  const int nmy = nitems > cid ? (nitems - 1 - cid) / ncl + 1 : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < F_STAGES; s++) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_hfull), 1);
    mbar_init(smem_u32(&bar_hempty), PAIR ? 8 : 4);
    for (int s = 0; s < 2; s++) {
      mbar_init(smem_u32(&bar_gfull[s]), 1);
      mbar_init(smem_u32(&bar_gempty[s]), PAIR ? 8 : 4);
      for (int qd = 0; qd < 4; qd++) {
        mbar_init(smem_u32(&bar_efull[s][qd]), 1);
        mbar_init(smem_u32(&bar_eempty[s][qd]), 1);
      }
    }
    mbar_init(smem_u32(&bar_final), 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      tmem_alloc_pair(smem_u32(&tmem_base_sh), TMEM_COLS);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(&tmem_base_sh), TMEM_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();  // both CTAs' barriers and tensor memory exist
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  // the leader's barriers that the pair's loads and epilogue warps signal
  const uint32_t full_c0 = PAIR ? cluster_addr(smem_u32(&bar_full[0]), 0) : smem_u32(&bar_full[0]);
  const uint32_t hempty_c = PAIR ? cluster_addr(smem_u32(&bar_hempty), 0) : smem_u32(&bar_hempty);
  const uint32_t gempty_c0 = PAIR ? cluster_addr(smem_u32(&bar_gempty[0]), 0) : smem_u32(&bar_gempty[0]);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    int issued[F_STAGES];
#pragma unroll
    for (int s = 0; s < F_STAGES; s++) issued[s] = 0;
    uint32_t it = 0;
    bool ok = true;
    // one group: the A rows of q tile qt (ah, al) and the B boxes (brows rows for the pair,
    // hi and lo) from row0, nkb K blocks; rank r of a pair loads its box from row0 + r hoff
    auto load_group = [&](int qt, const CUtensorMap *ah, const CUtensorMap *al, const CUtensorMap *bh,
                          const CUtensorMap *bl, int row0, uint32_t brows, int hoff, int nkb) {
      for (int kb = 0; kb < nkb && ok; kb++, it++) {
        const int s = it % F_STAGES;
        const uint32_t par = ((it / F_STAGES) & 1u) ^ 1u;
        if (lane == 0) {
          ok = wait_bar(smem_u32(&bar_empty[s]), par, abort_flag, a.dstatus);
          if (ok) {
            const uint32_t base = smem0 + s * STAGE;
            if constexpr (PAIR) {
              // this CTA's A tile and its half of the B rows; the leader's barrier counts
              // the bytes of both CTAs
              const uint32_t fb = full_c0 + 8u * (uint32_t)s;
              if (leader) mbar_expect_tx(smem_u32(&bar_full[s]), 2 * (2 * A_BYTES + brows * F_RB));
              const int hrow = row0 + (int)rank * hoff;
              tma_load_2d_pair(base, ah, kb * BK, qt * BM, fb);
              tma_load_2d_pair(base + A_BYTES, al, kb * BK, qt * BM, fb);
              tma_load_2d_pair(base + 2 * A_BYTES, bh, kb * BK, hrow, fb);
              tma_load_2d_pair(base + 2 * A_BYTES + BROWS * F_RB, bl, kb * BK, hrow, fb);
            } else {
              const uint32_t fb = smem_u32(&bar_full[s]);
              mbar_expect_tx(fb, 2 * A_BYTES + 2 * brows * F_RB);
              tma_load_2d(base, ah, kb * BK, qt * BM, fb);
              tma_load_2d(base + A_BYTES, al, kb * BK, qt * BM, fb);
              tma_load_2d(base + 2 * A_BYTES, bh, kb * BK, row0, fb);
              tma_load_2d(base + 2 * A_BYTES + BNG * F_RB, bl, kb * BK, row0, fb);
            }
            issued[s] = (int)(it / F_STAGES) + 1;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
      }
    };
    for (int st = 0; st <= nmy && ok; st++) {
      if (st < nmy) {
        int kl, qt;
        f_coords<PAIR>(a, cid + st * ncl, rank, kl, qt);
        load_group(qt, &mAhi, &mAlo, &mEhi, &mElo, kl * CPK, CPK, CPK / 2, a.nkb);
      }
      if (st >= 1) {
        int kl, qt;
        f_coords<PAIR>(a, cid + (st - 1) * ncl, rank, kl, qt);
        for (int c = 0; c < NCH && ok; c++)
          load_group(qt, &mAGhi, &mAGlo, &mGhi, &mGlo, (kl * NCH + c) * BNG, BNG,
                     (ODD && c == NCH - 1 ? S::ENTP : BNG) / 2, a.nkbG);
      }
    }
    if (lane == 0 && leader) {  // (a pair's loads complete on the leader's barriers)
#pragma unroll
      for (int s = 0; s < F_STAGES; s++)
        if (issued[s] > 0) drain_bar(smem_u32(&bar_full[s]), (uint32_t)((issued[s] - 1) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    uint32_t it = 0;
    int hcount = 0, gcount = 0;
    bool ok = true;
    auto mma_group = [&](uint32_t dcol, uint32_t idesc, int nkb, int kpad) {
      for (int kb = 0; kb < nkb && ok; kb++, it++) {
        const int s = it % F_STAGES;
        const uint32_t par = (it / F_STAGES) & 1u;
        if (lane == 0) {
          ok = wait_bar(smem_u32(&bar_full[s]), par, abort_flag, a.dstatus);
          if (ok) {
            tc_fence_after();
            const uint32_t base = smem0 + s * STAGE;
            const uint64_t dAh = sdesc_sw<F_RB>(base), dAl = sdesc_sw<F_RB>(base + A_BYTES);
            const uint64_t dBh = sdesc_sw<F_RB>(base + 2 * A_BYTES);
            const uint64_t dBl = sdesc_sw<F_RB>(base + 2 * A_BYTES + BROWS * F_RB);
            const int ksteps = min(BK, kpad - kb * BK) / O::KSTEP;
            for (int ks = 0; ks < ksteps; ks++) {
              const uint64_t off = (uint64_t)((ks * 32) >> 4);
              const uint32_t acc = (kb == 0 && ks == 0) ? 0u : 1u;
              if constexpr (PAIR) {
                umma_pair<O::F16>(dcol, dAl + off, dBh + off, idesc, acc);
                umma_pair<O::F16>(dcol, dAh + off, dBl + off, idesc, 1u);
                umma_pair<O::F16>(dcol, dAh + off, dBh + off, idesc, 1u);
              } else {
                umma_id<O::F16>(dcol, dAl + off, dBh + off, idesc, acc);
                umma_id<O::F16>(dcol, dAh + off, dBl + off, idesc, 1u);
                umma_id<O::F16>(dcol, dAh + off, dBh + off, idesc, 1u);
              }
            }
            if constexpr (PAIR)
              umma_commit_pair(smem_u32(&bar_empty[s]));
            else
              umma_commit(smem_u32(&bar_empty[s]));
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
      }
    };
    auto commit = [&](uint32_t bar) {
      if constexpr (PAIR)
        umma_commit_pair(bar);
      else
        umma_commit(bar);
    };
    // a pair's second CTA issues no MMAs: the leader's land in both CTAs' tensor memory
    for (int st = 0; st <= nmy && ok && leader; st++) {
      if (st < nmy) {
        if (lane == 0) ok = wait_bar(smem_u32(&bar_hempty), (uint32_t)((hcount & 1) ^ 1), abort_flag, a.dstatus);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        tc_fence_after();
        mma_group(tmem, ID_H, a.nkb, a.kpad);
        if (!ok) break;
        if (lane == 0) commit(smem_u32(&bar_hfull));
        __syncwarp();
        hcount++;
      }
      if (st >= 1) {
        for (int c = 0; c < NCH && ok; c++, gcount++) {
          const int gs = gcount & 1;
          if (lane == 0)
            ok = wait_bar(smem_u32(&bar_gempty[gs]), (uint32_t)(((gcount >> 1) & 1) ^ 1), abort_flag, a.dstatus);
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) break;
          tc_fence_after();
          mma_group(tmem + GCOL0 + gs * BNG, ODD && c == NCH - 1 ? ID_G1 : ID_G, a.nkbG, a.kpadG);
          if (!ok) break;
          if (lane == 0) commit(smem_u32(&bar_gfull[gs]));
          __syncwarp();
        }
      }
    }
    if (lane == 0 && leader) {
      commit(smem_u32(&bar_final));
      drain_bar(smem_u32(&bar_final), 0);  // every MMA (into both CTAs' tensor memory) is complete
    }
    __syncwarp();
  } else if (warp < 6) {
    // --------------------------------------------------------- eigensolve
    const int quad = warp & 3;
    const int idx = quad * 32 + lane;
    for (int j = 0; j < nmy; j++) {
      int kl, qt;
      f_coords<PAIR>(a, cid + j * ncl, rank, kl, qt);
      const int q = qt * BM + idx;
      const bool valid = q < a.nq && kl < a.kc;
      bool ok = wait_bar(smem_u32(&bar_hfull), (uint32_t)(j & 1), abort_flag, a.dstatus);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const int slot = j & 1;
      const size_t so = ((size_t)blockIdx.x * 2 + slot);
      const EigView v{a.epsq + so * NW * BM, a.Uq + so * NW * NW * BM, (size_t)BM, idx};
      ok = eig_pair<NW, true>(a, tmem + ((uint32_t)(quad * 32) << 16), q, a.k0 + kl, v, valid, hempty_c,
                              smem_u32(&bar_eempty[slot][quad]), (uint32_t)(((j >> 1) & 1) ^ 1), abort_flag, PAIR);
      if (!ok) break;
      __threadfence_block();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_efull[slot][quad]));
    }
  } else {
    // ------------------------------------------------------- vertex terms
    const int quad = warp & 3;
    const int idx = quad * 32 + lane;
    // this warp's per-q tables in shared memory (after the operand stages)
    constexpr int EROWS = f_erows<NW, NM, PAIR>();
    uint8_t *tab = smem_raw + (smem0 - smem_u32(smem_raw)) + F_STAGES * STAGE + (warp - 6) * f_tab_bytes<NW, NM, PAIR>();
    const float2 *tabE = reinterpret_cast<const float2 *>(tab);
    const float *tabW = reinterpret_cast<const float *>(tab + 32 * 8 * NM * EROWS);
    const uint32_t tabE_s = smem_u32(tab), tabW_s = tabE_s + 32 * 8 * NM * EROWS;
    int gcount = 0;
    bool ok = true;
    for (int j = 0; j < nmy && ok; j++) {
      int kl, qt;
      f_coords<PAIR>(a, cid + j * ncl, rank, kl, qt);
      const int q = qt * BM + idx;
      const bool kval = kl < a.kc && qt < a.nqt;
      const bool valid = q < a.nq && kval;
      const int qq = valid ? q : 0;
      const int kg = kval ? a.k0 + kl : 0;
      // per-q tables of the item's rows: E [EROWS][nm] complex, w [nm], n [nm]
      __syncwarp();
#pragma unroll 1
      for (int e = 0; e < EROWS * NM; e++) cp_async8(tabE_s + 8u * (e * 32 + lane), a.ET + (size_t)e * a.nq + qq);
#pragma unroll 1
      for (int nu = 0; nu < NM; nu++) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tabW_s + 4u * (nu * 32 + lane)),
                     "l"(__cvta_generic_to_global(a.omegaT + (size_t)nu * a.nq + qq))
                     : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tabW_s + 4u * ((NM + nu) * 32 + lane)),
                     "l"(__cvta_generic_to_global(a.nbT + (size_t)nu * a.nq + qq))
                     : "memory");
      }
      const float wqv = valid ? __ldg(a.wq + q) : 0.0f;
      const float thr = valid ? __ldg(a.thr + q) : -1.0f;
      float ek[NW];
#pragma unroll
      for (int n = 0; n < NW; n++) ek[n] = __ldg(a.epsk + (size_t)kg * NW + n);
      const int slot = j & 1;
      const size_t so = ((size_t)blockIdx.x * 2 + slot);
      const EigView v{a.epsq + so * NW * BM, a.Uq + so * NW * NW * BM, (size_t)BM, idx};
      ok = wait_bar(smem_u32(&bar_efull[slot][quad]), (uint32_t)((j >> 1) & 1), abort_flag, a.dstatus);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        cp_async_wait_all();
        break;
      }
      // eigenvalues at k+q and the reachable (m, n) as 8-bit masks per n
      float em[NW];
#pragma unroll
      for (int m = 0; m < NW; m++) em[m] = valid ? v.eps[(size_t)m * v.ld + v.idx] : 0.0f;
      uint32_t rel[NW];
#pragma unroll
      for (int n = 0; n < NW; n++) {
        rel[n] = 0;
#pragma unroll
        for (int m = 0; m < NW; m++)
          if (valid && reachable(ek[n], em[m], thr)) rel[n] |= 1u << m;
      }
      cp_async_wait_all();
      __syncwarp();
      for (int c = 0; c < NCH; c++, gcount++) {
        const int gs = gcount & 1;
        ok = wait_bar(smem_u32(&bar_gfull[gs]), (uint32_t)((gcount >> 1) & 1), abort_flag, a.dstatus);
        if (!__all_sync(0xffffffffu, ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tcol = tmem + ((uint32_t)(quad * 32) << 16) + GCOL0 + gs * BNG;
        const int n0 = c * CN;
        uint32_t r0 = 0, r1 = 0;  // rel[n0], rel[n0 + 1] by masks (keeps rel in registers)
#pragma unroll
        for (int n = 0; n < NW; n++) {
          r0 |= rel[n] & (0u - (uint32_t)(n == n0));
          r1 |= rel[n] & (0u - (uint32_t)(n == n0 + 1));
        }
        float acc0, acc1;
        g_chunk<NW, NM, EROWS>(a, tcol, n0, qq, kg, v, em, ek, r0, r1, tabE, tabW, acc0, acc1);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if constexpr (PAIR)
            mbar_arrive_cluster(gempty_c0 + 8u * (uint32_t)gs);
          else
            mbar_arrive(smem_u32(&bar_gempty[gs]));
        }
        float v0 = acc0 * wqv, v1 = acc1 * wqv;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          v0 += __shfl_down_sync(0xffffffffu, v0, o);
          v1 += __shfl_down_sync(0xffffffffu, v1, o);
        }
        if (lane == 0 && kval) {
          double *dst = a.partial + ((size_t)(a.k0 + kl) * (4 * a.nqt) + qt * 4 + quad) * NW;
          dst[n0] = (double)v0 * (double)a.gnorm;
          if (n0 + 1 < NW) dst[n0 + 1] = (double)v1 * (double)a.gnorm;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_eempty[slot][quad]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();  // neither CTA frees tensor memory the pair still uses
  if (warp == 1) {
    tc_fence_after();
    if constexpr (PAIR)
      tmem_dealloc_pair(tmem, TMEM_COLS);
    else
      tmem_dealloc(tmem, TMEM_COLS);
  }
  if constexpr (PAIR) cluster_sync();
}

// ------------------------------------------------------- operand builder G
template <typename T>
__device__ __forceinline__ void wsplit(float v, T *hi, T *lo, size_t i);
template <>
__device__ __forceinline__ void wsplit<__nv_bfloat16>(float v, __nv_bfloat16 *hi, __nv_bfloat16 *lo, size_t i) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[i] = h;
  lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
}
template <>
__device__ __forceinline__ void wsplit<float>(float v, float *hi, float *lo, size_t i) {
  const float h = tf32_rn(v);
  hi[i] = h;
  lo[i] = tf32_rn(v - h);
}

// B rows of the vertex contraction: row = c bng + i entp + 2 (a nw + j) + s for entry
// e = c cn + i = (kl, n) = (e / epk, e % epk) (epk = nw: entries of consecutive k packed;
// epk = cn ceil(nw / cn): each k starts a chunk, entries n >= nw are zero); K index kk = 2 rr + t, R index r = nR - 1 - rr
// (far shells first, as the A operand); value from b = Bg[kl][r][a][j][n]:
//   (s,t) = (0,0): Re b, (0,1): -Im b, (1,0): Im b, (1,1): Re b.
// Rows past 2 nm nw in an entry, entries with kl >= kc and K >= 2 nR are 0.
template <typename T>
__global__ void k_build_bg(int kc, int nchunk, int nR, int nw, int nm, int cn, int entp, int bng, int kpad, int epk,
                           const cx<float> *__restrict__ Bg, T *hi, T *lo) {
  const size_t n = (size_t)nchunk * bng * kpad;
  const int nw2 = nw * nw, ent = 2 * nm * nw;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % kpad);
    const int row = (int)(idx / kpad);
    const int c = row / bng, rc = row % bng;
    const int i = rc / entp, re = rc % entp;
    const int e = c * cn + i;
    const int kl = e / epk, nb = e % epk;
    float v = 0.0f;
    if (re < ent && nb < nw && kl < kc && kk < 2 * nR) {
      const int al = re / (2 * nw), j = (re >> 1) % nw, s = re & 1;
      const int r = nR - 1 - (kk >> 1), t = kk & 1;
      const cx<float> b = Bg[((size_t)kl * nR + r) * nm * nw2 + al * nw2 + j * nw + nb];
      v = s == 0 ? (t == 0 ? b.x : -b.y) : (t == 0 ? b.y : b.x);
    }
    wsplit<T>(v, hi, lo, idx);
  }
}

// thr[q] = max over kept modes of w_q,nu + CUT_SIGMAS sigma (-1 when no mode is kept)
__global__ void k_tcw_thr(int nq, int nm, const float *__restrict__ omF, float omega_min, float cut, float *thr) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    float w = -1.0f;
    for (int nu = 0; nu < nm; nu++) {
      const float o = omF[(size_t)nu * nq + q];
      if (o >= omega_min && o > 0.0f) w = fmaxf(w, o);
    }
    thr[q] = w >= 0.0f ? w + cut : -1.0f;
  }
}

inline int grid_n(size_t n, int bs) {
  size_t b = (n + bs - 1) / bs;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

template <int OP, int NW, int NM, int KIND>
cudaError_t launch_tcw(const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &bh, const CUtensorMap &bl,
                       const TcwArgs &a, cudaStream_t st) {
  constexpr int SMEM = w_smem<NW, NM, KIND>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tcw<OP, NW, NM, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int items = a.ngrp * a.nqt;
  k_tcw<OP, NW, NM, KIND><<<std::min(items, sms), nthreads<KIND>(), SMEM, st>>>(ah, al, bh, bl, a);
  epw_count_launch();
  return cudaGetLastError();
}

template <int OP, int NW, int NM, bool PAIR>
cudaError_t launch_tcwf(const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &eh, const CUtensorMap &el,
                        const CUtensorMap &agh, const CUtensorMap &agl, const CUtensorMap &gh, const CUtensorMap &gl,
                        const TcwArgs &a, int grid, cudaStream_t st) {
  constexpr int SMEM = f_smem<NW, NM, PAIR>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tcwf<OP, NW, NM, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if constexpr (PAIR) {
    // clusters of two CTAs (grid even)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(32 * F_WARPS, 1, 1);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_tcwf<OP, NW, NM, true>, ah, al, eh, el, agh, agl, gh, gl, a);
    epw_count_launch();
    if (e != cudaSuccess) return e;
  } else {
    k_tcwf<OP, NW, NM, false><<<grid, 32 * F_WARPS, SMEM, st>>>(ah, al, eh, el, agh, agl, gh, gl, a);
    epw_count_launch();
  }
  return cudaGetLastError();
}

// compiled (nw, 3nat) pairs
#define EPW_TCW_SHAPES(X) X(8, 6) X(5, 9)

template <int OP, int KIND>
cudaError_t launch_tcw_shape(int nw, int nm, const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &bh,
                             const CUtensorMap &bl, const TcwArgs &a, cudaStream_t st) {
#define EPW_TCW_CASE(W, M) \
  if (nw == W && nm == M) return launch_tcw<OP, W, M, KIND>(ah, al, bh, bl, a, st);
  EPW_TCW_SHAPES(EPW_TCW_CASE)
#undef EPW_TCW_CASE
  return cudaErrorInvalidValue;
}

template <int OP, bool PAIR>
cudaError_t launch_tcwf_shape(int nw, int nm, const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &eh,
                              const CUtensorMap &el, const CUtensorMap &agh, const CUtensorMap &agl,
                              const CUtensorMap &gh, const CUtensorMap &gl, const TcwArgs &a, int grid, cudaStream_t st) {
#define EPW_TCWF_CASE(W, M) \
  if (nw == W && nm == M) return launch_tcwf<OP, W, M, PAIR>(ah, al, eh, el, agh, agl, gh, gl, a, grid, st);
  EPW_TCW_SHAPES(EPW_TCWF_CASE)
#undef EPW_TCWF_CASE
  return cudaErrorInvalidValue;
}

bool tcw_shape(int nw, int nm, int &cpk, int &kpt, int &entp, int &cn, int &bng) {
#define EPW_TCW_INFO(W, M)          \
  if (nw == W && nm == M) {         \
    cpk = WShape<W, M>::CPK;        \
    kpt = WShape<W, M>::KPT;        \
    entp = WShape<W, M>::ENTP;      \
    cn = WShape<W, M>::CN;          \
    bng = WShape<W, M>::BNG;        \
    return true;                    \
  }
  EPW_TCW_SHAPES(EPW_TCW_INFO)
#undef EPW_TCW_INFO
  return false;
}

constexpr size_t TCW_EIG_BYTES = (size_t)6 << 30;  // split kernels: per-chunk eigenvalue + eigenvector buffers
constexpr size_t TCWF_OPERAND_BYTES = (size_t)4 << 30;  // fused kernel: operands of one chunk of k
constexpr int TCWF_MAX_CTAS = 256;  // eigen-data ring slots are laid out for up to this many CTAs

}  // namespace

bool tcw_supported(const epw_model *m) {
  int cpk, kpt, entp, cn, bng;
  return tcw_shape(m->nw, m->nm, cpk, kpt, entp, cn, bng);
}

epw_status tcw_plan(Arena &A, const epw_model *m, int nk, int nq, int op, size_t bytes, TcwBuffers &b, int form) {
  b = TcwBuffers{};
  b.op = op;
  b.ok = tcw_shape(m->nw, m->nm, b.cpk, b.kpt, b.entp, b.cn, b.bng);
  if (!b.ok) return EPW_OK;
  b.fused = form != TCW_FORM_SPLIT;
  b.pair = form == TCW_FORM_PAIR;
  nk = std::max(nk, 1);
  nq = std::max(nq, 1);
  const int nw = m->nw, nm = m->nm;
  const int esz = op == TC_OP_BF16 ? 2 : 4;
  const int kal = op == TC_OP_BF16 ? 16 : 8;
  // K extents: H(k+q) over the Re phases, the vertex over the Rp phases (a second A
  // operand when the sets differ)
  b.kpad = (2 * m->nRe + kal - 1) / kal * kal;
  b.kpadG = (2 * m->nRp + kal - 1) / kal * kal;
  b.nqt = (nq + BM - 1) / BM;
  b.ldq = b.nqt * BM;
  b.Ahi = A.take<char>((size_t)nq * b.kpad * esz);
  b.Alo = A.take<char>((size_t)nq * b.kpad * esz);
  b.AGhi = m->same_ep ? b.Ahi : A.take<char>((size_t)nq * b.kpadG * esz);
  b.AGlo = m->same_ep ? b.Alo : A.take<char>((size_t)nq * b.kpadG * esz);
  if (b.fused) {
    // one k per item: its H(k+q) rows, then its vertex chunks (each k starts a chunk)
    const int nch = (nw + b.cn - 1) / b.cn;
    const size_t per_k = ((size_t)b.cpk * b.kpad + (size_t)nch * b.bng * b.kpadG) * esz * 2;
    b.kc = (int)std::min<size_t>((size_t)nk, std::max<size_t>(1, (bytes ? bytes : TCWF_OPERAND_BYTES) / per_k));
    b.BEhi = A.take<char>((size_t)b.kc * b.cpk * b.kpad * esz);
    b.BElo = A.take<char>((size_t)b.kc * b.cpk * b.kpad * esz);
    b.BGhi = A.take<char>((size_t)b.kc * nch * b.bng * b.kpadG * esz);
    b.BGlo = A.take<char>((size_t)b.kc * nch * b.bng * b.kpadG * esz);
    // eigen-data ring: [cta][slot][nw][128] eigenvalues, [cta][slot][nw][nw][128] eigenvectors
    b.epsq = A.take<float>((size_t)TCWF_MAX_CTAS * 2 * nw * BM);
    b.Uq = A.take<float2>((size_t)TCWF_MAX_CTAS * 2 * nw * nw * BM);
  } else {
    const size_t per_k = (size_t)b.ldq * nw * (4 + 8 * (size_t)nw);
    const size_t budget = bytes ? bytes : TCW_EIG_BYTES;
    b.kc = (int)std::min<size_t>((size_t)nk, std::max<size_t>(1, budget / per_k));
    const int kc_pad = (b.kc + b.kpt - 1) / b.kpt * b.kpt;
    const int nchunk = (b.kc * nw + b.cn - 1) / b.cn;
    b.BEhi = A.take<char>((size_t)kc_pad * b.cpk * b.kpad * esz);
    b.BElo = A.take<char>((size_t)kc_pad * b.cpk * b.kpad * esz);
    b.BGhi = A.take<char>((size_t)nchunk * b.bng * b.kpadG * esz);
    b.BGlo = A.take<char>((size_t)nchunk * b.bng * b.kpadG * esz);
    b.epsq = A.take<float>((size_t)b.kc * nw * b.ldq);
    b.Uq = A.take<float2>((size_t)b.kc * nw * nw * b.ldq);
  }
  b.nbT = A.take<float>((size_t)nq * nm);
  b.omF = A.take<float>((size_t)nq * nm);
  b.wqF = A.take<float>((size_t)nq);
  b.ekF = A.take<float>((size_t)nk * nw);
  b.thr = A.take<float>((size_t)nq);
  b.partial = A.take<double>((size_t)nk * 4 * b.nqt * nw);
  b.UkF = m->polar ? A.take<float2>((size_t)nk * nw * nw) : nullptr;
  return EPW_OK;
}

epw_status tcw_linewidth(const epw_model *m, int nk, int nq, const double *q, const double *wq,
                         const epw_params *par, const double *epsk, const double *omegaT, const cx<float> *ET32,
                         const cx<float> *Bg32, const cx<float> *BH32, const cx<double> *P64,
                         const cx<double> *Uk, const float2 *Cpol, TcwBuffers &b, double *out, cudaStream_t st) {
  if (!b.ok) return EPW_ERR_UNSUPPORTED;
  const int nw = m->nw, nm = m->nm, nR = m->nRe, nRp = m->nRp, op = b.op;
  const int esz = op == TC_OP_BF16 ? 2 : 4;
  tc_build_a_raw(op, nq, nR, b.kpad, q, m->Re, P64, b.Ahi, b.Alo, st);
  if (!m->same_ep) tc_build_a_raw(op, nq, nRp, b.kpadG, q, m->Rp, nullptr, b.AGhi, b.AGlo, st);
  tc_tables(nq, nm, nk, nw, omegaT, par->T_K, wq, epsk, b.nbT, b.omF, b.wqF, b.ekF, st);
  const float cut = (float)(CUT_SIGMAS * par->sigma_eV);
  k_tcw_thr<<<grid_n(nq, 256), 256, 0, st>>>(nq, nm, b.omF, (float)par->omega_min_eV, cut, b.thr);
  epw_count_launch();
  if (Cpol) launch_cast_c64_to_c32((size_t)nk * nw * nw, Uk, (cx<float> *)b.UkF, st);
  TcwArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nq = nq;
  a.nqt = b.nqt;
  a.kpad = b.kpad;
  a.kpadG = b.kpadG;
  const int nkb_e = (b.kpad * esz + 127) / 128, nkb_g = (b.kpadG * esz + 63) / 64;
  a.ldq = b.ldq;
  a.epsk = b.ekF;
  a.thr = b.thr;
  a.omegaT = b.omF;
  a.nbT = b.nbT;
  a.ET = (const float2 *)ET32;
  a.wq = b.wqF;
  a.EF = (float)par->EF_eV;
  a.invkT = par->T_K > 0.0 ? (float)(1.0 / (EPW_KB * par->T_K)) : 0.0f;
  a.sc = (float)(1.2011224087864498 / par->sigma_eV);  // sqrt(log2 e) / sigma
  a.gnorm = (float)(1.0 / (par->sigma_eV * 1.7724538509055160273));
  a.omega_min = (float)par->omega_min_eV;
  a.epsq = b.epsq;
  a.Uq = b.Uq;
  a.partial = b.partial;
  a.dstatus = m->dstatus;
  a.Cpol = Cpol;
  a.UkF = Cpol ? b.UkF : nullptr;
  {
    const size_t atile = (size_t)BM * b.kpad * esz * 2;
    int qb = (int)(A_BLOCK_BYTES / atile);
    qb = std::max(qb, 152);
    a.qblock = std::max(1, std::min(qb, b.nqt));
  }
  if (b.fused) {
    const int nch = (nw + b.cn - 1) / b.cn;
    CUtensorMap ah, al, eh, el, agh, agl, gh, gl;
    // a CTA pair loads half of the B rows in each CTA
    const uint32_t ebox = b.pair ? (uint32_t)b.cpk / 2 : (uint32_t)b.cpk;
    const uint32_t gbox = b.pair ? (uint32_t)b.bng / 2 : (uint32_t)b.bng;
    const int rb = b.pair ? f_rb<true>() : f_rb<false>();
    if (!tc_make_map_rb(&ah, b.Ahi, op, b.kpad, nq, BM, rb) || !tc_make_map_rb(&al, b.Alo, op, b.kpad, nq, BM, rb) ||
        !tc_make_map_rb(&agh, b.AGhi, op, b.kpadG, nq, BM, rb) ||
        !tc_make_map_rb(&agl, b.AGlo, op, b.kpadG, nq, BM, rb) ||
        !tc_make_map_rb(&eh, b.BEhi, op, b.kpad, (uint64_t)b.kc * b.cpk, ebox, rb) ||
        !tc_make_map_rb(&el, b.BElo, op, b.kpad, (uint64_t)b.kc * b.cpk, ebox, rb) ||
        !tc_make_map_rb(&gh, b.BGhi, op, b.kpadG, (uint64_t)b.kc * nch * b.bng, gbox, rb) ||
        !tc_make_map_rb(&gl, b.BGlo, op, b.kpadG, (uint64_t)b.kc * nch * b.bng, gbox, rb))
      return EPW_ERR_CUDA;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sms = std::min(sms, TCWF_MAX_CTAS);
    a.nkb = (b.kpad * esz + rb - 1) / rb;
    a.nkbG = (b.kpadG * esz + rb - 1) / rb;
    const size_t nw2 = (size_t)nw * nw;
    epw_model *mm = const_cast<epw_model *>(m);
    for (int k0 = 0; k0 < nk; k0 += b.kc) {
      const int kc = std::min(b.kc, nk - k0);
      tc_build_b_raw(op, kc, kc, nR, nw, 0, b.cpk, b.kpad, BH32 + (size_t)k0 * nR * nw2, nullptr, b.BEhi, b.BElo, st);
      {
        const int nchunk = kc * nch;
        const size_t n = (size_t)nchunk * b.bng * b.kpadG;
        const cx<float> *bg = Bg32 + (size_t)k0 * nRp * nm * nw2;
        if (op == TC_OP_BF16)
          k_build_bg<__nv_bfloat16><<<grid_n(n, 256), 256, 0, st>>>(kc, nchunk, nRp, nw, nm, b.cn, b.entp, b.bng,
                                                                    b.kpadG, nch * b.cn, bg, (__nv_bfloat16 *)b.BGhi,
                                                                    (__nv_bfloat16 *)b.BGlo);
        else
          k_build_bg<float><<<grid_n(n, 256), 256, 0, st>>>(kc, nchunk, nRp, nw, nm, b.cn, b.entp, b.bng, b.kpadG,
                                                            nch * b.cn, bg, (float *)b.BGhi, (float *)b.BGlo);
        epw_count_launch();
      }
      a.k0 = k0;
      a.kc = kc;
      a.ngrp = kc;
      epw_timing_begin_tag(mm, st, 0);
      cudaError_t e;
      if (b.pair) {
        // clusters of two CTAs, each cluster two q tiles of one k per item
        const int grid = 2 * (int)std::min<long>((long)kc * ((b.nqt + 1) / 2), (long)(sms / 2));
        e = op == TC_OP_BF16 ? launch_tcwf_shape<TC_OP_BF16, true>(nw, nm, ah, al, eh, el, agh, agl, gh, gl, a, grid, st)
                             : launch_tcwf_shape<TC_OP_TF32, true>(nw, nm, ah, al, eh, el, agh, agl, gh, gl, a, grid, st);
      } else {
        const int grid = (int)std::min<long>((long)kc * b.nqt, (long)sms);
        e = op == TC_OP_BF16 ? launch_tcwf_shape<TC_OP_BF16, false>(nw, nm, ah, al, eh, el, agh, agl, gh, gl, a, grid, st)
                             : launch_tcwf_shape<TC_OP_TF32, false>(nw, nm, ah, al, eh, el, agh, agl, gh, gl, a, grid, st);
      }
      epw_timing_end(mm, st);
      if (e != cudaSuccess) return EPW_ERR_CUDA;
    }
    launch_finalize(nk, 4 * b.nqt, nw, b.partial, out, st);
    return cudaGetLastError() == cudaSuccess ? EPW_OK : EPW_ERR_CUDA;
  }
  CUtensorMap ah, al, eh, el, gh, gl;
  CUtensorMap ah64, al64;
  if (!tc_make_map(&ah, b.Ahi, op, b.kpad, nq, BM) || !tc_make_map(&al, b.Alo, op, b.kpad, nq, BM) ||
      !tc_make_map_rb(&ah64, b.AGhi, op, b.kpadG, nq, BM, 64) ||
      !tc_make_map_rb(&al64, b.AGlo, op, b.kpadG, nq, BM, 64))
    return EPW_ERR_CUDA;
  const int kc_pad = (b.kc + b.kpt - 1) / b.kpt * b.kpt;
  const int nchunk_max = (b.kc * nw + b.cn - 1) / b.cn;
  if (!tc_make_map(&eh, b.BEhi, op, b.kpad, (uint64_t)kc_pad * b.cpk, 256) ||
      !tc_make_map(&el, b.BElo, op, b.kpad, (uint64_t)kc_pad * b.cpk, 256) ||
      !tc_make_map_rb(&gh, b.BGhi, op, b.kpadG, (uint64_t)nchunk_max * b.bng, (uint32_t)b.bng, 64) ||
      !tc_make_map_rb(&gl, b.BGlo, op, b.kpadG, (uint64_t)nchunk_max * b.bng, (uint32_t)b.bng, 64))
    return EPW_ERR_CUDA;
  const size_t nw2 = (size_t)nw * nw;
  epw_model *mm = const_cast<epw_model *>(m);
  for (int k0 = 0; k0 < nk; k0 += b.kc) {
    const int kc = std::min(b.kc, nk - k0);
    const int kcp = (kc + b.kpt - 1) / b.kpt * b.kpt;
    const int nchunk = (kc * nw + b.cn - 1) / b.cn;
    tc_build_b_raw(op, kc, kcp, nR, nw, 0, b.cpk, b.kpad, BH32 + (size_t)k0 * nR * nw2, nullptr, b.BEhi, b.BElo, st);
    {
      const size_t n = (size_t)nchunk * b.bng * b.kpadG;
      const cx<float> *bg = Bg32 + (size_t)k0 * nRp * nm * nw2;
      if (op == TC_OP_BF16)
        k_build_bg<__nv_bfloat16><<<grid_n(n, 256), 256, 0, st>>>(kc, nchunk, nRp, nw, nm, b.cn, b.entp, b.bng,
                                                                  b.kpadG, nw, bg, (__nv_bfloat16 *)b.BGhi,
                                                                  (__nv_bfloat16 *)b.BGlo);
      else
        k_build_bg<float><<<grid_n(n, 256), 256, 0, st>>>(kc, nchunk, nRp, nw, nm, b.cn, b.entp, b.bng, b.kpadG, nw,
                                                          bg, (float *)b.BGhi, (float *)b.BGlo);
      epw_count_launch();
    }
    a.k0 = k0;
    a.kc = kc;
    cudaError_t e;
    a.ngrp = kcp / b.kpt;
    a.nkb = nkb_e;
    a.kpad = b.kpad;
    epw_timing_begin_tag(mm, st, 1);
    e = op == TC_OP_BF16 ? launch_tcw_shape<TC_OP_BF16, 0>(nw, nm, ah, al, eh, el, a, st)
                         : launch_tcw_shape<TC_OP_TF32, 0>(nw, nm, ah, al, eh, el, a, st);
    epw_timing_end(mm, st);
    if (e != cudaSuccess) return EPW_ERR_CUDA;
    a.ngrp = nchunk;
    a.nkb = nkb_g;
    a.kpad = b.kpadG;
    epw_timing_begin_tag(mm, st, 0);
    e = op == TC_OP_BF16 ? launch_tcw_shape<TC_OP_BF16, 1>(nw, nm, ah64, al64, gh, gl, a, st)
                         : launch_tcw_shape<TC_OP_TF32, 1>(nw, nm, ah64, al64, gh, gl, a, st);
    epw_timing_end(mm, st);
    if (e != cudaSuccess) return EPW_ERR_CUDA;
  }
  launch_finalize(nk, 4 * b.nqt, nw, b.partial, out, st);
  return cudaGetLastError() == cudaSuccess ? EPW_OK : EPW_ERR_CUDA;
}
