// Fused linewidth kernel on the 5th-generation tensor cores (sm_103a).
//
// Per (k,q) pair the interpolation contraction (EPW, Sec. "Electron-phonon
// coupling in polar materials", step iii, with the U rotations of the overlap
// equation there) is a complex GEMM over the real-space index R:
//
//   C[q][c] = sum_R P_q(R) B_k[R][c],   c = (H(k+q)_ij | (g_a(k,q) U_k)_jn)
//
// with P_q(R) = e^{2 pi i q.R}.  It runs as a real GEMM with K = 2 nR (re/im
// interleaved) on tcgen05.  Each operand is split into two terms x = hi + lo
// and three MMAs (lo*hi + hi*lo + hi*hi) accumulate in FP32 in tensor memory:
//   OP_BF16: bfloat16 terms, kind::f16   (about 2^-17 relative per product)
//   OP_TF32: tf32 terms,     kind::tf32  (about 2^-21 relative per product)
// The epilogue of each 128 x 256 tile (128 q rows x a group of k) is the
// per-pair work of Eq. (linewidthel): a Jacobi eigensolve of H(k+q), the mode
// projection with e_q / sqrt(2 M w), the U_k+q^dagger rotation, |g|^2, the
// Gaussian deltas and occupations, summed over each warp's 32 q rows.
//
// CTA layout (persistent, one CTA per SM):
//   warp 0      TMA producer (A = q-phase tile, B = k-vertex tile, 2 stages)
//   warp 1      TMEM allocator and MMA issuer (one elected thread)
//   warps 2..   epilogue: warp w reads TMEM lanes 32*(w%4)..; the (tile, k slot)
//               items of its lane quadrant are shared round-robin by the
//               quadrant's warps (three in the linewidth form, two otherwise)
// Tensor memory holds two accumulator stages of 256 columns (512 in total),
// so the MMA of the next tile overlaps the epilogue of the current one.
// Tiles are visited in q-blocks (so that a block of A stays in L2) and, inside
// a block, k-group-major (so that the CTAs running together share one B tile).
// Every wait is bounded; a wait that runs out raises EPW_DEV_TIMEOUT, drains
// outstanding copies and MMAs, frees tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "epw_eig4.cuh"
#include "epw_tc.cuh"
#include "epw_tcgen05.cuh"

namespace {

constexpr int BM = 128;               // q rows per tile
constexpr int BN = 256;               // real accumulator columns per tile
constexpr int STAGES = 2;
constexpr int A_BYTES = BM * ROWB;    // 16 KiB
constexpr int B_BYTES = BN * ROWB;    // 32 KiB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
// A CTA pair (cluster of two CTAs, cta_group::2 MMAs with M = 256 over two neighbouring q
// tiles) holds half of the B rows per CTA, so its stages are smaller and three fit.
template <bool PAIR>
constexpr int tc_stages() { return PAIR ? 3 : STAGES; }
template <bool PAIR>
constexpr int tc_stage_bytes() { return 2 * A_BYTES + 2 * (PAIR ? B_BYTES / 2 : B_BYTES); }
template <bool PAIR>
constexpr int tc_smem_bytes() { return tc_stages<PAIR>() * tc_stage_bytes<PAIR>() + 1024; }
constexpr int EPI_WARP0 = 2;
constexpr int ITEMS_PER_TILE = 8;     // (lane quadrant, k slot) items per tile
// Epilogue warps per form, a multiple of 4 (one group per TMEM lane quadrant; a
// quadrant's (tile, k slot) items are taken round-robin by its warps): the
// linewidth form runs three per quadrant so that more warps hide each other's
// latency; the adjoint one, with the registers of a whole sub-partition for its
// conjugate-gradient accumulators; interpolation two.
constexpr int EPI_WARPS_LW = 12;
constexpr int EPI_WARPS_ADJ = 4;
template <int MODE>
constexpr int epi_warps() { return MODE == 0 ? EPI_WARPS_LW : MODE == 2 ? EPI_WARPS_ADJ : 8; }
template <int MODE>
constexpr int nthreads() { return 32 * (EPI_WARP0 + epi_warps<MODE>()); }
constexpr uint32_t TMEM_COLS = 512;
constexpr size_t A_BLOCK_BYTES = 48u << 20;      // q-block size target (A operand bytes)

template <int OP>
struct OpT;
template <>
struct OpT<TC_OP_BF16> {
  using T = __nv_bfloat16;
  static constexpr int ESZ = 2;
  static constexpr int BK = ROWB / ESZ;  // 64 elements per stage
  static constexpr int KSTEP = 16;      // K per MMA (32 bytes)
  // kind::f16 instruction descriptor: D=F32, A=B=BF16, K-major, N=256, M=128
  static constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  static constexpr uint32_t IDESC_PAIR =  // M = 256 (128 rows in each CTA of the pair)
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)((2 * BM) >> 4) << 24);
  static constexpr bool F16 = true;
};
template <>
struct OpT<TC_OP_TF32> {
  using T = float;
  static constexpr int ESZ = 4;
  static constexpr int BK = ROWB / ESZ;  // 32 elements per stage
  static constexpr int KSTEP = 8;       // K per MMA (32 bytes)
  // kind::tf32 instruction descriptor: D=F32, A=B=TF32, K-major, N=256, M=128
  static constexpr uint32_t IDESC =
      (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  static constexpr uint32_t IDESC_PAIR =
      (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)((2 * BM) >> 4) << 24);
  static constexpr bool F16 = false;
};

template <int OP>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  if constexpr (OP == TC_OP_BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(OpT<OP>::IDESC), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(OpT<OP>::IDESC), "r"(acc)
        : "memory");
  }
}

// Self-test of the failure path: one thread waits, with the kernels' bounded
// wait, on an mbarrier that nothing arrives at; after `limit` cycles the wait
// raises EPW_DEV_TIMEOUT in dstatus and returns, and the kernel exits.
__global__ void k_wait_selftest(long long limit, unsigned *dstatus, int *waited_out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_sh;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    volatile int *ab = &abort_sh;
    *waited_out = wait_bar_limit(smem_u32(&bar), 0, ab, dstatus, limit) ? 0 : 1;
  }
}

struct TcArgs {
  int nk, nq, nqt, nkg, kpad, nkb, qblock;
  const float *epsk;     // [nk][nw]
  const float *omegaT;   // [nm][nq]
  const float *nbT;      // [nm][nq]
  const float2 *ET;      // [nm*nm][nq]
  const float *wq;       // [nq]
  float EF, invkT, inv_sigma, gnorm, omega_min;
  double *partial;  // [nk][4*nqt][nw]            (linewidth)
  double *eps_kq;   // [nk][nq][nw] or null        (interp)
  double2 *gout;    // [nk][nq][nm][nw][nw] or null (interp)
  // adjoint (MODE 2)
  const float *cot;      // [nk][nw] cotangent of Im Sigma
  float *xhi, *xlo;      // [nk*nm*nw*nw][ldx] conjugate-gradient rows, K = 2q+t (tf32 split)
  int ldx;
  double *partT, *partE;  // [nk][4*nqt] per-warp sums of dL/dT and dL/dE_F
  float T;
  unsigned *dstatus;
  // long-range vertex (polar models; null otherwise): C_nu(q) [nm][nq], U_k [nk][nw][nw]
  const float2 *Cpol;
  const float2 *UkF;
};

template <int NW, int NM>
struct Shape {
  static constexpr int NC = NW * NW * (NM + 1);  // complex columns per k
  static constexpr int CPK_RAW = 2 * NC;
  static constexpr int CPK = CPK_RAW <= 8 ? 8 : CPK_RAW <= 16 ? 16 : CPK_RAW <= 32 ? 32 : CPK_RAW <= 64 ? 64 : 128;
  static constexpr int KPS = 128 / CPK;  // k per slot (per epilogue warp)
  static constexpr int KPT = 2 * KPS;    // k per tile
  static constexpr int H2 = 2 * NW * NW; // real columns of one NW x NW complex block
  // planar column pairs (k_build_b): shapes that fill the 128-column slot with an even NW
  static constexpr bool PLANAR = (NW % 2 == 0) && (CPK == 128);
  static_assert(CPK_RAW <= 128, "one k must fit in a 128-column slot");
  static_assert(CPK <= 32 || H2 == 32, "wide shapes read 32-column blocks");
};

// Per-q tables of the packed linewidth epilogue, fetched when a pair starts and
// read after its eigensolve: the mode factors E are copied with cp.async into
// shared memory after the operand stages, one column per epilogue thread
// (E [nm*nm][NT] float2); w and n are prefetched into L1.
constexpr int NEPI_THREADS = 32 * EPI_WARPS_LW;
template <int NW, int NM, int MODE>
constexpr int tab_bytes() {
  return (MODE == 0 && Shape<NW, NM>::PLANAR) ? NEPI_THREADS * NM * NM * 8 : 0;
}

// Tile -> (k group, q tile) in q-blocks of `qblock` tiles, k-group-major inside a block.
__device__ __forceinline__ void item_coords_n(int nqt, int qblock, int nkg, int item, int &kg, int &qt) {
  const int per = qblock * nkg;
  const int nb = (nqt + qblock - 1) / qblock;
  int b = item / per;
  if (b > nb - 1) b = nb - 1;
  const int r = item - b * per;
  const int qbs = min(qblock, nqt - b * qblock);
  kg = r / qbs;
  qt = b * qblock + r % qbs;
}
__device__ __forceinline__ void item_coords(const TcArgs &a, int item, int &kg, int &qt) {
  item_coords_n(a.nqt, a.qblock, a.nkg, item, kg, qt);
}
// A CTA pair takes two neighbouring q tiles per item, rank r the tile 2 u + r (the second may
// lie past nq: its rows are invalid and its partial sums are not written).
template <bool PAIR>
__device__ __forceinline__ void item_coords_p(const TcArgs &a, int item, uint32_t rank, int &kg, int &qt) {
  if constexpr (PAIR) {
    int u;
    item_coords_n((a.nqt + 1) / 2, a.qblock > 1 ? a.qblock / 2 : 1, a.nkg, item, kg, u);
    qt = 2 * u + (int)rank;
  } else {
    item_coords(a, item, kg, qt);
  }
}

// Real column of the re (s = 0) or im (s = 1) part of complex column c of one
// NW x NW block of the accumulator (planar pairs: see k_build_b).
template <bool PLANAR>
__device__ __forceinline__ int ccol(int c, int s) {
  return PLANAR ? 4 * (c >> 1) + 2 * s + (c & 1) : 2 * c + s;
}


// Linewidth terms of Eq. (linewidthel) for one pair from planar accumulator
// columns (NW even).  Entries (i, j) and (i, j+1) of a block travel as one
// float2 of real parts and one of imaginary parts, so the mode projection
// G_nu = sum_a E[a][nu] X_a, the rotation y_nu = U_k+q^dagger G_nu, |y|^2 and
// the Gaussian arguments each handle two n columns per packed instruction.
// The Gaussian argument is formed as -(x s)^2 with s = sqrt(log2 e)/sigma, so
// that exp(-(x/sigma)^2) = 2^(-(x s)^2).
template <int NW, int NM>
__device__ __forceinline__ void tables_prefetch(const TcArgs &a, int qq, float *tab) {
  const int te = threadIdx.x - 32 * EPI_WARP0;
  const uint32_t t0 = smem_u32(tab);
#pragma unroll
  for (int j = 0; j < NM * NM; j++) cp_async8(t0 + 8u * (j * NEPI_THREADS + te), a.ET + (size_t)j * a.nq + qq);
#pragma unroll
  for (int nu = 0; nu < NM; nu++) {
    prefetch_l1(a.omegaT + (size_t)nu * a.nq + qq);
    prefetch_l1(a.nbT + (size_t)nu * a.nq + qq);
  }
}

template <int NW, int NM>
__device__ __forceinline__ void modes_linewidth_packed(const TcArgs &a, uint32_t tcol, int qq, int kk,
                                                       const float *tab, const cx<float> (&V)[NW][NW],
                                                       const float (&em)[NW], const float (&fm)[NW],
                                                       const float (&ek)[NW], float (&acc)[NW]) {
  const int te = threadIdx.x - 32 * EPI_WARP0;
  const float2 *tE = reinterpret_cast<const float2 *>(tab) + te;
  cp_async_wait_all();
  constexpr int NP = NW / 2;
  constexpr int H2 = 2 * NW * NW;
  const float sc = a.inv_sigma * 1.2011224087864498f;  // sqrt(log2 e) / sigma
  float2 eks[NP], accp[NP];
#pragma unroll
  for (int p = 0; p < NP; p++) {
    eks[p] = make_float2(ek[2 * p] * sc, ek[2 * p + 1] * sc);
    accp[p] = make_float2(0.0f, 0.0f);
  }
#pragma unroll 1
  for (int nu = 0; nu < NM; nu++) {
    const float wnu = __ldg(a.omegaT + (size_t)nu * a.nq + qq);
    const float nbnu = __ldg(a.nbT + (size_t)nu * a.nq + qq);
    float2 E[NM];
#pragma unroll
    for (int al = 0; al < NM; al++) E[al] = tE[(al * NM + nu) * NEPI_THREADS];
    const bool keep = (wnu >= a.omega_min) && (wnu > 0.0f);
    // G_nu, planar: Gr[i][p] = Re (G_i,2p, G_i,2p+1), Gi[i][p] = Im (...)
    float2 Gr[NW][NP], Gi[NW][NP];
#pragma unroll
    for (int al = 0; al < NM; al++) {
      float x[H2];
      tmem_load<H2>(tcol + H2 * (1 + al), x);
      const float2 er = bc2(E[al].x), ei = bc2(E[al].y), nei = bc2(-E[al].y);
#pragma unroll
      for (int i = 0; i < NW; i++)
#pragma unroll
        for (int p = 0; p < NP; p++) {
          const int o = 4 * (i * NP + p);
          const float2 xr = make_float2(x[o], x[o + 1]), xi = make_float2(x[o + 2], x[o + 3]);
          if (al == 0) {
            Gr[i][p] = ffma2(nei, xi, fmul2(er, xr));
            Gi[i][p] = ffma2(ei, xr, fmul2(er, xi));
          } else {
            Gr[i][p] = ffma2(nei, xi, ffma2(er, xr, Gr[i][p]));
            Gi[i][p] = ffma2(ei, xr, ffma2(er, xi, Gi[i][p]));
          }
        }
    }
    if (a.Cpol) {
      // long-range part: G_nu += i C_nu(q) U_k
      const float2 c = __ldg(a.Cpol + (size_t)nu * a.nq + qq);
      const float2 *Uk = a.UkF + (size_t)kk * NW * NW;
      const float2 ncy = bc2(-c.y), ncx = bc2(-c.x), cx2 = bc2(c.x);
#pragma unroll
      for (int i = 0; i < NW; i++)
#pragma unroll
        for (int p = 0; p < NP; p++) {
          const float2 u0 = __ldg(Uk + i * NW + 2 * p), u1 = __ldg(Uk + i * NW + 2 * p + 1);
          const float2 ur = make_float2(u0.x, u1.x), ui = make_float2(u0.y, u1.y);
          Gr[i][p] = ffma2(ncy, ur, ffma2(ncx, ui, Gr[i][p]));
          Gi[i][p] = ffma2(cx2, ur, ffma2(ncy, ui, Gi[i][p]));
        }
    }
    const float ws = wnu * sc;
#pragma unroll
    for (int m = 0; m < NW; m++) {
      // y = (U^dagger G)_m,(2p, 2p+1)
      float2 yr[NP], yi[NP];
#pragma unroll
      for (int i = 0; i < NW; i++) {
        const float2 vr = bc2(V[i][m].x), vi = bc2(V[i][m].y), nvi = bc2(-V[i][m].y);
#pragma unroll
        for (int p = 0; p < NP; p++) {
          if (i == 0) {
            yr[p] = ffma2(vi, Gi[i][p], fmul2(vr, Gr[i][p]));
            yi[p] = ffma2(nvi, Gr[i][p], fmul2(vr, Gi[i][p]));
          } else {
            yr[p] = ffma2(vi, Gi[i][p], ffma2(vr, Gr[i][p], yr[p]));
            yi[p] = ffma2(nvi, Gr[i][p], ffma2(vr, Gi[i][p], yi[p]));
          }
        }
      }
      const float2 cp = bc2(keep ? nbnu + fm[m] : 0.0f), cm = bc2(keep ? nbnu + 1.0f - fm[m] : 0.0f);
      const float ems = em[m] * sc;
      const float2 op = bc2(ws - ems), om = bc2(-ws - ems);  // x+- = e_nk - e_mk+q +- w, scaled
#pragma unroll
      for (int p = 0; p < NP; p++) {
        const float2 g2 = ffma2(yi[p], yi[p], fmul2(yr[p], yr[p]));
        const float2 xp = fadd2(eks[p], op), xm = fadd2(eks[p], om);
        const float2 tp = fmul2(xp, xp), tm = fmul2(xm, xm);
        const float2 dp = make_float2(ex2_approx(-tp.x), ex2_approx(-tp.y));
        const float2 dm = make_float2(ex2_approx(-tm.x), ex2_approx(-tm.y));
        accp[p] = ffma2(g2, ffma2(cm, dm, fmul2(cp, dp)), accp[p]);
      }
    }
  }
#pragma unroll
  for (int p = 0; p < NP; p++) {
    acc[2 * p] = accp[p].x;
    acc[2 * p + 1] = accp[p].y;
  }
}

// Adjoint terms (MODE 2) of one pair from planar accumulator columns (NW even),
// the packed counterpart of the generic MODE 2 loop in epilogue_pair: per mode
// W_nu,mn = c_nk pi w_q [(n+f) d+ + (n+1-f) d-], Z_nu = U (2 W_nu o y_nu) with
// y_nu = U^dagger G_nu, and Xbar_a = sum_nu conj(E[a][nu]) Z_nu, written as the
// ep - en for ep = 2^(-(x + w)^2 s2), en = 2^(-(x - w)^2 s2) (the Gaussians of the
// forward sums in base 2).  The exponents differ by 4 x w s2, so
//   ep - en = -2 * 2^(-(x^2 + w^2) s2) * sinh(2 ln2 x w s2),
// with sinh(y) from its Taylor series through y^9/9! for |y| <= 1 (truncation below
// 3e-8 relative): no subtraction of close values when w << sigma.  For |y| > 1 the
// two values differ by a factor e^2 or more and the plain difference is taken.
__device__ __forceinline__ float gauss_diff2(float x, float w, float s2, float ep, float en) {
  const float y = 1.3862943611198906f * x * w * s2;  // 2 ln2 x w s2
  const float y2 = y * y;
  const float sh =
      y * fmaf(y2, fmaf(y2, fmaf(y2, fmaf(y2, 1.0f / 362880.0f, 1.0f / 5040.0f), 1.0f / 120.0f), 1.0f / 6.0f), 1.0f);
  const float small = -2.0f * ex2_approx(-fmaf(x, x, w * w) * s2) * sh;
  return fabsf(y) <= 1.0f ? small : ep - en;
}

// tf32-split rows (k, a, j, n); the dL/dT and dL/dE_F terms go to sT and sE.
// Two n columns per packed FP32 instruction, as in modes_linewidth_packed.
template <int NW, int NM>
__device__ __forceinline__ void modes_adjoint_packed(const TcArgs &a, uint32_t tcol, int q, int qq, int k, int kk,
                                                     bool valid, const cx<float> (&V)[NW][NW],
                                                     const float (&em)[NW], const float (&fm)[NW],
                                                     const float (&ek)[NW], const float (&cw)[NW], float &sT,
                                                     float &sE) {
  constexpr int NP = NW / 2;
  constexpr int H2 = 2 * NW * NW;
  const float sc = a.inv_sigma * 1.2011224087864498f;  // sqrt(log2 e) / sigma
  float2 eks[NP], cw2[NP], sT2 = make_float2(0.0f, 0.0f), sE2 = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int p = 0; p < NP; p++) {
    eks[p] = make_float2(ek[2 * p] * sc, ek[2 * p + 1] * sc);
    cw2[p] = make_float2(cw[2 * p], cw[2 * p + 1]);
  }
  // per band m at k+q: df/dT and df/dE_F (mode independent)
  float dfT[NW], dfE[NW];
#pragma unroll
  for (int m = 0; m < NW; m++) {
    const float ff = fermi_ff_f(em[m] - a.EF, a.invkT);
    dfT[m] = ff * (em[m] - a.EF) * a.invkT / a.T;
    dfE[m] = ff * a.invkT;
  }
  float2 Xr[NM][NW][NP], Xi[NM][NW][NP];
#pragma unroll
  for (int al = 0; al < NM; al++)
#pragma unroll
    for (int j = 0; j < NW; j++)
#pragma unroll
      for (int p = 0; p < NP; p++) Xr[al][j][p] = Xi[al][j][p] = make_float2(0.0f, 0.0f);
#pragma unroll 1
  for (int nu = 0; nu < NM; nu++) {
    const float wnu = __ldg(a.omegaT + (size_t)nu * a.nq + qq);
    const float nbnu = __ldg(a.nbT + (size_t)nu * a.nq + qq);
    float2 E[NM];
#pragma unroll
    for (int al = 0; al < NM; al++) E[al] = __ldg(a.ET + ((size_t)al * NM + nu) * a.nq + qq);
    const bool keep = (wnu >= a.omega_min) && (wnu > 0.0f);
    const float kf = keep ? 1.0f : 0.0f;
    const float dn = kf * nbnu * (nbnu + 1.0f) * wnu * a.invkT / a.T;
    float2 Gr[NW][NP], Gi[NW][NP];
#pragma unroll
    for (int al = 0; al < NM; al++) {
      float x[H2];
      tmem_load<H2>(tcol + H2 * (1 + al), x);
      const float2 er = bc2(E[al].x), ei = bc2(E[al].y), nei = bc2(-E[al].y);
#pragma unroll
      for (int i = 0; i < NW; i++)
#pragma unroll
        for (int p = 0; p < NP; p++) {
          const int o = 4 * (i * NP + p);
          const float2 xr = make_float2(x[o], x[o + 1]), xi = make_float2(x[o + 2], x[o + 3]);
          if (al == 0) {
            Gr[i][p] = ffma2(nei, xi, fmul2(er, xr));
            Gi[i][p] = ffma2(ei, xr, fmul2(er, xi));
          } else {
            Gr[i][p] = ffma2(nei, xi, ffma2(er, xr, Gr[i][p]));
            Gi[i][p] = ffma2(ei, xr, ffma2(er, xi, Gi[i][p]));
          }
        }
    }
    if (a.Cpol) {
      // long-range part: G_nu += i C_nu(q) U_k
      const float2 c = __ldg(a.Cpol + (size_t)nu * a.nq + qq);
      const float2 *Uk = a.UkF + (size_t)kk * NW * NW;
      const float2 ncy = bc2(-c.y), ncx = bc2(-c.x), cx2 = bc2(c.x);
#pragma unroll
      for (int i = 0; i < NW; i++)
#pragma unroll
        for (int p = 0; p < NP; p++) {
          const float2 u0 = __ldg(Uk + i * NW + 2 * p), u1 = __ldg(Uk + i * NW + 2 * p + 1);
          const float2 ur = make_float2(u0.x, u1.x), ui = make_float2(u0.y, u1.y);
          Gr[i][p] = ffma2(ncy, ur, ffma2(ncx, ui, Gr[i][p]));
          Gi[i][p] = ffma2(cx2, ur, ffma2(ncy, ui, Gi[i][p]));
        }
    }
    float2 Zr[NW][NP], Zi[NW][NP];
#pragma unroll
    for (int j = 0; j < NW; j++)
#pragma unroll
      for (int p = 0; p < NP; p++) Zr[j][p] = Zi[j][p] = make_float2(0.0f, 0.0f);
    const float ws = wnu * sc;
    float2 kcw[NP], cw2x[NP];
#pragma unroll
    for (int p = 0; p < NP; p++) {
      kcw[p] = fmul2(bc2(kf), cw2[p]);
      cw2x[p] = fmul2(bc2(2.0f), cw2[p]);
    }
#pragma unroll
    for (int m = 0; m < NW; m++) {
      float2 yr[NP], yi[NP];
#pragma unroll
      for (int i = 0; i < NW; i++) {
        const float2 vr = bc2(V[i][m].x), vi = bc2(V[i][m].y), nvi = bc2(-V[i][m].y);
#pragma unroll
        for (int p = 0; p < NP; p++) {
          if (i == 0) {
            yr[p] = ffma2(vi, Gi[i][p], fmul2(vr, Gr[i][p]));
            yi[p] = ffma2(nvi, Gr[i][p], fmul2(vr, Gi[i][p]));
          } else {
            yr[p] = ffma2(vi, Gi[i][p], ffma2(vr, Gr[i][p], yr[p]));
            yi[p] = ffma2(nvi, Gr[i][p], ffma2(vr, Gi[i][p], yi[p]));
          }
        }
      }
      const float2 cp = bc2(kf * (nbnu + fm[m])), cm = bc2(kf * (nbnu + 1.0f - fm[m]));
      const float2 dn2 = bc2(dn), dT2 = bc2(dfT[m]), dE = bc2(dfE[m]);
      const float ems = em[m] * sc;
      const float2 op = bc2(ws - ems), om = bc2(-ws - ems);
      float2 ybr[NP], ybi[NP];
#pragma unroll
      for (int p = 0; p < NP; p++) {
        const float2 g2 = ffma2(yi[p], yi[p], fmul2(yr[p], yr[p]));
        const float2 xp = fadd2(eks[p], op), xm = fadd2(eks[p], om);
        const float2 tp = fmul2(xp, xp), tm = fmul2(xm, xm);
        const float2 ep = make_float2(ex2_approx(-tp.x), ex2_approx(-tp.y));
        const float2 en = make_float2(ex2_approx(-tm.x), ex2_approx(-tm.y));
        const float2 wv = fmul2(cw2x[p], ffma2(cm, en, fmul2(cp, ep)));
        const float2 kg = fmul2(kcw[p], g2);
        // (dn + dfT) ep + (dn - dfT) en = dn (ep + en) + dfT (ep - en); ep - en in the sinh form
        const float2 dd = make_float2(gauss_diff2(eks[p].x - ems, ws, 1.0f, ep.x, en.x),
                                      gauss_diff2(eks[p].y - ems, ws, 1.0f, ep.y, en.y));
        sT2 = ffma2(kg, ffma2(dT2, dd, fmul2(dn2, fadd2(ep, en))), sT2);
        sE2 = ffma2(fmul2(kg, dE), dd, sE2);
        ybr[p] = fmul2(wv, yr[p]);
        ybi[p] = fmul2(wv, yi[p]);
      }
      // Z[j][n] += U[j][m] yb[n]
#pragma unroll
      for (int j = 0; j < NW; j++) {
        const float2 vr = bc2(V[j][m].x), vi = bc2(V[j][m].y), nvi = bc2(-V[j][m].y);
#pragma unroll
        for (int p = 0; p < NP; p++) {
          Zr[j][p] = ffma2(nvi, ybi[p], ffma2(vr, ybr[p], Zr[j][p]));
          Zi[j][p] = ffma2(vi, ybr[p], ffma2(vr, ybi[p], Zi[j][p]));
        }
      }
    }
    // Xbar_a += conj(E[a][nu]) Z_nu
#pragma unroll
    for (int al = 0; al < NM; al++) {
      const float2 er = bc2(E[al].x), ei = bc2(E[al].y), nei = bc2(-E[al].y);
#pragma unroll
      for (int j = 0; j < NW; j++)
#pragma unroll
        for (int p = 0; p < NP; p++) {
          Xr[al][j][p] = ffma2(ei, Zi[j][p], ffma2(er, Zr[j][p], Xr[al][j][p]));
          Xi[al][j][p] = ffma2(nei, Zr[j][p], ffma2(er, Zi[j][p], Xi[al][j][p]));
        }
    }
  }
  sT = sT2.x + sT2.y;
  sE = sE2.x + sE2.y;
  if (valid) {
    // Xbar rows (k, a, j, n), K index 2q + (re, im), split into two tf32 terms
#pragma unroll
    for (int al = 0; al < NM; al++)
#pragma unroll
      for (int j = 0; j < NW; j++)
#pragma unroll
        for (int n = 0; n < NW; n++) {
          const size_t row = (size_t)k * (NM * NW * NW) + (al * NW + j) * NW + n;
          const float re = (n & 1) ? Xr[al][j][n >> 1].y : Xr[al][j][n >> 1].x;
          const float im = (n & 1) ? Xi[al][j][n >> 1].y : Xi[al][j][n >> 1].x;
          const float hr = tf32_rn(re), hi = tf32_rn(im);
          *reinterpret_cast<float2 *>(a.xhi + row * a.ldx + 2 * (size_t)q) = make_float2(hr, hi);
          *reinterpret_cast<float2 *>(a.xlo + row * a.ldx + 2 * (size_t)q) =
              make_float2(tf32_rn(re - hr), tf32_rn(im - hi));
        }
  }
}

// ------------------------------------------------------------------ epilogue
// One (k,q) pair per thread; the accumulator holds [H(k+q) | (g_a U_k)_a=0..NM-1].
// MODE 0: linewidth terms summed over the warp's q rows; MODE 1: write e_k+q
// (ascending) and g_mn,nu; MODE 2: adjoint of L = sum c_nk Im Sigma_nk:
//   W_nu,mn = c_nk pi w_q [(n+f) d+ + (n+1-f) d-],   Ybar_nu = 2 W_nu (U^dagger G_nu)
//   Xbar_a  = sum_nu conj(E[a][nu]) U Ybar_nu   (= dL/d(g_a U_k)(k,q)*, written out)
//   dL/dT, dL/dE_F through n(w, T) and f(e, T, E_F) (deltas hold neither).
template <int NW, int NM, int MODE>
__device__ __forceinline__ void epilogue_pair(const TcArgs &a, uint32_t tcol, int q, int k, bool valid, int quad,
                                              int qt, float *tab) {
  using S = Shape<NW, NM>;
  constexpr int H2 = S::H2;
  const int qq = q < a.nq ? q : 0;
  const int kk = k < a.nk ? k : 0;
  if constexpr (MODE == 0 && S::PLANAR) tables_prefetch<NW, NM>(a, qq, tab);
  if constexpr (MODE == 2 && S::PLANAR) {
#pragma unroll
    for (int j = 0; j < NM * NM; j++) prefetch_l1(a.ET + (size_t)j * a.nq + qq);
#pragma unroll
    for (int nu = 0; nu < NM; nu++) {
      prefetch_l1(a.omegaT + (size_t)nu * a.nq + qq);
      prefetch_l1(a.nbT + (size_t)nu * a.nq + qq);
    }
  }
  // per-q and per-k data first, so their latency overlaps the eigensolve
  float ek[NW];
#pragma unroll
  for (int n = 0; n < NW; n++) ek[n] = __ldg(a.epsk + (size_t)kk * NW + n);
  const float wqf = valid ? __ldg(a.wq + q) : 0.0f;
  // data of the first mode (each later mode is fetched one iteration ahead)


  constexpr bool ONE_LOAD = S::CPK <= 32;
  float all[ONE_LOAD ? S::CPK : 8];
  float hb[ONE_LOAD ? 8 : H2];
  if constexpr (ONE_LOAD) {
    tmem_load<S::CPK>(tcol, all);
  } else {
    tmem_load<H2>(tcol, hb);
  }
  constexpr bool PL = S::PLANAR;
  Herm<NW> H;
#pragma unroll
  for (int i = 0; i < NW; i++)
#pragma unroll
    for (int j = i; j < NW; j++) {
      const int o = ccol<PL>(i * NW + j, 0), oi = ccol<PL>(i * NW + j, 1);
      const int o2 = ccol<PL>(j * NW + i, 0), o2i = ccol<PL>(j * NW + i, 1);
      float re, im;
      if constexpr (ONE_LOAD) {
        re = 0.5f * (all[o] + all[o2]);
        im = 0.5f * (all[oi] - all[o2i]);
      } else {
        re = 0.5f * (hb[o] + hb[o2]);
        im = 0.5f * (hb[oi] - hb[o2i]);
      }
      H.a[i][j] = mkc(re, i == j ? 0.0f : im);
    }
  cx<float> V[NW][NW];
  const bool conv = jacobi_fast<NW>(H, V);
  if (!conv && valid) atomicOr(a.dstatus, EPW_DEV_NOT_CONVERGED);
  float em[NW], fm[NW];
#pragma unroll
  for (int m = 0; m < NW; m++) em[m] = H.a[m][m].x;
  if constexpr (MODE == 1) {
    // ascending order (odd-even transposition network), eigenvector columns follow
#pragma unroll
    for (int r = 0; r < NW; r++)
#pragma unroll
      for (int m = r & 1; m + 1 < NW; m += 2) {
        const bool sw = em[m + 1] < em[m];
        const float lo = sw ? em[m + 1] : em[m], hi = sw ? em[m] : em[m + 1];
        em[m] = lo;
        em[m + 1] = hi;
#pragma unroll
        for (int i = 0; i < NW; i++) {
          const cx<float> v0 = V[i][m], v1 = V[i][m + 1];
          V[i][m] = sw ? v1 : v0;
          V[i][m + 1] = sw ? v0 : v1;
        }
      }
    if (valid && a.eps_kq) {
#pragma unroll
      for (int m = 0; m < NW; m++) a.eps_kq[((size_t)k * a.nq + q) * NW + m] = (double)em[m];
    }
  }
#pragma unroll
  for (int m = 0; m < NW; m++) fm[m] = fermi_fast(em[m] - a.EF, a.invkT);
  float acc[NW];
#pragma unroll
  for (int n = 0; n < NW; n++) acc[n] = 0.0f;
  const float s2 = a.inv_sigma * a.inv_sigma * 1.4426950408889634f;
  // adjoint state (MODE 2): c_nk pi w_q / (sigma sqrt(pi)) per n, Xbar accumulators, dT / dE_F sums
  float cw[MODE == 2 ? NW : 1];
  cx<float> Xb[MODE == 2 ? NM : 1][NW][NW];
  float sT = 0.0f, sE = 0.0f;
  if constexpr (MODE == 2) {
#pragma unroll
    for (int n = 0; n < NW; n++)
      cw[n] = valid ? __ldg(a.cot + (size_t)kk * NW + n) * 3.14159265358979f * wqf * a.gnorm : 0.0f;
#pragma unroll
    for (int al = 0; al < NM; al++)
#pragma unroll
      for (int i = 0; i < NW; i++)
#pragma unroll
        for (int j = 0; j < NW; j++) Xb[al][i][j] = mkc(0.0f, 0.0f);
  }
  if constexpr (MODE == 0 && PL) {
    modes_linewidth_packed<NW, NM>(a, tcol, qq, kk, tab, V, em, fm, ek, acc);
  } else if constexpr (MODE == 2 && PL) {
    modes_adjoint_packed<NW, NM>(a, tcol, q, qq, k, kk, valid, V, em, fm, ek, cw, sT, sE);
  } else {
  // one mode per iteration (not unrolled: keeps the code within the instruction cache)
#pragma unroll 1
  for (int nu = 0; nu < NM; nu++) {
    const float wnu = __ldg(a.omegaT + (size_t)nu * a.nq + qq);
    const float nbnu = __ldg(a.nbT + (size_t)nu * a.nq + qq);
    cx<float> E[NM];
#pragma unroll
    for (int al = 0; al < NM; al++) {
      const float2 e = __ldg(a.ET + ((size_t)al * NM + nu) * a.nq + qq);
      E[al] = mkc(e.x, e.y);
    }
    const bool keep = (wnu >= a.omega_min) && (wnu > 0.0f);
    cx<float> G[NW][NW];
#pragma unroll
    for (int i = 0; i < NW; i++)
#pragma unroll
      for (int j = 0; j < NW; j++) G[i][j] = mkc(0.0f, 0.0f);
#pragma unroll
    for (int al = 0; al < NM; al++) {
      if constexpr (ONE_LOAD) {
#pragma unroll
        for (int i = 0; i < NW; i++)
#pragma unroll
          for (int j = 0; j < NW; j++) {
            const int o = H2 * (1 + al) + 2 * (i * NW + j);
            cfma(G[i][j], E[al], mkc(all[o], all[o + 1]));
          }
      } else {
        float x[H2];
        tmem_load<H2>(tcol + H2 * (1 + al), x);
#pragma unroll
        for (int i = 0; i < NW; i++)
#pragma unroll
          for (int j = 0; j < NW; j++) cfma(G[i][j], E[al], mkc(x[ccol<PL>(i * NW + j, 0)], x[ccol<PL>(i * NW + j, 1)]));
      }
    }

    if (a.Cpol) {
      // long-range part: G_nu += i C_nu(q) U_k, so that U_k+q^dagger G picks up i C [U_k+q^dagger U_k]
      const float2 c = __ldg(a.Cpol + (size_t)nu * a.nq + qq);
      const float2 *Uk = a.UkF + (size_t)kk * NW * NW;
#pragma unroll
      for (int i = 0; i < NW; i++)
#pragma unroll
        for (int j = 0; j < NW; j++) {
          const float2 u = __ldg(Uk + i * NW + j);
          G[i][j].x = fmaf(-c.y, u.x, fmaf(-c.x, u.y, G[i][j].x));
          G[i][j].y = fmaf(c.x, u.x, fmaf(-c.y, u.y, G[i][j].y));
        }
    }
    if constexpr (MODE == 2) {
      const float kf = keep ? 1.0f : 0.0f;
      const float dn = kf * nbnu * (nbnu + 1.0f) * wnu * a.invkT / a.T;
      cx<float> Z[NW][NW];  // U Ybar_nu
#pragma unroll
      for (int i = 0; i < NW; i++)
#pragma unroll
        for (int j = 0; j < NW; j++) Z[i][j] = mkc(0.0f, 0.0f);
#pragma unroll
      for (int m = 0; m < NW; m++) {
        const float f = fm[m];
        const float ff = fermi_ff_f(em[m] - a.EF, a.invkT);
        const float dfT = ff * (em[m] - a.EF) * a.invkT / a.T;
        const float dfE = ff * a.invkT;
        const float cp = kf * (nbnu + f), cm = kf * (nbnu + 1.0f - f);
#pragma unroll
        for (int n = 0; n < NW; n++) {
          cx<float> y = mkc(0.0f, 0.0f);
#pragma unroll
          for (int i = 0; i < NW; i++) cfma(y, conjc(V[i][m]), G[i][n]);
          const float g2 = cabs2(y);
          const float xd = ek[n] - em[m];
          const float xp = xd + wnu, xm = xd - wnu;
          const float ep = ex2_approx(-xp * xp * s2), en = ex2_approx(-xm * xm * s2);
          const float wv = 2.0f * cw[n] * (cp * ep + cm * en);
          const float dd = gauss_diff2(xd, wnu, s2, ep, en);  // ep - en without cancellation
          sT = fmaf(kf * cw[n] * g2, fmaf(dn, ep + en, dfT * dd), sT);
          sE = fmaf(kf * cw[n] * g2, dfE * dd, sE);
          const cx<float> yb = mkc(wv * y.x, wv * y.y);
#pragma unroll
          for (int j = 0; j < NW; j++) cfma(Z[j][n], V[j][m], yb);
        }
      }
#pragma unroll
      for (int al = 0; al < NM; al++) {
        const cx<float> ec = conjc(E[al]);
#pragma unroll
        for (int j = 0; j < NW; j++)
#pragma unroll
          for (int n = 0; n < NW; n++) cfma(Xb[al][j][n], ec, Z[j][n]);
      }
    } else {
      // |(U^dagger G)_mn|^2 with the delta terms of Eq. (linewidthel)
#pragma unroll
      for (int m = 0; m < NW; m++) {
        const float cp = keep ? nbnu + fm[m] : 0.0f;
        const float cm = keep ? nbnu + 1.0f - fm[m] : 0.0f;
#pragma unroll
        for (int n = 0; n < NW; n++) {
          cx<float> y = mkc(0.0f, 0.0f);
#pragma unroll
          for (int i = 0; i < NW; i++) cfma(y, conjc(V[i][m]), G[i][n]);
          if constexpr (MODE == 1) {
            if (valid && a.gout)
              a.gout[(((size_t)k * a.nq + q) * NM + nu) * NW * NW + m * NW + n] = make_double2(y.x, y.y);
            continue;
          }
          const float g2 = cabs2(y);
          const float xd = ek[n] - em[m];
          const float xp = xd + wnu, xm = xd - wnu;
          const float d = cp * ex2_approx(-xp * xp * s2) + cm * ex2_approx(-xm * xm * s2);
          acc[n] = fmaf(g2, d, acc[n]);
        }
      }
    }
  }
  }
  if constexpr (MODE == 2) {
    // Xbar rows (k, a, j, n), K index 2q + (re, im), split into two tf32 terms
    if (valid && !PL) {
#pragma unroll
      for (int al = 0; al < NM; al++)
#pragma unroll
        for (int j = 0; j < NW; j++)
#pragma unroll
          for (int n = 0; n < NW; n++) {
            const size_t row = (size_t)k * (NM * NW * NW) + (al * NW + j) * NW + n;
            const float re = Xb[al][j][n].x, im = Xb[al][j][n].y;
            const float hr = tf32_rn(re), hi = tf32_rn(im);
            *reinterpret_cast<float2 *>(a.xhi + row * a.ldx + 2 * (size_t)q) = make_float2(hr, hi);
            *reinterpret_cast<float2 *>(a.xlo + row * a.ldx + 2 * (size_t)q) =
                make_float2(tf32_rn(re - hr), tf32_rn(im - hi));
          }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sT += __shfl_down_sync(0xffffffffu, sT, o);
      sE += __shfl_down_sync(0xffffffffu, sE, o);
    }
    if ((threadIdx.x & 31) == 0 && k < a.nk) {
      a.partT[(size_t)k * (4 * a.nqt) + qt * 4 + quad] = (double)sT;
      a.partE[(size_t)k * (4 * a.nqt) + qt * 4 + quad] = (double)sE;
    }
  }
  if constexpr (MODE == 0) {
#pragma unroll
    for (int n = 0; n < NW; n++) {
      // 32 positive terms: an FP32 tree sum is accurate to a few ulp
      float v = acc[n] * wqf;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0 && k < a.nk)
        a.partial[((size_t)k * (4 * a.nqt) + qt * 4 + quad) * NW + n] = (double)v * (double)a.gnorm;
    }
  }
}

template <int OP, int NW, int NM, int MODE, bool PAIR>
__global__ void __launch_bounds__(nthreads<MODE>(), 1)
    k_tc_linewidth(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                   const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, TcArgs a) {
  using S = Shape<NW, NM>;
  using O = OpT<OP>;
  static_assert(!PAIR || MODE == 0, "CTA pairs serve the linewidth form");
  constexpr int NSTAGE = tc_stages<PAIR>();
  constexpr int STAGE = tc_stage_bytes<PAIR>();
  constexpr int BROWS = PAIR ? BN / 2 : BN;  // B rows of a stage held by this CTA
  __shared__ __align__(8) uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_tfull[2], bar_tempty[2], bar_final;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t smem0 = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int *abort_flag = &abort_sh;
  // a pair (cluster of two CTAs) shares each item: the leader (rank 0) issues the MMAs for
  // both, the epilogue warps of both release tensor memory on the leader's barriers
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const bool leader = rank == 0;
  const int cid = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int ncl = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  const int nitems = a.nkg * (PAIR ? (a.nqt + 1) / 2 : a.nqt);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; s++) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int s = 0; s < 2; s++) {
      mbar_init(smem_u32(&bar_tfull[s]), 1);
      mbar_init(smem_u32(&bar_tempty[s]), PAIR ? 2 * ITEMS_PER_TILE : ITEMS_PER_TILE);
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
  const uint32_t full_c0 = PAIR ? cluster_addr(smem_u32(&bar_full[0]), 0) : smem_u32(&bar_full[0]);
  const uint32_t tempty_c0 = PAIR ? cluster_addr(smem_u32(&bar_tempty[0]), 0) : smem_u32(&bar_tempty[0]);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    // The whole warp walks the schedule; lane 0 waits and issues the copies.
    int issued[NSTAGE];
#pragma unroll
    for (int s = 0; s < NSTAGE; s++) issued[s] = 0;
    uint32_t it = 0;
    bool ok = true;
    for (int item = cid; item < nitems && ok; item += ncl) {
      int kg, qt;
      item_coords_p<PAIR>(a, item, rank, kg, qt);
      for (int kb = 0; kb < a.nkb; kb++, it++) {
        const int s = it % NSTAGE;
        const uint32_t par = ((it / NSTAGE) & 1u) ^ 1u;
        if (lane == 0) {
          ok = wait_bar(smem_u32(&bar_empty[s]), par, abort_flag, a.dstatus);
          if (ok) {
            const uint32_t base = smem0 + s * STAGE;
            const int brow = kg * (S::KPT * S::CPK) + (int)rank * BROWS;
            if constexpr (PAIR) {
              // this CTA's A tile and half of the B rows; the leader's barrier counts both CTAs'
              const uint32_t fb = full_c0 + 8u * (uint32_t)s;
              if (leader) mbar_expect_tx(smem_u32(&bar_full[s]), 2 * STAGE);
              tma_load_2d_pair(base, &mAhi, kb * O::BK, qt * BM, fb);
              tma_load_2d_pair(base + A_BYTES, &mAlo, kb * O::BK, qt * BM, fb);
              tma_load_2d_pair(base + 2 * A_BYTES, &mBhi, kb * O::BK, brow, fb);
              tma_load_2d_pair(base + 2 * A_BYTES + BROWS * ROWB, &mBlo, kb * O::BK, brow, fb);
            } else {
              const uint32_t fb = smem_u32(&bar_full[s]);
              mbar_expect_tx(fb, STAGE);
              tma_load_2d(base, &mAhi, kb * O::BK, qt * BM, fb);
              tma_load_2d(base + A_BYTES, &mAlo, kb * O::BK, qt * BM, fb);
              tma_load_2d(base + 2 * A_BYTES, &mBhi, kb * O::BK, brow, fb);
              tma_load_2d(base + 2 * A_BYTES + B_BYTES, &mBlo, kb * O::BK, brow, fb);
            }
            issued[s] = (int)(it / NSTAGE) + 1;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
      }
    }
    // drain: every issued copy must land before the CTA exits (a pair's loads complete on
    // the leader's barriers)
    if (lane == 0 && leader) {
#pragma unroll
      for (int s = 0; s < NSTAGE; s++)
        if (issued[s] > 0) drain_bar(smem_u32(&bar_full[s]), (uint32_t)((issued[s] - 1) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    // The whole warp walks the schedule; lane 0 waits and issues the MMAs.
    uint32_t it = 0;
    int titer = 0;
    bool ok = true;
    auto commit = [&](uint32_t bar) {
      if constexpr (PAIR)
        umma_commit_pair(bar);
      else
        umma_commit(bar);
    };
    // a pair's second CTA issues no MMAs: the leader's land in both CTAs' tensor memory
    for (int item = cid; item < nitems && ok && leader; item += ncl, titer++) {
      const int ts = titer & 1;
      const uint32_t tpar = ((titer >> 1) & 1) ^ 1;
      if (lane == 0) ok = wait_bar(smem_u32(&bar_tempty[ts]), tpar, abort_flag, a.dstatus);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
      const uint32_t dcol = tmem + ts * BN;
      for (int kb = 0; kb < a.nkb; kb++, it++) {
        const int s = it % NSTAGE;
        const uint32_t par = (it / NSTAGE) & 1u;
        if (lane == 0) {
          ok = wait_bar(smem_u32(&bar_full[s]), par, abort_flag, a.dstatus);
          if (ok) {
            tc_fence_after();
            const uint32_t base = smem0 + s * STAGE;
            const uint64_t dAh = sdesc_sw128(base), dAl = sdesc_sw128(base + A_BYTES);
            const uint64_t dBh = sdesc_sw128(base + 2 * A_BYTES), dBl = sdesc_sw128(base + 2 * A_BYTES + BROWS * ROWB);
            const int ksteps = min(O::BK, a.kpad - kb * O::BK) / O::KSTEP;
            for (int ks = 0; ks < ksteps; ks++) {
              const uint64_t off = (uint64_t)((ks * 32) >> 4);  // 32 bytes of K per MMA
              const uint32_t acc = (kb == 0 && ks == 0) ? 0u : 1u;
              if constexpr (PAIR) {
                umma_pair<O::F16>(dcol, dAl + off, dBh + off, O::IDESC_PAIR, acc);
                umma_pair<O::F16>(dcol, dAh + off, dBl + off, O::IDESC_PAIR, 1u);
                umma_pair<O::F16>(dcol, dAh + off, dBh + off, O::IDESC_PAIR, 1u);
              } else {
                umma<OP>(dcol, dAl + off, dBh + off, acc);
                umma<OP>(dcol, dAh + off, dBl + off, 1u);
                umma<OP>(dcol, dAh + off, dBh + off, 1u);
              }
            }
            commit(smem_u32(&bar_empty[s]));
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
      }
      if (!ok) break;
      if (lane == 0) commit(smem_u32(&bar_tfull[ts]));
      __syncwarp();
    }
    // drain: all issued MMAs (into both CTAs' tensor memory) complete before it is released
    if (lane == 0 && leader) {
      commit(smem_u32(&bar_final));
      drain_bar(smem_u32(&bar_final), 0);
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------------- epilogue
    // Items of a lane quadrant: (tile titer, k slot) in order it = 2 titer + slot;
    // the quadrant's NG warps take them round-robin.  A tile's accumulator is
    // released once all ITEMS_PER_TILE items are done, so no warp can fall two
    // phases behind a tensor-memory stage.
    constexpr int NG = epi_warps<MODE>() / 4;
    const int quad = warp & 3;
    const int widx = (warp - EPI_WARP0) >> 2;
    float *tab = reinterpret_cast<float *>(smem_raw + (smem0 - smem_u32(smem_raw)) + NSTAGE * STAGE);
    for (int it = widx;; it += NG) {
      const int titer = it >> 1, slot = it & 1;
      const int item = cid + titer * ncl;
      if (item >= nitems) break;
      const int ts = titer & 1;
      const uint32_t tpar = (titer >> 1) & 1;
      const bool ok = wait_bar(smem_u32(&bar_tfull[ts]), tpar, abort_flag, a.dstatus);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      int kg, qt;
      item_coords_p<PAIR>(a, item, rank, kg, qt);
      const int q = qt * BM + quad * 32 + lane;
      const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + ts * BN + slot * 128;
      if (qt < a.nqt) {  // (a pair's second tile may lie past the q list)
#pragma unroll 1
        for (int j = 0; j < S::KPS; j++) {
          const int k = kg * S::KPT + slot * S::KPS + j;
          epilogue_pair<NW, NM, MODE>(a, tbase + j * S::CPK, q, k, q < a.nq && k < a.nk, quad, qt, tab);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if constexpr (PAIR)
          mbar_arrive_cluster(tempty_c0 + 8u * (uint32_t)ts);
        else
          mbar_arrive(smem_u32(&bar_tempty[ts]));
      }
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

// ------------------------------------------------------- operand builders
template <typename T>
__device__ __forceinline__ void split_store(double v, T *hi, T *lo, size_t i);
template <>
__device__ __forceinline__ void split_store<__nv_bfloat16>(double v, __nv_bfloat16 *hi, __nv_bfloat16 *lo, size_t i) {
  const __nv_bfloat16 h = __double2bfloat16(v);
  hi[i] = h;
  lo[i] = __double2bfloat16(v - (double)__bfloat162float(h));
}
// tf32 term: an fp32 with its 13 low mantissa bits cleared after rounding to nearest
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  return __uint_as_float(u);
}
template <>
__device__ __forceinline__ void split_store<float>(double v, float *hi, float *lo, size_t i) {
  const float h = tf32_round((float)v);
  hi[i] = h;
  lo[i] = tf32_round((float)(v - (double)h));
}

// A[q][kk] (K-major hi/lo): kk = 2r + t, value cos / sin of 2 pi (q.R_r mod 1), R
// reversed (far shells first).  With a second set R2 (the vertex's Rp when it
// differs from Re), its phases follow at K offset kg0 (a multiple of 64), zero between.
template <typename T>
__global__ void k_build_a(int nq, int nR, int kpad, const double *__restrict__ q, const int *__restrict__ R, T *hi,
                          T *lo, int nR2 = 0, const int *__restrict__ R2 = nullptr, int kg0 = 0) {
  size_t n = (size_t)nq * kpad;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    int kk = (int)(idx % kpad);
    int iq = (int)(idx / kpad);
    double d = 0.0;
    const int *Rs = R;
    int nRs = nR, kl = kk;
    if (R2 && kk >= kg0) {
      Rs = R2;
      nRs = nR2;
      kl = kk - kg0;
    }
    if (kl < 2 * nRs) {
      int r = nRs - 1 - (kl >> 1);
      // argument q.R reduced to [-1/2, 1/2] in FP64; 2x = xh + xl with xh in FP32,
      // then sin/cos(pi xh) in FP32 and the first-order correction in pi xl
      // (|xl| <= 2^-25): about 1 FP32 ulp, below the 2^-22 of the two-term split.
      double x = q[3 * iq] * Rs[3 * r] + q[3 * iq + 1] * Rs[3 * r + 1] + q[3 * iq + 2] * Rs[3 * r + 2];
      x -= rint(x);
      const double x2 = 2.0 * x;
      const float xh = (float)x2;
      const float xl = (float)(x2 - (double)xh) * 3.14159265358979f;
      float s, c;
      sincospif(xh, &s, &c);
      d = (kl & 1) ? (double)fmaf(xl, c, s) : (double)fmaf(-xl, s, c);
    }
    split_store<T>(d, hi, lo, idx);
  }
}

// The same A operand from the FP64 q phases P [nR][nq] already formed for the
// phonons (same R set): a 32 x 32 tile transpose, no trigonometry.  Columns
// kk >= 2 nR (padding) are written by k_a_pad.
template <typename T>
__global__ void k_build_a_from(int nq, int nR, int kpad, const cx<double> *__restrict__ P, T *hi, T *lo) {
  __shared__ cx<double> tile[32][33];
  const int q0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = r0 + j, q = q0 + threadIdx.x;
    tile[j][threadIdx.x] = (r < nR && q < nq) ? P[(size_t)r * nq + q] : mkc(0.0, 0.0);
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int q = q0 + j;
    if (q >= nq) continue;
    for (int u = threadIdx.x; u < 64; u += 32) {
      const int rl = u >> 1, t = u & 1, r = r0 + rl;
      if (r >= nR) continue;
      const cx<double> v = tile[rl][j];
      split_store<T>(t ? v.y : v.x, hi, lo, (size_t)q * kpad + 2 * (nR - 1 - r) + t);
    }
  }
}
template <typename T>
__global__ void k_a_pad(int nq, int k0, int kpad, T *hi, T *lo) {
  const int w = kpad - k0;
  const size_t n = (size_t)nq * w;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    split_store<T>(0.0, hi, lo, (i / w) * kpad + k0 + i % w);
}

// hi/lo split of an FP32 value, in FP32: v - hi is exact (hi is v rounded to
// fewer mantissa bits), so this equals split_store of (double)v.
template <typename T>
__device__ __forceinline__ void split_store_f(float v, T *hi, T *lo, size_t i);
template <>
__device__ __forceinline__ void split_store_f<__nv_bfloat16>(float v, __nv_bfloat16 *hi, __nv_bfloat16 *lo, size_t i) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[i] = h;
  lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
}
template <>
__device__ __forceinline__ void split_store_f<float>(float v, float *hi, float *lo, size_t i) {
  const float h = tf32_round(v);
  hi[i] = h;
  lo[i] = tf32_round(v - h);
}

// B[k][col][kk] (K-major hi/lo) of the real GEMM:
//   col = 2c + s (s: re/im of output column c), kk = 2r + t (t: re/im of P_q(R_r)),
//   (s,t) = (0,0): Re b, (0,1): -Im b, (1,0): Im b, (1,1): Re b,  b = B_k[r][c].
// Output columns c: [0, nw^2) H(k+q)_ij, then (a, j, n) of g_a(k,q) U_k.
// planar != 0: columns in pairs, col = 4 (c/2) + 2s + c%2 (two real parts, then
// the two imaginary parts of the neighbouring output columns c, c+1), so that
// the epilogue reads one float2 of real parts and one of imaginary parts.
// Built through a shared-memory tile: a block reads 32 output columns c x 32 R
// vectors of B_k along c (coalesced) and writes the matching 64 real columns x 64
// K entries along K (coalesced).  Rows k >= nk, columns c >= nc and K >= 2 nR are 0.
template <typename T>
__global__ void k_build_b(int nk, int nk_pad, int nR, int nw, int nm, int cpk, int kpad, int planar,
                          const cx<float> *__restrict__ BH, const cx<float> *__restrict__ Bg, T *hi, T *lo, int nRp,
                          int kg0) {
  __shared__ cx<float> tile[32][33];  // [R index from the K tile][c - c0]
  const int nw2 = nw * nw;
  const int nc = nw2 * (nm + 1);
  const int c0 = blockIdx.y * 32;
  const int kk0 = blockIdx.x * 64;
  // K parts: one R set shared by H and the vertex (kg0 = 0), or H over Re in [0, 2 nRe)
  // and the vertex over Rp from kg0 (a multiple of 64, so a K tile lies in one part)
  const bool partG = kg0 > 0 && kk0 >= kg0;
  const int kb = partG ? kg0 : 0;
  const int rr0 = (kk0 - kb) >> 1;
  const int nRH = nR, nRG = kg0 > 0 ? nRp : nR;
  const int nRt = partG ? nRG : nRH;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int k = blockIdx.z; k < nk_pad; k += gridDim.z) {
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
      const int rr = rr0 + j, c = c0 + threadIdx.x;
      cx<float> b = mkc(0.0f, 0.0f);
      if (k < nk && rr < nRt && c < nc) {
        const int r = nRt - 1 - rr;
        if (c < nw2) {
          if (!partG) b = BH[((size_t)k * nRH + r) * nw2 + c];
        } else if (kg0 == 0 || partG) {
          b = Bg[((size_t)k * nRG + r) * nm * nw2 + (c - nw2)];
        }
      }
      tile[j][threadIdx.x] = b;
    }
    __syncthreads();
    for (int e = tid; e < 64 * 64; e += blockDim.x * blockDim.y) {
      const int kl = e & 63, cl = e >> 6;
      const int col = 2 * c0 + cl, kk = kk0 + kl;
      if (col >= cpk || kk >= kpad) continue;
      const int c = planar ? 2 * (col >> 2) + (col & 1) : col >> 1;
      const int sr = planar ? (col >> 1) & 1 : col & 1;
      float v = 0.0f;
      if (kk - kb < 2 * nRt) {
        const cx<float> b = tile[((kk - kb) >> 1) - rr0][c - c0];
        const int t = kk & 1;
        v = sr == 0 ? (t == 0 ? b.x : -b.y) : (t == 0 ? b.y : b.x);
      }
      split_store_f<T>(v, hi, lo, ((size_t)k * cpk + col) * kpad + kk);
    }
    __syncthreads();
  }
}

// nRp, kg0: the vertex's R set and its K offset when it differs from Re (else nRp = nR, kg0 = 0)
template <typename T>
void launch_build_b(int nk, int nk_pad, int nR, int nw, int nm, int cpk, int kpad, int planar, const cx<float> *BH,
                    const cx<float> *Bg, T *hi, T *lo, cudaStream_t st, int nRp = 0, int kg0 = 0) {
  const dim3 grid((kpad + 63) / 64, (cpk + 63) / 64, std::min(nk_pad, 65535));
  k_build_b<T><<<grid, dim3(32, 8), 0, st>>>(nk, nk_pad, nR, nw, nm, cpk, kpad, planar, BH, Bg, hi, lo,
                                             nRp > 0 ? nRp : nR, kg0);
  epw_count_launch();
}

// FP32 tables of the epilogue, evaluated once per call: Bose factors n(w_qnu, T)
// (in FP64), frequencies, q weights (wq null: 1/nq) and band energies at k.
__global__ void k_tc_tables(int nq, int nm, int nk, int nw, const double *__restrict__ omegaT, double T,
                            const double *__restrict__ wq, const double *__restrict__ epsk, float *nbT, float *omF,
                            float *wqF, float *ekF) {
  const size_t nqm = (size_t)nq * nm, nkw = (size_t)nk * nw;
  const size_t n = nqm + (size_t)nq + nkw;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (i < nqm) {
      const double w = omegaT[i];
      nbT[i] = (w > 0.0) ? (float)bose_d(w, T) : 0.0f;
      omF[i] = (float)w;
    } else if (i < nqm + nq) {
      const size_t j = i - nqm;
      wqF[j] = (float)(wq ? wq[j] : 1.0 / nq);
    } else {
      const size_t j = i - nqm - nq;
      ekF[j] = (float)epsk[j];
    }
  }
}

inline int grid_for(size_t n, int bs) {
  size_t b = (n + bs - 1) / bs;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

// A operand (q phases, split): from the FP64 phases when they exist, else computed here.
template <typename T>
void build_a(int nq, int nR, int kpad, const double *q, const int *R, const cx<double> *P64, T *hi, T *lo,
             cudaStream_t st, int nR2 = 0, const int *R2 = nullptr, int kg0 = 0) {
  if (R2 && kg0 > 0) {
    // two R sets (Re, then Rp at kg0): computed from q
    const size_t n = (size_t)nq * kpad;
    k_build_a<T><<<grid_for(n, 256), 256, 0, st>>>(nq, nR, kpad, q, R, hi, lo, nR2, R2, kg0);
    epw_count_launch();
  } else if (P64) {
    dim3 grid((nq + 31) / 32, (nR + 31) / 32);
    k_build_a_from<T><<<grid, dim3(32, 8), 0, st>>>(nq, nR, kpad, P64, hi, lo);
    epw_count_launch();
    if (kpad > 2 * nR) {
      const size_t n = (size_t)nq * (kpad - 2 * nR);
      k_a_pad<T><<<grid_for(n, 256), 256, 0, st>>>(nq, 2 * nR, kpad, hi, lo);
      epw_count_launch();
    }
  } else {
    const size_t n = (size_t)nq * kpad;
    k_build_a<T><<<grid_for(n, 256), 256, 0, st>>>(nq, nR, kpad, q, R, hi, lo);
    epw_count_launch();
  }
}

// ----------------------------------------------- q side in double-float
// An FP64 value carried as hi + lo (two FP32, |lo| <= ulp(hi)/2): products by the
// error-free FMA product of the high parts plus the cross terms (Dekker), sums by
// Knuth's TwoSum of the high parts; about 2^-47 relative per operation.  The
// *_rn intrinsics keep the compiler from contracting the error terms into FMAs.
struct dflt {
  float h, l;
};
__device__ __forceinline__ dflt df_make(double x) {
  const float h = (float)x;
  dflt r;
  r.h = h;
  r.l = (float)(x - (double)h);
  return r;
}
__device__ __forceinline__ dflt df_norm(float s, float e) {
  dflt r;
  r.h = __fadd_rn(s, e);
  r.l = __fsub_rn(e, __fsub_rn(r.h, s));
  return r;
}
__device__ __forceinline__ dflt df_mul(dflt a, dflt b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return df_norm(p, e);
}
__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
  const float s = __fadd_rn(a.h, b.h);
  const float v = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fadd_rn(__fsub_rn(a.h, __fsub_rn(s, v)), __fsub_rn(b.h, v)), __fadd_rn(a.l, b.l));
  return df_norm(s, e);
}
__device__ __forceinline__ dflt df_neg(dflt a) {
  a.h = -a.h;
  a.l = -a.l;
  return a;
}
struct dfcx {
  dflt x, y;
};
__device__ __forceinline__ dfcx dfc_mul(dfcx a, dfcx b) {
  dfcx r;
  r.x = df_add(df_mul(a.x, b.x), df_neg(df_mul(a.y, b.y)));
  r.y = df_add(df_mul(a.x, b.y), df_mul(a.y, b.x));
  return r;
}

template <typename T>
__device__ __forceinline__ void split_df(dflt v, T &hi, T &lo);
template <>
__device__ __forceinline__ void split_df<__nv_bfloat16>(dflt v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(v.h);
  lo = __float2bfloat16_rn(__fadd_rn(__fsub_rn(v.h, __bfloat162float(hi)), v.l));
}
template <>
__device__ __forceinline__ void split_df<float>(dflt v, float &hi, float &lo) {
  hi = tf32_round(v.h);
  lo = tf32_round(__fadd_rn(__fsub_rn(v.h, hi), v.l));
}

// Accumulator of a double-float sum: the high parts are added exactly by TwoSum
// and every rounding error (of the sums and of the products) gathers in lo,
// which is folded in once at the end.
struct dfacc {
  float h, l;
};
// acc += a * b (a, b double-float; the error-free product of the high parts)
__device__ __forceinline__ void dfa_fma(dfacc &acc, dflt a, dflt b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  const float s = __fadd_rn(acc.h, p);
  const float v = __fsub_rn(s, acc.h);
  const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, v)), __fsub_rn(p, v));
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(err, e));
}

// The q side of the fused tensor-core form in one pass, one thread per q
// (R = Rph = Re): the one-axis factors e^{2 pi i q_j n}, |n| <= rmax, from
// e^{2 pi i (q_j mod 1)} (FP64 argument reduction, sincospi) by double-float
// powers (negative n as conjugates), kept in shared memory; the phases
// P_q(R) = prod_j factor_j in double-float; the A operand row of q written
// directly (K index 2 (nR-1-r) + re/im, split hi/lo, zero up to kpad) in 16-byte
// chunks; and the mass-scaled dynamical matrix D(q) = sum_R P_q(R) Phi(R)
// accumulated in double-float and written in FP64 for the eigensolve.
constexpr int QS_RMAX = 8;
constexpr int QS_THREADS = 64;
template <typename T, int NM2>
__global__ void __launch_bounds__(QS_THREADS) k_qside_df(int nq, const double *__restrict__ q, int nR,
                                                         const int *__restrict__ R, int rmax,
                                                         const float4 *__restrict__ Phidf, int kpad, T *Ahi, T *Alo,
                                                         cx<double> *D) {
  extern __shared__ float4 fsh[];  // [3][2 rmax + 1][QS_THREADS]: (Re hi, Re lo, Im hi, Im lo)
  const int i = blockIdx.x * QS_THREADS + threadIdx.x;
  const int nf = 2 * rmax + 1;
  const int ii = i < nq ? i : nq - 1;
  for (int j = 0; j < 3; j++) {
    double a = q[3 * ii + j];
    a -= rint(a);
    double sn, cs;
    sincospi(2.0 * a, &sn, &cs);
    dfcx f1, f;
    f1.x = df_make(cs);
    f1.y = df_make(sn);
    f.x = df_make(1.0);
    f.y = df_make(0.0);
    float4 *col = fsh + (size_t)j * nf * QS_THREADS + threadIdx.x;
    col[rmax * QS_THREADS] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    for (int n = 1; n <= rmax; n++) {
      f = dfc_mul(f, f1);
      col[(rmax + n) * QS_THREADS] = make_float4(f.x.h, f.x.l, f.y.h, f.y.l);
      col[(rmax - n) * QS_THREADS] = make_float4(f.x.h, f.x.l, -f.y.h, -f.y.l);
    }
  }
  // each thread reads only its own column: no barrier needed
  if (i >= nq) return;
  dfacc ax[NM2], ay[NM2];
#pragma unroll
  for (int e = 0; e < NM2; e++) ax[e].h = ax[e].l = ay[e].h = ay[e].l = 0.0f;
  constexpr int PER = 16 / (int)sizeof(T);  // elements per 16-byte chunk
  constexpr int RB = PER / 2;               // R vectors per chunk
  T *hrow = Ahi + (size_t)i * kpad, *lrow = Alo + (size_t)i * kpad;
  const float4 *F0 = fsh + threadIdx.x + rmax * QS_THREADS;
  const float4 *F1 = F0 + nf * QS_THREADS, *F2 = F1 + nf * QS_THREADS;
  for (int rr0 = 0; rr0 < kpad / 2; rr0 += RB) {
    __align__(16) T hb[PER];
    __align__(16) T lb[PER];
#pragma unroll
    for (int u = 0; u < RB; u++) {
      const int rr = rr0 + u;  // K order: R index r = nR - 1 - rr
      T h0 = T(0.0f), l0 = T(0.0f), h1 = T(0.0f), l1 = T(0.0f);
      if (rr < nR) {
        const int r = nR - 1 - rr;
        const float4 g0 = F0[R[3 * r] * QS_THREADS], g1 = F1[R[3 * r + 1] * QS_THREADS],
                     g2 = F2[R[3 * r + 2] * QS_THREADS];
        dfcx a, b, c;
        a.x = {g0.x, g0.y};
        a.y = {g0.z, g0.w};
        b.x = {g1.x, g1.y};
        b.y = {g1.z, g1.w};
        c.x = {g2.x, g2.y};
        c.y = {g2.z, g2.w};
        const dfcx p = dfc_mul(dfc_mul(a, b), c);
        split_df<T>(p.x, h0, l0);
        split_df<T>(p.y, h1, l1);
        const dflt npy = df_neg(p.y);
        const float4 *ph = Phidf + (size_t)r * NM2;
#pragma unroll
        for (int e = 0; e < NM2; e++) {
          const float4 f = __ldg(ph + e);
          const dflt fx = {f.x, f.y}, fy = {f.z, f.w};
          dfa_fma(ax[e], p.x, fx);
          dfa_fma(ax[e], npy, fy);
          dfa_fma(ay[e], p.x, fy);
          dfa_fma(ay[e], p.y, fx);
        }
      }
      hb[2 * u] = h0;
      hb[2 * u + 1] = h1;
      lb[2 * u] = l0;
      lb[2 * u + 1] = l1;
    }
    *reinterpret_cast<uint4 *>(hrow + 2 * rr0) = *reinterpret_cast<const uint4 *>(hb);
    *reinterpret_cast<uint4 *>(lrow + 2 * rr0) = *reinterpret_cast<const uint4 *>(lb);
  }
  cx<double> *d = D + (size_t)i * NM2;
#pragma unroll
  for (int e = 0; e < NM2; e++)
    d[e] = mkc((double)ax[e].h + (double)ax[e].l, (double)ay[e].h + (double)ay[e].l);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2D tensor [rows][inner] (inner contiguous), box [box_rows][128 bytes], 128-byte swizzle.
bool make_map(CUtensorMap *map, const void *base, int op, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int esz = op == TC_OP_BF16 ? 2 : 4;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * esz};
  cuuint32_t box[2] = {(cuuint32_t)(ROWB / esz), box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, op == TC_OP_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool shape_info(int nw, int nm, int &cpk, int &kpt, int &planar) {
#define EPW_TC_SHAPE(W, M)                 \
  if (nw == W && nm == M) {                \
    cpk = Shape<W, M>::CPK;                \
    kpt = Shape<W, M>::KPT;                \
    planar = Shape<W, M>::PLANAR ? 1 : 0;  \
    return true;                           \
  }
  EPW_TC_SHAPE(4, 3)
  EPW_TC_SHAPE(1, 3)
  EPW_TC_SHAPE(2, 3)
#undef EPW_TC_SHAPE
  return false;
}

template <int OP, int NW, int NM, int MODE, bool PAIR = false>
cudaError_t launch_tc(const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &bh, const CUtensorMap &bl,
                      const TcArgs &a, cudaStream_t st) {
  constexpr int SMEM = tc_smem_bytes<PAIR>() + tab_bytes<NW, NM, MODE>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_tc_linewidth<OP, NW, NM, MODE, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if constexpr (PAIR) {
    // clusters of two CTAs, each cluster two q tiles of one k group per item
    const int items = a.nkg * ((a.nqt + 1) / 2);
    const int grid = 2 * (items < sms / 2 ? items : sms / 2);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(nthreads<MODE>(), 1, 1);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_tc_linewidth<OP, NW, NM, MODE, true>, ah, al, bh, bl, a);
    if (e != cudaSuccess) return e;
  } else {
    int items = a.nkg * a.nqt;
    int grid = items < sms ? items : sms;
    k_tc_linewidth<OP, NW, NM, MODE, false><<<grid, nthreads<MODE>(), SMEM, st>>>(ah, al, bh, bl, a);
  }
  return cudaGetLastError();
}

template <int OP, int MODE, bool PAIR = false>
cudaError_t launch_tc_shape(int nw, int nm, const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &bh,
                            const CUtensorMap &bl, const TcArgs &a, cudaStream_t st) {
  if (nw == 4 && nm == 3) return launch_tc<OP, 4, 3, MODE, PAIR>(ah, al, bh, bl, a, st);
  if (nw == 1 && nm == 3) return launch_tc<OP, 1, 3, MODE, PAIR>(ah, al, bh, bl, a, st);
  if (nw == 2 && nm == 3) return launch_tc<OP, 2, 3, MODE, PAIR>(ah, al, bh, bl, a, st);
  return cudaErrorInvalidValue;
}

}  // namespace

// K extent of the contraction: 2 nRe, or, when Rp differs from Re, the Re part padded
// to a multiple of 64 (kg0) followed by 2 nRp; rounded up to the K step kal.
static int k_layout(const epw_model *m, int kal, int &kg0) {
  if (m->same_ep) {
    kg0 = 0;
    return (2 * m->nRe + kal - 1) / kal * kal;
  }
  kg0 = (2 * m->nRe + 63) / 64 * 64;
  return (kg0 + 2 * m->nRp + kal - 1) / kal * kal;
}

// Operand builders, tensor maps and FP32 tables for the other tensor-core kernels.
void tc_build_b_raw(int op, int nk, int nk_pad, int nR, int nw, int nm, int cpk, int kpad, const cx<float> *BH,
                    const cx<float> *Bg, void *hi, void *lo, cudaStream_t st) {
  if (op == TC_OP_BF16)
    launch_build_b<__nv_bfloat16>(nk, nk_pad, nR, nw, nm, cpk, kpad, 0, BH, Bg, (__nv_bfloat16 *)hi,
                                  (__nv_bfloat16 *)lo, st);
  else
    launch_build_b<float>(nk, nk_pad, nR, nw, nm, cpk, kpad, 0, BH, Bg, (float *)hi, (float *)lo, st);
}
void tc_build_a_raw(int op, int nq, int nR, int kpad, const double *q, const int *R, const cx<double> *P64, void *hi,
                    void *lo, cudaStream_t st) {
  if (op == TC_OP_BF16)
    build_a<__nv_bfloat16>(nq, nR, kpad, q, R, P64, (__nv_bfloat16 *)hi, (__nv_bfloat16 *)lo, st);
  else
    build_a<float>(nq, nR, kpad, q, R, P64, (float *)hi, (float *)lo, st);
}
bool tc_make_map(CUtensorMap *map, const void *base, int op, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  return make_map(map, base, op, inner, rows, box_rows);
}
bool tc_make_map_rb(CUtensorMap *map, const void *base, int op, uint64_t inner, uint64_t rows, uint32_t box_rows,
                    int row_bytes) {
  auto fn = encode_fn();
  if (!fn || (row_bytes != 128 && row_bytes != 64)) return false;
  const int esz = op == TC_OP_BF16 ? 2 : 4;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * esz};
  cuuint32_t box[2] = {(cuuint32_t)(row_bytes / esz), box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, op == TC_OP_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}
void tc_tables(int nq, int nm, int nk, int nw, const double *omegaT, double T, const double *wq, const double *epsk,
               float *nbT, float *omF, float *wqF, float *ekF, cudaStream_t st) {
  const size_t n = (size_t)nq * nm + nq + (size_t)nk * nw;
  k_tc_tables<<<grid_for(n, 256), 256, 0, st>>>(nq, nm, nk, nw, omegaT, T, wq, epsk, nbT, omF, wqF, ekF);
  epw_count_launch();
}

void tc_build_b(const epw_model *m, int nk, const cx<float> *Bg32, const cx<float> *BH32, TcBuffers &b,
                cudaStream_t st) {
  if (b.op == TC_OP_BF16)
    launch_build_b<__nv_bfloat16>(nk, b.nk_pad, m->nRe, m->nw, m->nm, b.cpk, b.kpad, b.planar, BH32, Bg32,
                                  (__nv_bfloat16 *)b.Bhi, (__nv_bfloat16 *)b.Blo, st, m->nRp, b.kg0);
  else
    launch_build_b<float>(nk, b.nk_pad, m->nRe, m->nw, m->nm, b.cpk, b.kpad, b.planar, BH32, Bg32, (float *)b.Bhi,
                          (float *)b.Blo, st, m->nRp, b.kg0);
}

void tc_build_a(const epw_model *m, int nq, const double *q, TcBuffers &b, cudaStream_t st) {
  if (b.op == TC_OP_BF16)
    build_a<__nv_bfloat16>(nq, m->nRe, b.kpad, q, m->Re, b.Pq64, (__nv_bfloat16 *)b.Ahi, (__nv_bfloat16 *)b.Alo, st,
                           m->nRp, m->Rp, b.kg0);
  else
    build_a<float>(nq, m->nRe, b.kpad, q, m->Re, b.Pq64, (float *)b.Ahi, (float *)b.Alo, st, m->nRp, m->Rp, b.kg0);
}

bool tc_qside(const epw_model *m, int nq, const double *q, TcBuffers &b, cx<double> *D, cudaStream_t st) {
  if (!b.ok || !m->same_ep || !m->same_eph || m->nm != 3 || m->rmax > QS_RMAX || nq <= 0) return false;
  const int grid = (nq + QS_THREADS - 1) / QS_THREADS;
  const size_t sh = (size_t)3 * (2 * m->rmax + 1) * QS_THREADS * sizeof(float4);  // <= 52 KB
  static bool attr = false;
  if (!attr) {
    const int mx = (int)((size_t)3 * (2 * QS_RMAX + 1) * QS_THREADS * sizeof(float4));
    if (cudaFuncSetAttribute(k_qside_df<__nv_bfloat16, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_qside_df<float, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess)
      return false;
    attr = true;
  }
  if (b.op == TC_OP_BF16)
    k_qside_df<__nv_bfloat16, 9><<<grid, QS_THREADS, sh, st>>>(nq, q, m->nRe, m->Re, m->rmax, m->Phidf, b.kpad,
                                                                (__nv_bfloat16 *)b.Ahi, (__nv_bfloat16 *)b.Alo, D);
  else
    k_qside_df<float, 9><<<grid, QS_THREADS, sh, st>>>(nq, q, m->nRe, m->Re, m->rmax, m->Phidf, b.kpad,
                                                        (float *)b.Ahi, (float *)b.Alo, D);
  epw_count_launch();
  return true;
}

bool tc_supported(const epw_model *m) {
  int cpk, kpt, planar;
  return shape_info(m->nw, m->nm, cpk, kpt, planar);
}

epw_status tc_plan(Arena &A, const epw_model *m, int nk, int nq, int op, TcBuffers &b) {
  b = TcBuffers{};
  b.op = op;
  b.ok = shape_info(m->nw, m->nm, b.cpk, b.kpt, b.planar);
  if (!b.ok) return EPW_OK;
  const int esz = op == TC_OP_BF16 ? 2 : 4;
  const int kal = op == TC_OP_BF16 ? 16 : 8;  // K per MMA
  b.kpad = k_layout(m, kal, b.kg0);
  b.nk_pad = (nk + b.kpt - 1) / b.kpt * b.kpt;
  b.nqt = (nq + BM - 1) / BM;
  b.Ahi = A.take<char>((size_t)nq * b.kpad * esz);
  b.Alo = A.take<char>((size_t)nq * b.kpad * esz);
  b.Bhi = A.take<char>((size_t)b.nk_pad * b.cpk * b.kpad * esz);
  b.Blo = A.take<char>((size_t)b.nk_pad * b.cpk * b.kpad * esz);
  b.nbT = A.take<float>((size_t)nq * m->nm);
  b.omF = A.take<float>((size_t)nq * m->nm);
  b.wqF = A.take<float>((size_t)nq);
  b.ekF = A.take<float>((size_t)nk * m->nw);
  b.partial = A.take<double>((size_t)nk * 4 * b.nqt * m->nw);
  b.UkF = m->polar ? A.take<float2>((size_t)nk * m->nw * m->nw) : nullptr;
  return EPW_OK;
}

static epw_status tc_run(int mode, const epw_model *m, int nk, int nq, const double *q, const double *wq,
                         const epw_params *par, const double *epsk, const double *omegaT, const cx<float> *ET32,
                         const cx<float> *Bg32, const cx<float> *BH32, TcBuffers &b, double *out, double *eps_kq,
                         double *gout, cudaStream_t st) {
  if (!b.ok) return EPW_ERR_UNSUPPORTED;
  const int nR = m->nRe;
  const int op = b.op;
  const int esz = op == TC_OP_BF16 ? 2 : 4;
  {
    if (!b.prebuilt_a) tc_build_a(m, nq, q, b, st);
    if (!b.prebuilt_b) tc_build_b(m, nk, Bg32, BH32, b, st);
    b.prebuilt_a = b.prebuilt_b = false;
    size_t n = (size_t)nq * m->nm + nq + (size_t)nk * m->nw;
    k_tc_tables<<<grid_for(n, 256), 256, 0, st>>>(nq, m->nm, nk, m->nw, omegaT, par->T_K, wq, epsk, b.nbT, b.omF,
                                                   b.wqF, b.ekF);
    epw_count_launch();
    if (b.Cpol) launch_cast_c64_to_c32((size_t)nk * m->nw * m->nw, b.Uk64, (cx<float> *)b.UkF, st);
  }
  // the linewidth form runs on CTA pairs unless EPW_NARROW_FORM=single (each CTA of a pair
  // loads half of the B rows)
  const char *nf = getenv("EPW_NARROW_FORM");
  const bool pair = mode == 0 && !(nf && strcmp(nf, "single") == 0);
  CUtensorMap ah, al, bh, bl;
  std::memset(&ah, 0, sizeof(ah));
  if (!make_map(&ah, b.Ahi, op, b.kpad, nq, BM) || !make_map(&al, b.Alo, op, b.kpad, nq, BM) ||
      !make_map(&bh, b.Bhi, op, b.kpad, (uint64_t)b.nk_pad * b.cpk, pair ? BN / 2 : BN) ||
      !make_map(&bl, b.Blo, op, b.kpad, (uint64_t)b.nk_pad * b.cpk, pair ? BN / 2 : BN))
    return EPW_ERR_CUDA;
  TcArgs a;
  a.nk = nk;
  a.nq = nq;
  a.nqt = b.nqt;
  a.nkg = b.nk_pad / b.kpt;
  a.kpad = b.kpad;
  const int bk = ROWB / esz;
  a.nkb = (b.kpad + bk - 1) / bk;
  {
    const size_t atile = (size_t)BM * b.kpad * esz * 2;
    int qb = (int)((b.a_block_bytes ? b.a_block_bytes : A_BLOCK_BYTES) / atile);
    if (qb < 152) qb = 152;
    if (qb > b.nqt) qb = b.nqt;
    a.qblock = qb < 1 ? 1 : qb;
  }
  a.epsk = b.ekF;
  a.omegaT = b.omF;
  a.nbT = b.nbT;
  a.ET = (const float2 *)ET32;
  a.wq = b.wqF;
  a.EF = (float)par->EF_eV;
  a.invkT = par->T_K > 0.0 ? (float)(1.0 / (EPW_KB * par->T_K)) : 0.0f;
  a.inv_sigma = (float)(1.0 / par->sigma_eV);
  a.gnorm = (float)(1.0 / (par->sigma_eV * 1.7724538509055160273));
  a.omega_min = (float)par->omega_min_eV;
  a.partial = b.partial;
  a.eps_kq = eps_kq;
  a.gout = (double2 *)gout;
  a.dstatus = m->dstatus;
  a.Cpol = b.Cpol;
  a.UkF = b.Cpol ? b.UkF : nullptr;
  cudaError_t e;
  if (mode == 0) {
    epw_timing_begin(const_cast<epw_model *>(m), st);
    if (pair)
      e = op == TC_OP_BF16 ? launch_tc_shape<TC_OP_BF16, 0, true>(m->nw, m->nm, ah, al, bh, bl, a, st)
                           : launch_tc_shape<TC_OP_TF32, 0, true>(m->nw, m->nm, ah, al, bh, bl, a, st);
    else
      e = op == TC_OP_BF16 ? launch_tc_shape<TC_OP_BF16, 0>(m->nw, m->nm, ah, al, bh, bl, a, st)
                           : launch_tc_shape<TC_OP_TF32, 0>(m->nw, m->nm, ah, al, bh, bl, a, st);
    epw_timing_end(const_cast<epw_model *>(m), st);
  } else {
    e = op == TC_OP_BF16 ? launch_tc_shape<TC_OP_BF16, 1>(m->nw, m->nm, ah, al, bh, bl, a, st)
                         : launch_tc_shape<TC_OP_TF32, 1>(m->nw, m->nm, ah, al, bh, bl, a, st);
  }
  epw_count_launch();
  if (e != cudaSuccess) return EPW_ERR_CUDA;
  if (mode == 0) launch_finalize(nk, 4 * b.nqt, m->nw, b.partial, out, st);
  return EPW_OK;
}

epw_status tc_linewidth(const epw_model *m, int nk, const double *k, int nq, const double *q, const double *wq,
                        const epw_params *par, const cx<double> *PkRM, const double *epsk, const cx<double> *Uk,
                        const double *omegaT, const cx<float> *ET32, const cx<float> *Bg32, const cx<float> *BH32,
                        TcBuffers &b, double *out, cudaStream_t st) {
  (void)k;
  (void)PkRM;
  (void)Uk;
  return tc_run(0, m, nk, nq, q, wq, par, epsk, omegaT, ET32, Bg32, BH32, b, out, nullptr, nullptr, st);
}

epw_status tc_interp(const epw_model *m, int nk, int nq, const double *q, double omega_min, const double *epsk,
                     const double *omegaT, const cx<float> *ET32, const cx<float> *Bg32, const cx<float> *BH32,
                     TcBuffers &b, double *eps_kq, double *g, cudaStream_t st) {
  epw_params par;
  std::memset(&par, 0, sizeof(par));
  par.T_K = 0.0;
  par.sigma_eV = 1.0;
  par.omega_min_eV = omega_min;
  return tc_run(1, m, nk, nq, q, nullptr, &par, epsk, omegaT, ET32, Bg32, BH32, b, nullptr, eps_kq, g, st);
}

void tc_free(epw_model *) {}

// ===================================================================== adjoint
// dL/dg on the tensor cores, for L = sum_{k,n} c_nk Im Sigma_nk.  Per chunk of k:
//  1. the fused kernel in MODE 2 recomputes the forward per pair and writes
//     Xbar(k,q) = dL/d(g U_k)(k,q)* as rows (k, a, j, n) with K index 2q + (re,im);
//  2. a split-K tcgen05 GEMM contracts them with conj(P_q(R)) over q:
//     Bbar[R][k][a j n] = sum_q conj(e^{2 pi i q.R}) Xbar(k,q)_{a j n};
//  3. the k-side adjoint (U_k rotation, conj(P_k(Re)) contraction) runs as in
//     the SIMT form.
namespace {

constexpr int G_NT = 144;                          // N tile: rows of the conj-phase operand
constexpr int G_A_BYTES = 128 * ROWB;              // 16 KiB
constexpr int G_B_BYTES = G_NT * ROWB;             // 18 KiB
constexpr int G_STAGE = 2 * G_A_BYTES + 2 * G_B_BYTES;
constexpr int G_STAGES = 3;
constexpr int G_SMEM = G_STAGES * G_STAGE + 1024;
constexpr int G_THREADS = 192;                     // producer, MMA, 4 epilogue warps
// D=F32, K-major, N=144, M=128; A=B=TF32 (kind::tf32) or BF16 (kind::f16)
template <int OP>
constexpr uint32_t g_idesc() {
  return (1u << 4) | ((OP == TC_OP_BF16 ? 1u : 2u) << 7) | ((OP == TC_OP_BF16 ? 1u : 2u) << 10) |
         ((uint32_t)(G_NT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

struct GemmArgs {
  int mtiles, ntiles, splits, kblocks, kb_per_split;
  int ldc;   // rows of Ct are padded to mtiles * 128
  int npad;  // ntiles * G_NT
  float *Ct; // [splits][npad][ldc]: transposed partial products
  int qmajor;  // instead Ct[m][n] with row length ldn (one split)
  size_t ldn;
  unsigned *dstatus;
};

template <int OP>
__device__ __forceinline__ void umma_n144(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  if constexpr (OP == TC_OP_BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(g_idesc<OP>()), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(g_idesc<OP>()), "r"(acc)
        : "memory");
  }
}

// Ct[sp][n][m] = sum_{K blocks of split sp} A[m][K] B[n][K]   (two-term split, three MMAs;
// a K block is one 128-byte row: 32 tf32 or 64 bf16 elements)
template <int OP>
__global__ void __launch_bounds__(G_THREADS, 1)
    k_tc_gemm_nt(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                 const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, GemmArgs g) {
  __shared__ __align__(8) uint64_t bar_full[G_STAGES], bar_empty[G_STAGES], bar_tfull[2], bar_tempty[2], bar_final;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t smem0 = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int *abort_flag = &abort_sh;
  const int nitems = g.mtiles * g.ntiles * g.splits;
  if (threadIdx.x == 0) {
    for (int s = 0; s < G_STAGES; s++) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int s = 0; s < 2; s++) {
      mbar_init(smem_u32(&bar_tfull[s]), 1);
      mbar_init(smem_u32(&bar_tempty[s]), 4);
    }
    mbar_init(smem_u32(&bar_final), 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(&tmem_base_sh), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  auto coords = [&](int item, int &mt, int &nt, int &sp, int &kb0, int &kb1) {
    sp = item % g.splits;
    const int rest = item / g.splits;
    nt = rest % g.ntiles;
    mt = rest / g.ntiles;
    kb0 = sp * g.kb_per_split;
    kb1 = min(g.kblocks, kb0 + g.kb_per_split);
  };
  if (warp == 0) {
    int issued[G_STAGES] = {0, 0, 0};
    uint32_t it = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      int mt, nt, sp, kb0, kb1;
      coords(item, mt, nt, sp, kb0, kb1);
      for (int kb = kb0; kb < kb1; kb++, it++) {
        const int s = it % G_STAGES;
        const uint32_t par = ((it / G_STAGES) & 1u) ^ 1u;
        if (lane == 0) {
          ok = wait_bar(smem_u32(&bar_empty[s]), par, abort_flag, g.dstatus);
          if (ok) {
            const uint32_t base = smem0 + s * G_STAGE;
            const uint32_t fb = smem_u32(&bar_full[s]);
            mbar_expect_tx(fb, G_STAGE);
            const int kx = kb * OpT<OP>::BK;
            tma_load_2d(base, &mAhi, kx, mt * 128, fb);
            tma_load_2d(base + G_A_BYTES, &mAlo, kx, mt * 128, fb);
            tma_load_2d(base + 2 * G_A_BYTES, &mBhi, kx, nt * G_NT, fb);
            tma_load_2d(base + 2 * G_A_BYTES + G_B_BYTES, &mBlo, kx, nt * G_NT, fb);
#pragma unroll
            for (int z = 0; z < G_STAGES; z++)
              if (z == s) issued[z] = (int)(it / G_STAGES) + 1;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int z = 0; z < G_STAGES; z++)
        if (issued[z] > 0) drain_bar(smem_u32(&bar_full[z]), (uint32_t)((issued[z] - 1) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    uint32_t it = 0;
    int titer = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, titer++) {
      int mt, nt, sp, kb0, kb1;
      coords(item, mt, nt, sp, kb0, kb1);
      const int ts = titer & 1;
      const uint32_t tpar = ((titer >> 1) & 1) ^ 1;
      if (lane == 0) ok = wait_bar(smem_u32(&bar_tempty[ts]), tpar, abort_flag, g.dstatus);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
      const uint32_t dcol = tmem + ts * 256;
      for (int kb = kb0; kb < kb1; kb++, it++) {
        const int s = it % G_STAGES;
        const uint32_t par = (it / G_STAGES) & 1u;
        if (lane == 0) {
          ok = wait_bar(smem_u32(&bar_full[s]), par, abort_flag, g.dstatus);
          if (ok) {
            tc_fence_after();
            const uint32_t base = smem0 + s * G_STAGE;
            const uint64_t dAh = sdesc_sw128(base), dAl = sdesc_sw128(base + G_A_BYTES);
            const uint64_t dBh = sdesc_sw128(base + 2 * G_A_BYTES), dBl = sdesc_sw128(base + 2 * G_A_BYTES + G_B_BYTES);
#pragma unroll
            for (int ks = 0; ks < 4; ks++) {  // 4 MMAs of 32 bytes of K each
              const uint64_t off = (uint64_t)((ks * 32) >> 4);
              const uint32_t acc = (kb == kb0 && ks == 0) ? 0u : 1u;
              umma_n144<OP>(dcol, dAl + off, dBh + off, acc);
              umma_n144<OP>(dcol, dAh + off, dBl + off, 1u);
              umma_n144<OP>(dcol, dAh + off, dBh + off, 1u);
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
    const int quad = warp & 3;
    int titer = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, titer++) {
      int mt, nt, sp, kb0, kb1;
      coords(item, mt, nt, sp, kb0, kb1);
      const int ts = titer & 1;
      const uint32_t tpar = (titer >> 1) & 1;
      const bool ok = wait_bar(smem_u32(&bar_tfull[ts]), tpar, abort_flag, g.dstatus);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const int m = mt * 128 + quad * 32 + lane;
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + ts * 256;
      // column-major partials (stride ldc), or one q-major row per thread (32-byte stores)
      const size_t cs = g.qmajor ? 1 : (size_t)g.ldc;
      float *out = g.qmajor ? g.Ct + (size_t)m * g.ldn + (size_t)nt * G_NT
                            : g.Ct + ((size_t)sp * g.npad + (size_t)nt * G_NT) * g.ldc + m;
#pragma unroll 1
      for (int c0 = 0; c0 < 128; c0 += 32) {
        float v[32];
        tmem_ld32(taddr + c0, v);
        if (g.qmajor) {
#pragma unroll
          for (int c = 0; c < 32; c += 4)
            *reinterpret_cast<float4 *>(out + c0 + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < 32; c++) out[(size_t)(c0 + c) * cs] = v[c];
        }
      }
#pragma unroll
      for (int c0 = 128; c0 < G_NT; c0 += 8) {
        float v[8];
        tmem_ld8(taddr + c0, v);
#pragma unroll
        for (int c = 0; c < 8; c++) out[(size_t)(c0 + c) * cs] = v[c];
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
    tmem_dealloc(tmem, 512);
  }
}

// conj-phase operand P[n][kk] (tf32 hi/lo), n = 2r + s, kk = 2q + t:
//   (s,t) = (0,0): cos, (0,1): sin, (1,0): -sin, (1,1): cos  of 2 pi (q.R_r mod 1)
// so that row 2r of Xbar P^T is Re sum_q conj(P_q(R_r)) Xbar and row 2r+1 its Im.
__global__ void k_build_pconj(int nq, int nR, int ld, const double *__restrict__ q, const int *__restrict__ R,
                              float *hi, float *lo) {
  size_t n = (size_t)nq * 2 * nR;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int iq = (int)(idx % nq);
    const int row = (int)(idx / nq);
    const int r = row >> 1, s = row & 1;
    double x = q[3 * iq] * R[3 * r] + q[3 * iq + 1] * R[3 * r + 1] + q[3 * iq + 2] * R[3 * r + 2];
    x -= rint(x);
    const double x2 = 2.0 * x;
    const float xh = (float)x2;
    const float xl = (float)(x2 - (double)xh) * 3.14159265358979f;
    float sn, cs;
    sincospif(xh, &sn, &cs);
    const float c = fmaf(-xl, sn, cs), sv = fmaf(xl, cs, sn);
    const float v0 = s == 0 ? c : -sv, v1 = s == 0 ? sv : c;
    const size_t o = (size_t)row * ld + 2 * (size_t)iq;
    const float h0 = tf32_rn(v0), h1 = tf32_rn(v1);
    *reinterpret_cast<float2 *>(hi + o) = make_float2(h0, h1);
    *reinterpret_cast<float2 *>(lo + o) = make_float2(tf32_rn(v0 - h0), tf32_rn(v1 - h1));
  }
}

// Bbar[r][kl][c] = sum_sp (Ct[sp][2r][m], Ct[sp][2r+1][m]),  m = kl*nc + c, fixed order.
__global__ void k_xbar_reduce(int nR, int kc, int nc, int splits, int npad, int ldc, const float *__restrict__ Ct,
                              cx<float> *Bbar) {
  size_t n = (size_t)nR * kc * nc;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % nc);
    const size_t rest = idx / nc;
    const int kl = (int)(rest % kc);
    const int r = (int)(rest / kc);
    const size_t m = (size_t)kl * nc + c;
    float re = 0.0f, im = 0.0f;
    for (int sp = 0; sp < splits; sp++) {
      re += Ct[((size_t)sp * npad + 2 * r) * ldc + m];
      im += Ct[((size_t)sp * npad + 2 * r + 1) * ldc + m];
    }
    Bbar[idx] = mkc(re, im);
  }
}

__global__ void k_cot_table(size_t n, const double *__restrict__ cot, float *cotF) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    cotF[i] = (float)cot[i];
}

bool make_map_f32(CUtensorMap *map, const void *base, uint64_t inner, uint64_t ld, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {ld * 4};
  cuuint32_t box[2] = {32, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

epw_status tc_bwd_plan(Arena &A, const epw_model *m, int nk, int nq, TcBuffers &b, TcBwdBuffers &w) {
  CKS_TC(tc_plan(A, m, nk, nq, TC_OP_TF32, b));
  w = TcBwdBuffers{};
  if (!b.ok) return EPW_OK;
  const int nc = m->nm * m->nw * m->nw;
  w.nc = nc;
  w.ld = (2 * nq + 31) / 32 * 32;
  const size_t row_bytes = (size_t)nc * w.ld * 4 * 2;  // per k, hi + lo
  int kc = (int)std::min<size_t>((size_t)nk, std::max<size_t>(2, ((size_t)2 << 30) / std::max<size_t>(row_bytes, 1)));
  kc = (kc + 1) / 2 * 2;
  w.kc = kc;
  w.mtiles = (kc * nc + 127) / 128;
  w.ntiles = (2 * m->nRe + G_NT - 1) / G_NT;
  w.kblocks = (2 * nq + 31) / 32;
  const int tiles = w.mtiles * w.ntiles;
  int splits = std::max(1, std::min(w.kblocks, (2 * 152 + tiles - 1) / tiles));
  w.kb_per_split = (w.kblocks + splits - 1) / splits;
  w.splits = (w.kblocks + w.kb_per_split - 1) / w.kb_per_split;
  w.ldc = w.mtiles * 128;
  w.npad = w.ntiles * G_NT;
  w.phi = A.take<float>((size_t)2 * m->nRe * w.ld);
  w.plo = A.take<float>((size_t)2 * m->nRe * w.ld);
  w.xhi = A.take<float>((size_t)kc * nc * w.ld);
  w.xlo = A.take<float>((size_t)kc * nc * w.ld);
  w.Ct = A.take<float>((size_t)w.splits * w.npad * w.ldc);
  w.Bbar = A.take<cx<float>>((size_t)m->nRp * kc * nc);
  w.G1bar = A.take<cx<float>>((size_t)m->nRp * kc * nc);
  w.cotF = A.take<float>((size_t)nk * m->nw);
  w.partT = A.take<double>((size_t)kc * 4 * b.nqt);
  w.partE = A.take<double>((size_t)kc * 4 * b.nqt);
  return EPW_OK;
}

// ------------------------------------------------------ staged adjoint
// The q contraction of the staged adjoint, Bbar[Rp][kl nc + c] = sum_q conj(P_q(Rp)) Xbar[q][kl][c],
// as the same split-TF32 GEMM on the tensor cores: Xbar (FP32 complex, q-major, written by the
// per-pair adjoint kernel) is transposed into K-major rows split into two tf32 terms, K index
// 2q + (re, im), against the conj-phase operand of the Rp set.

// xhi/xlo[m][2q + t] (t = re, im) from xbar[q][m], m < nrow: 32 x 32 tiles through shared memory
__global__ void k_xbar_split(int nq, int nrow, int ld, const float2 *__restrict__ xbar, float *hi, float *lo) {
  __shared__ float2 tile[32][33];
  const int tq = (nq + 31) / 32, tm = (nrow + 31) / 32;
  for (int t = blockIdx.x; t < tq * tm; t += gridDim.x) {
    const int q0 = (t / tm) * 32, m0 = (t % tm) * 32;
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
      const int q = q0 + i, mm = m0 + threadIdx.x;
      tile[i][threadIdx.x] = (q < nq && mm < nrow) ? xbar[(size_t)q * nrow + mm] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
      const int mm = m0 + i, q = q0 + threadIdx.x;
      if (mm < nrow && q < nq) {
        const float2 v = tile[threadIdx.x][i];
        const float h0 = tf32_rn(v.x), h1 = tf32_rn(v.y);
        const size_t o = (size_t)mm * ld + 2 * (size_t)q;
        *reinterpret_cast<float2 *>(hi + o) = make_float2(h0, h1);
        *reinterpret_cast<float2 *>(lo + o) = make_float2(tf32_rn(v.x - h0), tf32_rn(v.y - h1));
      }
    }
  }
}

epw_status tc_sbwd_plan(Arena &A, const epw_model *m, int nq, int kc, TcBwdBuffers &w) {
  w = TcBwdBuffers{};
  const int nc = m->nm * m->nw * m->nw;
  w.nc = nc;
  w.ld = (2 * nq + 31) / 32 * 32;
  w.kc = kc;
  w.mtiles = (kc * nc + 127) / 128;
  w.ntiles = (2 * m->nRp + G_NT - 1) / G_NT;
  w.kblocks = (2 * nq + 31) / 32;
  const int tiles = w.mtiles * w.ntiles;
  const int splits = std::max(1, std::min(w.kblocks, (2 * 152 + tiles - 1) / tiles));
  w.kb_per_split = (w.kblocks + splits - 1) / splits;
  w.splits = (w.kblocks + w.kb_per_split - 1) / w.kb_per_split;
  w.ldc = w.mtiles * 128;
  w.npad = w.ntiles * G_NT;
  w.phi = A.take<float>((size_t)2 * m->nRp * w.ld);
  w.plo = A.take<float>((size_t)2 * m->nRp * w.ld);
  w.xhi = A.take<float>((size_t)kc * nc * w.ld);
  w.xlo = A.take<float>((size_t)kc * nc * w.ld);
  w.Ct = A.take<float>((size_t)w.splits * w.npad * w.ldc);
  return EPW_OK;
}

epw_status tc_sbwd_phases(const epw_model *m, int nq, const double *q, TcBwdBuffers &w, cudaStream_t st) {
  const size_t n = (size_t)nq * 2 * m->nRp;
  k_build_pconj<<<grid_for(n, 256), 256, 0, st>>>(nq, m->nRp, w.ld, q, m->Rp, w.phi, w.plo);
  epw_count_launch();
  return cudaGetLastError() == cudaSuccess ? EPW_OK : EPW_ERR_CUDA;
}

epw_status tc_sbwd_contract(const epw_model *m, int kc, int nq, const cx<float> *xbar, TcBwdBuffers &w,
                            cx<float> *Bbar, cudaStream_t st) {
  if (kc > w.kc) return EPW_ERR_UNSUPPORTED;
  const int nc = w.nc, M = kc * nc;
  {
    const int tiles = ((nq + 31) / 32) * ((M + 31) / 32);
    k_xbar_split<<<std::min(tiles, 152 * 16), dim3(32, 8), 0, st>>>(nq, M, w.ld, (const float2 *)xbar, w.xhi, w.xlo);
    epw_count_launch();
  }
  CUtensorMap xh, xl, ph, pl;
  if (!make_map_f32(&xh, w.xhi, 2 * (uint64_t)nq, w.ld, (uint64_t)M, 128) ||
      !make_map_f32(&xl, w.xlo, 2 * (uint64_t)nq, w.ld, (uint64_t)M, 128) ||
      !make_map_f32(&ph, w.phi, 2 * (uint64_t)nq, w.ld, 2 * (uint64_t)m->nRp, G_NT) ||
      !make_map_f32(&pl, w.plo, 2 * (uint64_t)nq, w.ld, 2 * (uint64_t)m->nRp, G_NT))
    return EPW_ERR_CUDA;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_tc_gemm_nt<TC_OP_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM) !=
        cudaSuccess)
      return EPW_ERR_CUDA;
    attr = true;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  GemmArgs g;
  g.mtiles = (M + 127) / 128;
  g.ntiles = w.ntiles;
  g.kblocks = w.kblocks;
  g.kb_per_split = w.kb_per_split;
  g.splits = w.splits;
  g.ldc = w.ldc;
  g.npad = w.npad;
  g.Ct = w.Ct;
  g.qmajor = 0;
  g.ldn = 0;
  g.dstatus = m->dstatus;
  const int items = g.mtiles * g.ntiles * g.splits;
  k_tc_gemm_nt<TC_OP_TF32><<<std::min(items, sms), G_THREADS, G_SMEM, st>>>(xh, xl, ph, pl, g);
  epw_count_launch();
  if (cudaGetLastError() != cudaSuccess) return EPW_ERR_CUDA;
  const size_t nred = (size_t)m->nRp * kc * nc;
  k_xbar_reduce<<<grid_for(nred, 256), 256, 0, st>>>(m->nRp, kc, nc, g.splits, g.npad, g.ldc, w.Ct, Bbar);
  epw_count_launch();
  return cudaGetLastError() == cudaSuccess ? EPW_OK : EPW_ERR_CUDA;
}

epw_status tc_linewidth_backward(const epw_model *m, int nk, int nq, const double *q, const double *wq,
                                 const epw_params *par, const double *epsk, const cx<double> *Uk,
                                 const cx<float> *Pk32, const double *omegaT, const cx<float> *ET32,
                                 const cx<float> *Bg32, const cx<float> *BH32, const double *cot, TcBuffers &b,
                                 TcBwdBuffers &w, cx<float> *gwbar, double *scal, cudaStream_t st) {
  if (!b.ok) return EPW_ERR_UNSUPPORTED;
  const int nR = m->nRe, nw = m->nw, nc = w.nc;
  // forward operands (tf32 split), epilogue tables, conj-phase operand, cotangent table
  {
    build_a<float>(nq, nR, b.kpad, q, m->Re, b.Pq64, (float *)b.Ahi, (float *)b.Alo, st);
    launch_build_b<float>(nk, b.nk_pad, nR, nw, m->nm, b.cpk, b.kpad, b.planar, BH32, Bg32, (float *)b.Bhi,
                          (float *)b.Blo, st);
    size_t n = (size_t)nq * m->nm + nq + (size_t)nk * nw;
    k_tc_tables<<<grid_for(n, 256), 256, 0, st>>>(nq, m->nm, nk, nw, omegaT, par->T_K, wq, epsk, b.nbT, b.omF,
                                                   b.wqF, b.ekF);
    epw_count_launch();
    n = (size_t)nq * 2 * nR;
    k_build_pconj<<<grid_for(n, 256), 256, 0, st>>>(nq, nR, w.ld, q, m->Re, w.phi, w.plo);
    epw_count_launch();
    n = (size_t)nk * nw;
    k_cot_table<<<grid_for(n, 256), 256, 0, st>>>(n, cot, w.cotF);
    epw_count_launch();
    if (b.Cpol) launch_cast_c64_to_c32((size_t)nk * nw * nw, b.Uk64, (cx<float> *)b.UkF, st);
  }
  CUtensorMap ah, al, ph, pl;
  if (!make_map(&ah, b.Ahi, TC_OP_TF32, b.kpad, nq, BM) || !make_map(&al, b.Alo, TC_OP_TF32, b.kpad, nq, BM) ||
      !make_map_f32(&ph, w.phi, 2 * (uint64_t)nq, w.ld, 2 * (uint64_t)nR, G_NT) ||
      !make_map_f32(&pl, w.plo, 2 * (uint64_t)nq, w.ld, 2 * (uint64_t)nR, G_NT))
    return EPW_ERR_CUDA;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_tc_gemm_nt<TC_OP_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM) !=
        cudaSuccess)
      return EPW_ERR_CUDA;
    attr = true;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int k0 = 0; k0 < nk; k0 += w.kc) {
    const int kc = std::min(w.kc, nk - k0);
    const int kc_pad = (kc + b.kpt - 1) / b.kpt * b.kpt;
    CUtensorMap bh, bl;
    const size_t boff = (size_t)k0 * b.cpk * b.kpad;
    if (!make_map(&bh, (const float *)b.Bhi + boff, TC_OP_TF32, b.kpad, (uint64_t)kc_pad * b.cpk, BN) ||
        !make_map(&bl, (const float *)b.Blo + boff, TC_OP_TF32, b.kpad, (uint64_t)kc_pad * b.cpk, BN))
      return EPW_ERR_CUDA;
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nk = kc;
    a.nq = nq;
    a.nqt = b.nqt;
    a.nkg = kc_pad / b.kpt;
    a.kpad = b.kpad;
    a.nkb = (b.kpad + 31) / 32;
    {
      const size_t atile = (size_t)BM * b.kpad * 4 * 2;
      int qb = (int)(A_BLOCK_BYTES / atile);
      qb = std::max(qb, 152);
      qb = std::min(qb, b.nqt);
      a.qblock = std::max(qb, 1);
    }
    a.epsk = b.ekF + (size_t)k0 * nw;
    a.omegaT = b.omF;
    a.nbT = b.nbT;
    a.ET = (const float2 *)ET32;
    a.wq = b.wqF;
    a.EF = (float)par->EF_eV;
    a.invkT = (float)(1.0 / (EPW_KB * par->T_K));
    a.inv_sigma = (float)(1.0 / par->sigma_eV);
    a.gnorm = (float)(1.0 / (par->sigma_eV * 1.7724538509055160273));
    a.omega_min = (float)par->omega_min_eV;
    a.cot = w.cotF + (size_t)k0 * nw;
    a.xhi = w.xhi;
    a.xlo = w.xlo;
    a.ldx = w.ld;
    a.partT = w.partT;
    a.partE = w.partE;
    a.T = (float)par->T_K;
    a.dstatus = m->dstatus;
    a.Cpol = b.Cpol;
    a.UkF = b.Cpol ? b.UkF + (size_t)k0 * nw * nw : nullptr;
    cudaError_t e = launch_tc_shape<TC_OP_TF32, 2>(nw, m->nm, ah, al, bh, bl, a, st);
    epw_count_launch();
    if (e != cudaSuccess) return EPW_ERR_CUDA;
    launch_sum_scalar(kc * 4 * b.nqt, w.partT, 1.0, scal, st);
    launch_sum_scalar(kc * 4 * b.nqt, w.partE, 1.0, scal + 1, st);
    // q contraction on the tensor cores (split K), then the fixed-order reduction
    const int M = kc * nc;
    CUtensorMap xh, xl;
    if (!make_map_f32(&xh, w.xhi, 2 * (uint64_t)nq, w.ld, (uint64_t)M, 128) ||
        !make_map_f32(&xl, w.xlo, 2 * (uint64_t)nq, w.ld, (uint64_t)M, 128))
      return EPW_ERR_CUDA;
    GemmArgs g;
    g.mtiles = (M + 127) / 128;
    g.ntiles = w.ntiles;
    g.kblocks = w.kblocks;
    g.kb_per_split = w.kb_per_split;
    g.splits = w.splits;
    g.ldc = w.ldc;
    g.npad = w.npad;
    g.Ct = w.Ct;
    g.qmajor = 0;
    g.ldn = 0;
    g.dstatus = m->dstatus;
    const int items = g.mtiles * g.ntiles * g.splits;
    k_tc_gemm_nt<TC_OP_TF32><<<std::min(items, sms), G_THREADS, G_SMEM, st>>>(xh, xl, ph, pl, g);
    epw_count_launch();
    if (cudaGetLastError() != cudaSuccess) return EPW_ERR_CUDA;
    const size_t nred = (size_t)m->nRp * kc * nc;
    k_xbar_reduce<<<grid_for(nred, 256), 256, 0, st>>>(m->nRp, kc, nc, g.splits, g.npad, g.ldc, w.Ct, w.Bbar);
    epw_count_launch();
    // k side: rotation adjoint, then conj(P_k(Re)) contraction into gwbar
    launch_bg_adjoint_rotate_k0<float>(kc, k0, m->nRp, m->nm, nw, w.Bbar, Uk, w.G1bar, st);
    const int ncol2 = m->nRp * nc;
    launch_cgemm<float>(m->nRe, ncol2, kc, Pk32 + (size_t)k0 * m->nRe, m->nRe, true, true, w.G1bar, ncol2, gwbar,
                        ncol2, true, st);
  }
  return cudaGetLastError() == cudaSuccess ? EPW_OK : EPW_ERR_CUDA;
}

// =============================================================== staged form
// Shapes whose per-k columns 2 nw^2 (3nat + 1) exceed one 128-column slot of the
// fused kernel (e.g. nw = 5 or 8 with 6 to 9 modes) run the same real GEMM on
// the tensor cores per chunk of k with its result written to HBM,
//   Ct[kl cpk + col][q] = sum_kk A[q][kk] B[kl][col][kk],
// and the per-pair kernel (eigensolve, rotation, deltas) reads it from there.
bool tc_staged_supported(const epw_model *m) { return !tc_supported(m) && m->nw <= 18 && m->nm <= 18; }

epw_status tc_staged_plan(Arena &A, const epw_model *m, int nk, int nq, int op, size_t ct_budget, TcStaged &s,
                          bool any_shape) {
  s = TcStaged{};
  s.op = op;
  s.ok = any_shape ? (m->nw <= 18 && m->nm <= 18) : tc_staged_supported(m);
  if (!s.ok) return EPW_OK;
  const int esz = op == TC_OP_BF16 ? 2 : 4;
  const int kal = op == TC_OP_BF16 ? 16 : 8;  // K per MMA
  s.kpad = k_layout(m, kal, s.kg0);
  s.cpk = 2 * m->nw * m->nw * (m->nm + 1);
  s.mtiles = (std::max(nq, 1) + 127) / 128;
  s.ldc = s.mtiles * 128;
  const size_t per_k = (size_t)s.cpk * s.ldc * 4;
  s.kc = (int)std::min<size_t>((size_t)std::max(nk, 1), std::max<size_t>(1, ct_budget / per_k));
  const int ntiles = (s.kc * s.cpk + G_NT - 1) / G_NT;
  // shapes beyond the register-tile per-pair kernel read Ct q-major (a pair's
  // columns contiguous) in the warp-per-pair kernel
  s.qmajor = m->nw > 8 || m->nm > 9;
  s.ldn = (size_t)ntiles * G_NT;
  s.Ahi = A.take<char>((size_t)std::max(nq, 1) * s.kpad * esz);
  s.Alo = A.take<char>((size_t)std::max(nq, 1) * s.kpad * esz);
  s.Bhi = A.take<char>((size_t)s.kc * s.cpk * s.kpad * esz);
  s.Blo = A.take<char>((size_t)s.kc * s.cpk * s.kpad * esz);
  s.Ct = A.take<float>((size_t)ntiles * G_NT * s.ldc);
  return EPW_OK;
}

epw_status tc_staged_phases(const epw_model *m, int nq, const double *q, TcStaged &s, cudaStream_t st) {
  if (!s.ok) return EPW_ERR_UNSUPPORTED;
  if (s.op == TC_OP_BF16)
    build_a<__nv_bfloat16>(nq, m->nRe, s.kpad, q, m->Re, s.Pq64, (__nv_bfloat16 *)s.Ahi, (__nv_bfloat16 *)s.Alo, st,
                           m->nRp, m->Rp, s.kg0);
  else
    build_a<float>(nq, m->nRe, s.kpad, q, m->Re, s.Pq64, (float *)s.Ahi, (float *)s.Alo, st, m->nRp, m->Rp, s.kg0);
  return cudaGetLastError() == cudaSuccess ? EPW_OK : EPW_ERR_CUDA;
}

epw_status tc_staged_contract(const epw_model *m, int k0, int kc, int nq, const cx<float> *Bg32,
                              const cx<float> *BH32, TcStaged &s, cudaStream_t st) {
  if (!s.ok || kc > s.kc) return EPW_ERR_UNSUPPORTED;
  const int nR = m->nRe, nw2 = m->nw * m->nw;
  const cx<float> *bh = BH32 + (size_t)k0 * nR * nw2, *bg = Bg32 + (size_t)k0 * m->nRp * m->nm * nw2;
  if (s.op == TC_OP_BF16)
    launch_build_b<__nv_bfloat16>(kc, kc, nR, m->nw, m->nm, s.cpk, s.kpad, 0, bh, bg, (__nv_bfloat16 *)s.Bhi,
                                  (__nv_bfloat16 *)s.Blo, st, m->nRp, s.kg0);
  else
    launch_build_b<float>(kc, kc, nR, m->nw, m->nm, s.cpk, s.kpad, 0, bh, bg, (float *)s.Bhi, (float *)s.Blo, st,
                          m->nRp, s.kg0);
  const int rows = kc * s.cpk;
  CUtensorMap ah, al, bh_m, bl_m;
  if (!make_map(&ah, s.Ahi, s.op, s.kpad, nq, 128) || !make_map(&al, s.Alo, s.op, s.kpad, nq, 128) ||
      !make_map(&bh_m, s.Bhi, s.op, s.kpad, rows, G_NT) || !make_map(&bl_m, s.Blo, s.op, s.kpad, rows, G_NT))
    return EPW_ERR_CUDA;
  GemmArgs g;
  g.mtiles = (nq + 127) / 128;
  g.ntiles = (rows + G_NT - 1) / G_NT;
  g.kblocks = (s.kpad * (s.op == TC_OP_BF16 ? 2 : 4) + ROWB - 1) / ROWB;
  g.kb_per_split = g.kblocks;
  g.splits = 1;
  g.ldc = s.ldc;
  g.npad = g.ntiles * G_NT;
  g.Ct = s.Ct;
  g.qmajor = s.qmajor ? 1 : 0;
  g.ldn = s.ldn;
  g.dstatus = m->dstatus;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int items = g.mtiles * g.ntiles;
  if (s.op == TC_OP_BF16) {
    static bool attr = false;
    if (!attr) {
      if (cudaFuncSetAttribute(k_tc_gemm_nt<TC_OP_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM) !=
          cudaSuccess)
        return EPW_ERR_CUDA;
      attr = true;
    }
    k_tc_gemm_nt<TC_OP_BF16><<<std::min(items, sms), G_THREADS, G_SMEM, st>>>(ah, al, bh_m, bl_m, g);
  } else {
    static bool attr = false;
    if (!attr) {
      if (cudaFuncSetAttribute(k_tc_gemm_nt<TC_OP_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM) !=
          cudaSuccess)
        return EPW_ERR_CUDA;
      attr = true;
    }
    k_tc_gemm_nt<TC_OP_TF32><<<std::min(items, sms), G_THREADS, G_SMEM, st>>>(ah, al, bh_m, bl_m, g);
  }
  epw_count_launch();
  return cudaGetLastError() == cudaSuccess ? EPW_OK : EPW_ERR_CUDA;
}

epw_status tc_wait_selftest(long long cycles, unsigned *dstatus, int *waited_out, cudaStream_t st) {
  if (cycles < 1 || cycles > 4000000000LL) return EPW_ERR_INVALID_ARG;
  k_wait_selftest<<<1, 32, 0, st>>>(cycles, dstatus, waited_out);
  epw_count_launch();
  return cudaGetLastError() == cudaSuccess ? EPW_OK : EPW_ERR_CUDA;
}
