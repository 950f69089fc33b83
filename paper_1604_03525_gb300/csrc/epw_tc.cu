// Fused linewidth kernel on the 5th-generation tensor cores (sm_103a).
//
// Per (k,q) pair the interpolation contraction (EPW, Sec. "Electron-phonon
// coupling in polar materials", step iii, with the U rotations of the overlap
// equation there) is a complex GEMM over the real-space index R:
//
//   C[q][c] = sum_R P_q(R) B_k[R][c],   c = (H(k+q)_ij | (g_a(k,q) U_k)_jn)
//
// with P_q(R) = e^{2 pi i q.R}.  It runs as a real GEMM with K = 2 nR (re/im
// interleaved) on tcgen05: operands are split into two bfloat16 terms
// (x = hi + lo) and three MMAs (hi*hi + hi*lo + lo*hi) accumulate in FP32 in
// tensor memory.  The epilogue of each 128 x 256 tile (128 q rows x 2 k) is the
// per-pair work of Eq. (linewidthel): a Jacobi eigensolve of H(k+q), the mode
// projection with e_q/sqrt(2 M w), the U_k+q^dagger rotation, |g|^2, Gaussian
// deltas and occupations, reduced over the tile's q rows.
//
// CTA layout (persistent, one CTA per SM, 10 warps):
//   warp 0      TMA producer (A = q-phase tile, B = k-vertex tile, 2 stages)
//   warp 1      TMEM allocator and MMA issuer (one elected thread)
//   warps 2..9  epilogue: warp w reads TMEM lanes 32*(w%4).., k-slot (w-2)/4
// Tensor memory holds two accumulator stages of 256 columns (512 in total),
// so the MMA of the next tile overlaps the epilogue of the current one.
// Every wait is bounded; a wait that runs out raises EPW_DEV_TIMEOUT, drains
// outstanding copies and MMAs, frees tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>

#include "epw_tc.cuh"

namespace {

constexpr int BM = 128;                      // q rows per tile
constexpr int BN = 256;                      // real accumulator columns per tile
constexpr int BK = 64;                       // K elements per stage (128 B of bf16)
constexpr int STAGES = 2;
constexpr int A_BYTES = BM * BK * 2;         // 16 KiB
constexpr int B_BYTES = BN * BK * 2;         // 32 KiB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr int NTHREADS = 320;
constexpr int EPI_WARP0 = 2;
constexpr int NEPI_WARPS = 8;
constexpr uint32_t TMEM_COLS = 512;
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

// kind::f16 instruction descriptor: D=F32, A=B=BF16, K-major A and B, N=256, M=128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 bit, 8 consecutive columns per thread; waits for completion.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *r) {
  uint32_t u0, u1, u2, u3, u4, u5, u6, u7;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(u0), "=r"(u1), "=r"(u2), "=r"(u3), "=r"(u4), "=r"(u5), "=r"(u6), "=r"(u7)
      : "r"(taddr)
      : "memory");
  r[0] = __uint_as_float(u0);
  r[1] = __uint_as_float(u1);
  r[2] = __uint_as_float(u2);
  r[3] = __uint_as_float(u3);
  r[4] = __uint_as_float(u4);
  r[5] = __uint_as_float(u5);
  r[6] = __uint_as_float(u6);
  r[7] = __uint_as_float(u7);
}
// 32 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *r) {
  uint32_t u[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]),
        "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]),
        "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) r[i] = __uint_as_float(u[i]);
}
// n (multiple of 8) consecutive columns
template <int NCOL>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float *r) {
  static_assert(NCOL % 8 == 0, "columns come in groups of 8");
  int c = 0;
#pragma unroll
  for (; c + 32 <= NCOL; c += 32) tmem_ld32(taddr + c, r + c);
#pragma unroll
  for (; c < NCOL; c += 8) tmem_ld8(taddr + c, r + c);
}

// K-major, 128-byte-swizzled smem operand: rows of 128 B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Bounded wait on an mbarrier phase.  Returns false on abort or timeout.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int *abort_flag, unsigned *dstatus) {
  if (mbar_try(bar, parity)) return true;
  long long t0 = clock64();
  uint32_t it = 0;
  while (!mbar_try(bar, parity)) {
    if ((++it & 127u) == 0) {
      if (*abort_flag) return false;
      if (clock64() - t0 > WAIT_CYCLES) {
        *abort_flag = 1;
        atomicOr(dstatus, EPW_DEV_TIMEOUT);
        return false;
      }
    }
  }
  return true;
}
// Bounded wait that ignores the abort flag (used to drain in-flight work).
__device__ __forceinline__ void drain_bar(uint32_t bar, uint32_t parity) {
  long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > WAIT_CYCLES) break;
}

struct TcArgs {
  int nk, nq, nqt, nkg, kpad, nkb;
  const double *epsk;    // [nk][nw]
  const double *omegaT;  // [nm][nq]
  const float *nbT;      // [nm][nq]
  const float2 *ET;      // [nm*nm][nq]
  const double *wq;      // [nq] or null
  float EF, invkT, inv_sigma, gnorm, omega_min;
  double *partial;  // [nk][4*nqt][nw]
  unsigned *dstatus;
};

template <int NW, int NM>
struct Shape {
  static constexpr int NC = NW * NW * (NM + 1);  // complex columns per k
  static constexpr int CPK_RAW = 2 * NC;
  static constexpr int CPK = CPK_RAW <= 8 ? 8 : CPK_RAW <= 16 ? 16 : CPK_RAW <= 32 ? 32 : CPK_RAW <= 64 ? 64 : 128;
  static constexpr int KPS = 128 / CPK;  // k per slot (per epilogue warp)
  static constexpr int KPT = 2 * KPS;    // k per tile
  static_assert(CPK_RAW <= 128, "one k must fit in a 128-column slot");
};

// ------------------------------------------------------------------ epilogue
template <int NW, int NM>
__device__ __forceinline__ void epilogue_pair(const TcArgs &a, uint32_t tcol, int q, int k, bool valid, int quad,
                                              int qt) {
  using S = Shape<NW, NM>;
  constexpr int H2 = 2 * NW * NW;  // real columns of one NW x NW complex block
  constexpr int UR = NW <= 4 ? NW : 1;
  const int qq = q < a.nq ? q : 0;
  const int kk = k < a.nk ? k : 0;
  // H(k+q) (and, for small shapes, every column of this k) from the accumulator
  constexpr bool ONE_LOAD = S::CPK <= 32;
  float all[ONE_LOAD ? S::CPK : 1];
  float hbuf[ONE_LOAD ? 1 : H2];
  const float *h;
  if constexpr (ONE_LOAD) {
    tmem_load<S::CPK>(tcol, all);
    h = all;
  } else {
    tmem_load<H2>(tcol, hbuf);
    h = hbuf;
  }
  cx<float> A[NW][NW], V[NW][NW];
#pragma unroll
  for (int i = 0; i < NW; i++)
#pragma unroll
    for (int j = 0; j < NW; j++) A[i][j] = mkc(h[2 * (i * NW + j)], h[2 * (i * NW + j) + 1]);
  bool nc = false;
  jacobi_herm<float, NW>(A, V, NW, jacobi_tol<float>::tol2, jacobi_tol<float>::maxsweep, nc);
  if (nc && valid) atomicOr(a.dstatus, EPW_DEV_NOT_CONVERGED);
  float em[NW], cpf[NW];
#pragma unroll UR
  for (int m = 0; m < NW; m++) {
    em[m] = A[m][m].x;
    cpf[m] = fermi_f(em[m] - a.EF, a.invkT);
  }
  float ek[NW];
#pragma unroll UR
  for (int n = 0; n < NW; n++) ek[n] = (float)a.epsk[(size_t)kk * NW + n];
  float acc[NW];
#pragma unroll UR
  for (int n = 0; n < NW; n++) acc[n] = 0.0f;
  const float LOG2E = 1.4426950408889634f;
  const float s2 = a.inv_sigma * a.inv_sigma * LOG2E;
#pragma unroll 1
  for (int nu = 0; nu < NM; nu++) {
    const float w = (float)a.omegaT[(size_t)nu * a.nq + qq];
    const bool keep = (w >= a.omega_min) && (w > 0.0f);
    const float nb = a.nbT[(size_t)nu * a.nq + qq];
    cx<float> G[NW][NW];
#pragma unroll
    for (int i = 0; i < NW; i++)
#pragma unroll
      for (int j = 0; j < NW; j++) G[i][j] = mkc(0.0f, 0.0f);
#pragma unroll 1
    for (int al = 0; al < NM; al++) {
      float xbuf[ONE_LOAD ? 1 : H2];
      const float *x;
      if constexpr (ONE_LOAD) {
        x = all + H2 * (1 + al);
      } else {
        tmem_load<H2>(tcol + H2 * (1 + al), xbuf);
        x = xbuf;
      }
      float2 e2 = a.ET[((size_t)al * NM + nu) * a.nq + qq];
      cx<float> e = mkc(e2.x, e2.y);
#pragma unroll
      for (int i = 0; i < NW; i++)
#pragma unroll
        for (int j = 0; j < NW; j++) cfma(G[i][j], e, mkc(x[2 * (i * NW + j)], x[2 * (i * NW + j) + 1]));
    }
    // |(U^dagger G)_mn|^2 with the delta terms of Eq. (linewidthel)
#pragma unroll UR
    for (int m = 0; m < NW; m++) {
      const float f = cpf[m];
      const float cp = keep ? nb + f : 0.0f, cm = keep ? nb + 1.0f - f : 0.0f;
#pragma unroll UR
      for (int n = 0; n < NW; n++) {
        cx<float> y = mkc(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < NW; i++) cfma(y, conjc(V[i][m]), G[i][n]);
        const float g2 = cabs2(y);
        const float xd = ek[n] - em[m];
        const float xp = xd + w, xm = xd - w;
        const float d = cp * ex2_approx(-xp * xp * s2) + cm * ex2_approx(-xm * xm * s2);
        acc[n] = fmaf(g2, d, acc[n]);
      }
    }
  }
  const double wqi = valid ? (a.wq ? a.wq[q] : 1.0 / a.nq) * (double)a.gnorm : 0.0;
#pragma unroll UR
  for (int n = 0; n < NW; n++) {
    double v = (double)acc[n] * wqi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && k < a.nk)
      a.partial[((size_t)k * (4 * a.nqt) + qt * 4 + quad) * NW + n] = v;
  }
}

template <int NW, int NM>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_linewidth(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                   const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, TcArgs a) {
  using S = Shape<NW, NM>;
  __shared__ __align__(8) uint64_t bar_full[STAGES], bar_empty[STAGES], bar_tfull[2], bar_tempty[2], bar_final;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t smem0 = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int *abort_flag = &abort_sh;
  const int nitems = a.nkg * a.nqt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int s = 0; s < 2; s++) {
      mbar_init(smem_u32(&bar_tfull[s]), 1);
      mbar_init(smem_u32(&bar_tempty[s]), NEPI_WARPS);
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
    // The whole warp walks the schedule; lane 0 waits and issues the copies.
    int issued[STAGES] = {0, 0};
    uint32_t it = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const int kg = item / a.nqt, qt = item % a.nqt;
      for (int kb = 0; kb < a.nkb; kb++, it++) {
        const int s = it % STAGES;
        const uint32_t par = ((it / STAGES) & 1u) ^ 1u;
        if (lane == 0) {
          ok = wait_bar(smem_u32(&bar_empty[s]), par, abort_flag, a.dstatus);
          if (ok) {
            const uint32_t base = smem0 + s * STAGE_BYTES;
            const uint32_t fb = smem_u32(&bar_full[s]);
            mbar_expect_tx(fb, STAGE_BYTES);
            tma_load_2d(base, &mAhi, kb * BK, qt * BM, fb);
            tma_load_2d(base + A_BYTES, &mAlo, kb * BK, qt * BM, fb);
            tma_load_2d(base + 2 * A_BYTES, &mBhi, kb * BK, kg * (S::KPT * S::CPK), fb);
            tma_load_2d(base + 2 * A_BYTES + B_BYTES, &mBlo, kb * BK, kg * (S::KPT * S::CPK), fb);
            issued[s] = (int)(it / STAGES) + 1;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
      }
    }
    // drain: every issued copy must land before the CTA exits
    if (lane == 0)
      for (int s = 0; s < STAGES; s++)
        if (issued[s] > 0) drain_bar(smem_u32(&bar_full[s]), (uint32_t)((issued[s] - 1) & 1));
    __syncwarp();
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    // The whole warp walks the schedule; lane 0 waits and issues the MMAs.
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
      const uint32_t dcol = tmem + ts * BN;
      for (int kb = 0; kb < a.nkb; kb++, it++) {
        const int s = it % STAGES;
        const uint32_t par = (it / STAGES) & 1u;
        if (lane == 0) {
          ok = wait_bar(smem_u32(&bar_full[s]), par, abort_flag, a.dstatus);
          if (ok) {
            tc_fence_after();
            const uint32_t base = smem0 + s * STAGE_BYTES;
            const uint64_t dAh = sdesc_sw128(base), dAl = sdesc_sw128(base + A_BYTES);
            const uint64_t dBh = sdesc_sw128(base + 2 * A_BYTES), dBl = sdesc_sw128(base + 2 * A_BYTES + B_BYTES);
            const int ksteps = min(BK, a.kpad - kb * BK) / 16;
            for (int ks = 0; ks < ksteps; ks++) {
              const uint64_t off = (uint64_t)((ks * 32) >> 4);
              const uint32_t acc = (kb == 0 && ks == 0) ? 0u : 1u;
              umma_bf16(dcol, dAl + off, dBh + off, acc);
              umma_bf16(dcol, dAh + off, dBl + off, 1u);
              umma_bf16(dcol, dAh + off, dBh + off, 1u);
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
    // drain: all issued MMAs complete before tensor memory is released
    if (lane == 0) {
      umma_commit(smem_u32(&bar_final));
      drain_bar(smem_u32(&bar_final), 0);
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------------- epilogue
    const int quad = warp & 3;
    const int slot = (warp - EPI_WARP0) >> 2;
    int titer = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, titer++) {
      const int ts = titer & 1;
      const uint32_t tpar = (titer >> 1) & 1;
      const bool ok = wait_bar(smem_u32(&bar_tfull[ts]), tpar, abort_flag, a.dstatus);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const int kg = item / a.nqt, qt = item % a.nqt;
      const int q = qt * BM + quad * 32 + lane;
      const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + ts * BN + slot * 128;
#pragma unroll 1
      for (int j = 0; j < S::KPS; j++) {
        const int k = kg * S::KPT + slot * S::KPS + j;
        epilogue_pair<NW, NM>(a, tbase + j * S::CPK, q, k, q < a.nq && k < a.nk, quad, qt);
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

// ------------------------------------------------------- operand builders
// A[q][kk] (K-major bf16 hi/lo): kk = 2r + t, value cos / sin of 2 pi (q.R_r mod 1).
__global__ void k_build_a(int nq, int nR, int kpad, const double *__restrict__ q, const int *__restrict__ R,
                          __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
  size_t n = (size_t)nq * kpad;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    int kk = (int)(idx % kpad);
    int iq = (int)(idx / kpad);
    float v = 0.0f;
    if (kk < 2 * nR) {
      int r = kk >> 1;
      double x = q[3 * iq] * R[3 * r] + q[3 * iq + 1] * R[3 * r + 1] + q[3 * iq + 2] * R[3 * r + 2];
      x -= rint(x);
      double s, c;
      sincospi(2.0 * x, &s, &c);
      double d = (kk & 1) ? s : c;
      __nv_bfloat16 h = __double2bfloat16(d);
      hi[idx] = h;
      lo[idx] = __double2bfloat16(d - (double)__bfloat162float(h));
      continue;
    }
    hi[idx] = __float2bfloat16(v);
    lo[idx] = __float2bfloat16(v);
  }
}

// B[k][col][kk] (K-major bf16 hi/lo) of the real GEMM:
//   col = 2c + s (s: re/im of output column c), kk = 2r + t (t: re/im of P_q(R_r)),
//   (s,t) = (0,0): Re b, (0,1): -Im b, (1,0): Im b, (1,1): Re b,  b = B_k[r][c].
// Output columns c: [0, nw^2) H(k+q)_ij, then (a, j, n) of g_a(k,q) U_k.
__global__ void k_build_b(int nk, int nk_pad, int nR, int nw, int nm, int cpk, int kpad,
                          const cx<float> *__restrict__ BH, const cx<float> *__restrict__ Bg, __nv_bfloat16 *hi,
                          __nv_bfloat16 *lo) {
  const int nw2 = nw * nw;
  const int nc = nw2 * (nm + 1);
  size_t n = (size_t)nk_pad * cpk * kpad;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    int kk = (int)(idx % kpad);
    size_t rest = idx / kpad;
    int col = (int)(rest % cpk);
    int k = (int)(rest / cpk);
    float v = 0.0f;
    if (k < nk && col < 2 * nc && kk < 2 * nR) {
      int c = col >> 1, s = col & 1, r = kk >> 1, t = kk & 1;
      cx<float> b = c < nw2 ? BH[((size_t)k * nR + r) * nw2 + c] : Bg[((size_t)k * nR + r) * nm * nw2 + (c - nw2)];
      v = s == 0 ? (t == 0 ? b.x : -b.y) : (t == 0 ? b.y : b.x);
    }
    __nv_bfloat16 h = __float2bfloat16(v);
    hi[idx] = h;
    lo[idx] = __float2bfloat16(v - __bfloat162float(h));
  }
}

__global__ void k_bose_table(int nq, int nm, const double *__restrict__ omegaT, double T, float *nbT) {
  size_t n = (size_t)nq * nm;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double w = omegaT[i];
    nbT[i] = (w > 0.0) ? (float)bose_d(w, T) : 0.0f;
  }
}

inline int grid_for(size_t n, int bs) {
  size_t b = (n + bs - 1) / bs;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
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

// 2D bf16 tensor [rows][inner] (inner contiguous), box [box_rows][64], 128-byte swizzle.
bool make_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool shape_info(int nw, int nm, int &cpk, int &kpt) {
#define EPW_TC_SHAPE(W, M)            \
  if (nw == W && nm == M) {           \
    cpk = Shape<W, M>::CPK;           \
    kpt = Shape<W, M>::KPT;           \
    return true;                      \
  }
  EPW_TC_SHAPE(4, 3)
  EPW_TC_SHAPE(1, 3)
  EPW_TC_SHAPE(2, 3)
#undef EPW_TC_SHAPE
  return false;
}

template <int NW, int NM>
cudaError_t launch_tc(const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &bh, const CUtensorMap &bl,
                      const TcArgs &a, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_tc_linewidth<NW, NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int items = a.nkg * a.nqt;
  int grid = items < sms ? items : sms;
  k_tc_linewidth<NW, NM><<<grid, NTHREADS, SMEM_BYTES, st>>>(ah, al, bh, bl, a);
  return cudaGetLastError();
}

}  // namespace

epw_status tc_plan(Arena &A, const epw_model *m, int nk, int nq, TcBuffers &b) {
  b = TcBuffers{};
  b.ok = m->same_ep && shape_info(m->nw, m->nm, b.cpk, b.kpt);
  if (!b.ok) return EPW_OK;
  b.kpad = (2 * m->nRe + 15) / 16 * 16;
  b.nk_pad = (nk + b.kpt - 1) / b.kpt * b.kpt;
  b.nqt = (nq + BM - 1) / BM;
  b.Ahi = A.take<__nv_bfloat16>((size_t)nq * b.kpad);
  b.Alo = A.take<__nv_bfloat16>((size_t)nq * b.kpad);
  b.Bhi = A.take<__nv_bfloat16>((size_t)b.nk_pad * b.cpk * b.kpad);
  b.Blo = A.take<__nv_bfloat16>((size_t)b.nk_pad * b.cpk * b.kpad);
  b.nbT = A.take<float>((size_t)nq * m->nm);
  b.partial = A.take<double>((size_t)nk * 4 * b.nqt * m->nw);
  return EPW_OK;
}

epw_status tc_linewidth(const epw_model *m, int nk, const double *k, int nq, const double *q, const double *wq,
                        const epw_params *par, const cx<double> *PkRM, const double *epsk, const cx<double> *Uk,
                        const double *omegaT, const cx<float> *ET32, const cx<float> *Bg32, const cx<float> *BH32,
                        TcBuffers &b, double *out, cudaStream_t st) {
  (void)k;
  (void)PkRM;
  (void)Uk;
  if (!b.ok) return EPW_ERR_UNSUPPORTED;
  const int nR = m->nRe;
  {
    size_t n = (size_t)nq * b.kpad;
    k_build_a<<<grid_for(n, 256), 256, 0, st>>>(nq, nR, b.kpad, q, m->Re, (__nv_bfloat16 *)b.Ahi,
                                                 (__nv_bfloat16 *)b.Alo);
    epw_count_launch();
    n = (size_t)b.nk_pad * b.cpk * b.kpad;
    k_build_b<<<grid_for(n, 256), 256, 0, st>>>(nk, b.nk_pad, nR, m->nw, m->nm, b.cpk, b.kpad, BH32, Bg32,
                                                 (__nv_bfloat16 *)b.Bhi, (__nv_bfloat16 *)b.Blo);
    epw_count_launch();
    n = (size_t)nq * m->nm;
    k_bose_table<<<grid_for(n, 256), 256, 0, st>>>(nq, m->nm, omegaT, par->T_K, b.nbT);
    epw_count_launch();
  }
  CUtensorMap ah, al, bh, bl;
  std::memset(&ah, 0, sizeof(ah));
  if (!make_map(&ah, b.Ahi, b.kpad, nq, BM) || !make_map(&al, b.Alo, b.kpad, nq, BM) ||
      !make_map(&bh, b.Bhi, b.kpad, (uint64_t)b.nk_pad * b.cpk, BN) ||
      !make_map(&bl, b.Blo, b.kpad, (uint64_t)b.nk_pad * b.cpk, BN))
    return EPW_ERR_CUDA;
  TcArgs a;
  a.nk = nk;
  a.nq = nq;
  a.nqt = b.nqt;
  a.nkg = b.nk_pad / b.kpt;
  a.kpad = b.kpad;
  a.nkb = (b.kpad + BK - 1) / BK;
  a.epsk = epsk;
  a.omegaT = omegaT;
  a.nbT = b.nbT;
  a.ET = (const float2 *)ET32;
  a.wq = wq;
  a.EF = (float)par->EF_eV;
  a.invkT = par->T_K > 0.0 ? (float)(1.0 / (EPW_KB * par->T_K)) : 0.0f;
  a.inv_sigma = (float)(1.0 / par->sigma_eV);
  a.gnorm = (float)(1.0 / (par->sigma_eV * 1.7724538509055160273));
  a.omega_min = (float)par->omega_min_eV;
  a.partial = b.partial;
  a.dstatus = m->dstatus;
  cudaError_t e = cudaSuccess;
  epw_timing_begin(const_cast<epw_model *>(m), st);
  if (m->nw == 4 && m->nm == 3)
    e = launch_tc<4, 3>(ah, al, bh, bl, a, st);
  else if (m->nw == 1 && m->nm == 3)
    e = launch_tc<1, 3>(ah, al, bh, bl, a, st);
  else if (m->nw == 2 && m->nm == 3)
    e = launch_tc<2, 3>(ah, al, bh, bl, a, st);
  else
    return EPW_ERR_UNSUPPORTED;
  epw_timing_end(const_cast<epw_model *>(m), st);
  epw_count_launch();
  if (e != cudaSuccess) return EPW_ERR_CUDA;
  launch_finalize(nk, 4 * b.nqt, m->nw, b.partial, out, st);
  return EPW_OK;
}

void tc_free(epw_model *) {}
