// Tensor-core (tcgen05) form of the fused linewidth kernel.
#pragma once
#include <cuda.h>

#include "epw_internal.cuh"

// Operand split of the tensor-core contraction.
#define TC_OP_BF16 0  // two bfloat16 terms, kind::f16
#define TC_OP_TF32 1  // two tf32 terms, kind::tf32

struct TcBuffers {
  void *Ahi, *Alo;   // q phases, split, K-major [nq][kpad]
  void *Bhi, *Blo;   // k-side vertex, split, K-major [nk_pad][cpk][kpad]
  float *nbT;        // Bose factors [nm][nq]
  float *omF;        // frequencies [nm][nq]
  float *wqF;        // q weights [nq]
  float *ekF;        // band energies at k [nk][nw]
  double *partial;   // [nk][4*nqt][nw]
  int op, kpad, cpk, nk_pad, nqt, kpt;
  int kg0;           // K offset of the vertex's Rp phases when Rp differs from Re (0: one shared set)
  int planar;        // B columns in re/im pairs (see k_build_b)
  bool ok;           // shape has a tensor-core kernel
  bool prebuilt_a, prebuilt_b;  // A / B already built for the next tc_linewidth/tc_interp call
  size_t a_block_bytes;  // q-block of the A operand visited by all k groups (0: default)
  // long-range vertex (polar models): set by the caller before a call; UkF is laid out by tc_plan
  const float2 *Cpol;        // [nm][nq]
  const cx<double> *Uk64;    // [nk][nw][nw]
  float2 *UkF;               // FP32 copy of Uk64
  const cx<double> *Pq64;    // FP64 q phases of the Re set [nR][nq] when already formed (else null)
};

// True when the model's shape has a tensor-core kernel (a compiled (nw, 3nat)
// pair).  When Rp differs from Re the contraction runs over K = [Re phases | Rp
// phases]: H(k+q) columns are zero on the Rp part, vertex columns on the Re part.
bool tc_supported(const epw_model *m);
// Lay out (or measure, with a null arena base) the buffers of the tensor-core path.
epw_status tc_plan(Arena &A, const epw_model *m, int nk, int nq, int op, TcBuffers &b);
// Builds of the fused kernel's operands on stream st: B from the k-side vertex,
// A from the q phases (b.Pq64 when set, else from q).
void tc_build_b(const epw_model *m, int nk, const cx<float> *Bg32, const cx<float> *BH32, TcBuffers &b,
                cudaStream_t st);
void tc_build_a(const epw_model *m, int nq, const double *q, TcBuffers &b, cudaStream_t st);
// The q side of the fused form in one kernel (double-float phases and D(q), A
// operand written directly); false (nothing launched) when the model has no such
// form (R sets differ, 3nat != 3 or |R_j| beyond the factor table).
bool tc_qside(const epw_model *m, int nq, const double *q, TcBuffers &b, cx<double> *D, cudaStream_t st);
// Im Sigma [nk][nw] into `out` (device) from the shared preparation outputs.
epw_status tc_linewidth(const epw_model *m, int nk, const double *k, int nq, const double *q, const double *wq,
                        const epw_params *par, const cx<double> *PkRM, const double *epsk, const cx<double> *Uk,
                        const double *omegaT, const cx<float> *ET32, const cx<float> *Bg32, const cx<float> *BH32,
                        TcBuffers &b, double *out, cudaStream_t st);
// e_k+q [nk][nq][nw] (ascending) and g [nk][nq][nm][nw][nw] (device, either may be
// null) from the same contraction and eigensolve as tc_linewidth.
epw_status tc_interp(const epw_model *m, int nk, int nq, const double *q, double omega_min, const double *epsk,
                     const double *omegaT, const cx<float> *ET32, const cx<float> *Bg32, const cx<float> *BH32,
                     TcBuffers &b, double *eps_kq, double *g, cudaStream_t st);
void tc_free(epw_model *m);

// Raw operand builders and maps shared with the wide-shape kernels (epw_tcw.cu):
// B rows [nk_pad][cpk][kpad] from BH [nk][nR][nw][nw] and Bg [nk][nR][nm][nw][nw]
// (nm = 0: the H(k+q) block only); A [nq][kpad] from P64 [nR][nq] or from q.
void tc_build_b_raw(int op, int nk, int nk_pad, int nR, int nw, int nm, int cpk, int kpad, const cx<float> *BH,
                    const cx<float> *Bg, void *hi, void *lo, cudaStream_t st);
void tc_build_a_raw(int op, int nq, int nR, int kpad, const double *q, const int *R, const cx<double> *P64, void *hi,
                    void *lo, cudaStream_t st);
// 2D K-major map [rows][inner], box [box_rows][128 bytes], 128-byte swizzle.
bool tc_make_map(CUtensorMap *map, const void *base, int op, uint64_t inner, uint64_t rows, uint32_t box_rows);
// The same with rows of row_bytes (128: 128-byte swizzle; 64: 64-byte swizzle).
bool tc_make_map_rb(CUtensorMap *map, const void *base, int op, uint64_t inner, uint64_t rows, uint32_t box_rows,
                    int row_bytes);
// FP32 tables: Bose factors and frequencies [nm][nq], q weights [nq], band energies [nk][nw].
void tc_tables(int nq, int nm, int nk, int nw, const double *omegaT, double T, const double *wq, const double *epsk,
               float *nbT, float *omF, float *wqF, float *ekF, cudaStream_t st);

// Wide-shape form (epw_tcw.cu) for shapes whose per-k columns exceed the fused
// kernel's slot: H(k+q) is contracted on the tensor cores and diagonalised per
// pair (eigenvalues and the eigenvectors some band at k can reach within the
// Gaussian cutoff are kept), then (g_a(k,q) U_k) is contracted and only the
// (m, n) terms whose Gaussians do not underflow are evaluated: by default in one
// kernel (the eigensolve beside the vertex MMAs, eigen-data through an L2 ring),
// or as two kernels per chunk of k (E, then G; eigen-data through HBM).
struct TcwBuffers {
  void *Ahi, *Alo;     // q phases of the Re set [nq][kpad]
  void *AGhi, *AGlo;   // q phases of the Rp set [nq][kpadG] (the Re buffers when the sets agree)
  void *BEhi, *BElo;   // H(k+q) operand of one chunk [kc_pad][cpk][kpad]
  void *BGhi, *BGlo;   // vertex operand of one chunk [nchunk][bng][kpad]
  float *epsq;         // [kc][nw][ldq] eigenvalues of H(k+q)
  float2 *Uq;          // [kc][nw(m)][nw(i)][ldq] eigenvector m (reachable m only)
  float *nbT, *omF, *wqF, *ekF, *thr;
  double *partial;     // [nk][4 nqt][nw]
  float2 *UkF;         // polar models: FP32 U_k [nk][nw][nw]
  int op, kpad, kpadG, kc, ldq, nqt, cpk, kpt, entp, cn, bng;
  bool ok;
  bool fused;          // one kernel (E and G overlapped, eigen-data through a ring in L2); else two per chunk
  bool pair;           // the fused kernel on CTA pairs (cta_group::2 MMAs over 256 q rows)
};
// forms of the wide path: the fused kernel on CTA pairs (default), the two-kernel form, the
// fused kernel on single CTAs
enum { TCW_FORM_PAIR = 0, TCW_FORM_SPLIT = 1, TCW_FORM_SINGLE = 2 };
bool tcw_supported(const epw_model *m);
// bytes: budget of the per-chunk buffers (0: default); form: TCW_FORM_*
epw_status tcw_plan(Arena &A, const epw_model *m, int nk, int nq, int op, size_t bytes, TcwBuffers &b,
                    int form = TCW_FORM_PAIR);
// Im Sigma [nk][nw] into `out` (device) from the preparation outputs (P64: FP64 q phases of
// the Re set [nR][nq] or null; Cpol [nm][nq] and Uk for polar models, else null).
epw_status tcw_linewidth(const epw_model *m, int nk, int nq, const double *q, const double *wq,
                         const epw_params *par, const double *epsk, const double *omegaT, const cx<float> *ET32,
                         const cx<float> *Bg32, const cx<float> *BH32, const cx<double> *P64,
                         const cx<double> *Uk, const float2 *Cpol, TcwBuffers &b, double *out, cudaStream_t st);

// Buffers of the tensor-core adjoint (per chunk of kc k-points).
struct TcBwdBuffers {
  float *phi, *plo;        // conj-phase operand [2nR][ld]
  float *xhi, *xlo;        // Xbar rows [kc*nc][ld]
  float *Ct;               // split-K partials [splits][npad][ldc]
  cx<float> *Bbar, *G1bar; // [nRp][kc][nc], [kc][nRp][nc]
  float *cotF;             // [nk][nw]
  double *partT, *partE;   // [kc][4*nqt]
  int nc, ld, kc, mtiles, ntiles, kblocks, kb_per_split, splits, ldc, npad;
};

#define CKS_TC(expr)              \
  do {                            \
    epw_status s_ = (expr);       \
    if (s_ != EPW_OK) return s_;  \
  } while (0)

// Lay out the adjoint's buffers (forward operands at TF32 included).
epw_status tc_bwd_plan(Arena &A, const epw_model *m, int nk, int nq, TcBuffers &b, TcBwdBuffers &w);
// Staged adjoint's q contraction on the tensor cores (TF32 split), chunks of up to kc k:
// Bbar[Rp][kl][c] = sum_q conj(P_q(Rp)) xbar[q][kl][c] (xbar FP32 complex [nq][kc][nc]).
epw_status tc_sbwd_plan(Arena &A, const epw_model *m, int nq, int kc, TcBwdBuffers &w);
epw_status tc_sbwd_phases(const epw_model *m, int nq, const double *q, TcBwdBuffers &w, cudaStream_t st);
epw_status tc_sbwd_contract(const epw_model *m, int kc, int nq, const cx<float> *xbar, TcBwdBuffers &w,
                            cx<float> *Bbar, cudaStream_t st);
// Accumulates dL/dgw into gwbar [nRe][nRp][nm][nw][nw] and (dL/dT, dL/dE_F) into scal[0..1],
// for L = sum c_nk Im Sigma_nk with c = cot [nk][nw] (device).
epw_status tc_linewidth_backward(const epw_model *m, int nk, int nq, const double *q, const double *wq,
                                 const epw_params *par, const double *epsk, const cx<double> *Uk,
                                 const cx<float> *Pk32, const double *omegaT, const cx<float> *ET32,
                                 const cx<float> *Bg32, const cx<float> *BH32, const double *cot, TcBuffers &b,
                                 TcBwdBuffers &w, cx<float> *gwbar, double *scal, cudaStream_t st);

// Staged tensor-core form for shapes the fused kernel cannot hold (nw <= 18,
// 3nat <= 18; K = [Re phases | zero pad | Rp phases] when Re != Rp): per chunk of k, a tcgen05 GEMM writes
// Ct[kl*cpk + 2c + s][q] (c over [H(k+q)_ij | (g_a(k,q) U_k)_jn], s = re/im),
// or Ct[q][kl*cpk + 2c + s] for the warp-per-pair kernel, which the per-pair
// kernel reads.
struct TcStaged {
  void *Ahi, *Alo;  // q phases [nq][kpad]
  void *Bhi, *Blo;  // k-side operand of one chunk [kc][cpk][kpad]
  float *Ct;        // [ntiles*144 rows][ldc], or q-major [ldc][ldn] when qmajor
  int op, kpad, cpk, kc, mtiles, ldc;
  int kg0;          // K offset of the vertex's Rp phases when Rp differs from Re (0: one shared set)
  bool ok;
  bool qmajor;      // layout read by the warp-per-pair kernel (nw > 8 or 3nat > 9)
  size_t ldn;
  const cx<double> *Pq64;  // FP64 q phases of the Re set [nR][nq] when already formed (else null)
  // leading dimension for the per-pair kernel's reads
  size_t pair_ld() const { return qmajor ? ldn : (size_t)ldc; }
};
bool tc_staged_supported(const epw_model *m);
// Buffers for chunks of up to `kc` k-points, kc chosen so Ct stays within ct_budget bytes.
// any_shape: also for shapes the fused kernel serves (per-q sums over k use the staged form).
epw_status tc_staged_plan(Arena &A, const epw_model *m, int nk, int nq, int op, size_t ct_budget, TcStaged &s,
                          bool any_shape = false);
// Split q-phase operand (once per call).
epw_status tc_staged_phases(const epw_model *m, int nq, const double *q, TcStaged &s, cudaStream_t st);
// Contraction of k-points [k0, k0 + kc) into s.Ct.
epw_status tc_staged_contract(const epw_model *m, int k0, int kc, int nq, const cx<float> *Bg32,
                              const cx<float> *BH32, TcStaged &s, cudaStream_t st);

// One bounded mbarrier wait, on a barrier nothing arrives at, for `cycles` clock cycles
// (the kernels' wait with a short limit): sets EPW_DEV_TIMEOUT in dstatus and *waited_out = 1.
epw_status tc_wait_selftest(long long cycles, unsigned *dstatus, int *waited_out, cudaStream_t st);
