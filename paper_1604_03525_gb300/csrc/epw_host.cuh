// Host-side orchestration shared by the C entry points (epw_api.cu) and the
// batch runner (epw_batch.cu): argument checks, the per-call plan of one
// linewidth job and its execution on a stream with device buffers only.
#pragma once
#include "epw_internal.cuh"
#include "epw_tc.cuh"

// Records the message for epw_last_error (thread-local) and returns s.
epw_status epwi_fail(epw_status s, const char *fmt, ...);
bool epwi_is_device_ptr(const void *p);
epw_status epwi_check_common(const epw_model *m, int nk, const double *k, int nq, const double *q);
epw_status epwi_check_params(const epw_params *p);

// Tile choices of one linewidth job (the autotuner's knobs).
struct EpwTune {
  size_t a_block_bytes;    // fused kernel: q-block of the A operand kept in L2 across the k groups
  size_t staged_ct_bytes;  // staged form: contraction buffer per chunk of k
  int wide_form;           // wide-shape form: TCW_FORM_PAIR (fused, CTA pairs), _SPLIT (two kernels), _SINGLE
  size_t k_side_bytes;     // buffers that grow with nk stay within this: larger k lists run in k chunks
};
EpwTune epwi_default_tune();

// Per-call device state of the preparation steps shared by every entry point.
struct Prep {
  double *kd, *qd, *wqd;
  cx<double> *PkRM, *PkT;  // k phases [nk][nRe], [nRe][nk]
  cx<double> *Hk;          // [nk][nw][nw]
  double *epsk;            // [nk][nw]
  cx<double> *Uk;          // [nk][nw][nw]
  void *PqTe, *PqTp;       // [nR][nq] in working precision
  cx<double> *PqTph;       // [nRph][nq] FP64 (phonons)
  cx<double> *D;           // [nq][nm][nm]
  double *w2;              // [nq][nm]
  cx<double> *ev;          // [nq][nm][nm]
  double *omegaT;          // [nm][nq]
  void *ET;                // [nm*nm][nq] working precision
  void *G1, *Bg, *BH;      // working precision
  cx<float> *Pk32, *gw32;  // FP32 copies for the k-side contraction
  void *Cpol;              // [nm][nq] long-range factors C_nu(q), working precision (polar models)
};

// Buffers of one linewidth job.
struct LwPlan {
  Prep p;
  double *partial;
  double *out_d;
  TcBuffers tc;
  TcStaged sg;
  TcwBuffers w;  // wide-shape fused form
  int kchunk;    // k per pass (the buffers are laid out for this many); the k list runs in passes
};

// Lays out (or, with a null arena base, measures) the buffers of one job.
// sk/sq/swq/sout: k, q, w_q or the output are host buffers staged on the device.
epw_status epwi_plan_linewidth(Arena &A, const epw_model *m, int nk, int nq, int prec, bool sk, bool sq, bool swq,
                               bool sout, const EpwTune &tune, LwPlan &L);
// Im Sigma [nk][nw] into the device buffer `out` from device k, q, w_q (may be
// null), with the buffers of L; enqueues work on st only (no host sync, no
// allocation), so it can be captured into a CUDA graph.  nk, nq > 0.
epw_status epwi_linewidth_exec(epw_model *m, int nk, const double *kd, int nq, const double *qd, const double *wqd,
                               const epw_params *par, LwPlan &L, double *out, cudaStream_t st);
