// Tensor-core (tcgen05, split-BF16) form of the fused linewidth kernel.
#pragma once
#include "epw_internal.cuh"

struct TcBuffers {
  void *Ahi, *Alo;   // q phases, bf16 split, K-major [nq][kpad]
  void *Bhi, *Blo;   // k-side vertex, bf16 split, K-major [nk_pad][cpk][kpad]
  float *nbT;        // Bose factors [nm][nq]
  double *partial;   // [nk][4*nqt][nw]
  int kpad, cpk, nk_pad, nqt, kpt;
  bool ok;           // shape has a tensor-core kernel
};

// Lay out (or measure, with a null arena base) the buffers of the tensor-core path.
epw_status tc_plan(Arena &A, const epw_model *m, int nk, int nq, TcBuffers &b);
// Im Sigma [nk][nw] into `out` (device) from the shared preparation outputs.
epw_status tc_linewidth(const epw_model *m, int nk, const double *k, int nq, const double *q, const double *wq,
                        const epw_params *par, const cx<double> *PkRM, const double *epsk, const cx<double> *Uk,
                        const double *omegaT, const cx<float> *ET32, const cx<float> *Bg32, const cx<float> *BH32,
                        TcBuffers &b, double *out, cudaStream_t st);
void tc_free(epw_model *m);
