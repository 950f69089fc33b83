// Tensor-core (tcgen05, split-BF16) form of the fused linewidth kernel.
#pragma once
#include "epw_internal.cuh"

struct TcBuffers {
  void *Ahi, *Alo;   // q phases, bf16 split, K-major [nq_pad][Kpad]
  void *Bhi, *Blo;   // k-side vertex, bf16 split, K-major [nk][ncol][Kpad]
  double *partial;   // [nk][nqtiles][nw]
  int kpad, ncol, nqt;
};

epw_status tc_plan(Arena &A, const epw_model *m, int nk, int nq, TcBuffers &b);
epw_status tc_linewidth(const epw_model *m, int nk, const double *k, int nq, const double *q, const double *wq,
                        const epw_params *par, const cx<double> *PkRM, const double *epsk, const cx<double> *Uk,
                        const double *omegaT, const cx<float> *ET32, const cx<float> *Bg32, const cx<float> *BH32,
                        TcBuffers &b, double *out, cudaStream_t st);
void tc_free(epw_model *m);
