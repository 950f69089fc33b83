// Placeholder: the tensor-core path is not built yet.
#include "epw_tc.cuh"

epw_status tc_plan(Arena &, const epw_model *, int, int, TcBuffers &b) {
  b = TcBuffers{};
  return EPW_OK;
}
epw_status tc_linewidth(const epw_model *, int, const double *, int, const double *, const double *,
                        const epw_params *, const cx<double> *, const double *, const cx<double> *, const double *,
                        const cx<float> *, const cx<float> *, const cx<float> *, TcBuffers &, double *,
                        cudaStream_t) {
  return EPW_ERR_UNSUPPORTED;
}
void tc_free(epw_model *) {}
