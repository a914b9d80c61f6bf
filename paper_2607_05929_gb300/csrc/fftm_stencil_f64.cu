// The residual, commit, state and statistics kernels of fftm_stencil.cuh instantiated for
// FP64 fields.
#include "fftm_stencil.cuh"
#include "../../include/fftm.h"

namespace fftm {

template cudaError_t launch_residual<double>(const ResParams<double>&, int, bool, cudaStream_t, int*);
template int residual_blocks<double>(const ResParams<double>&, int);
template bool residual_one_pass<double>(const ResParams<double>&);
template cudaError_t launch_commit<double>(const ResParams<double>&, int, double*, cudaStream_t);
template cudaError_t launch_state_io<double>(const ResParams<double>&, int, double*, const double*, cudaStream_t);
template cudaError_t launch_voxel_fields<double>(const ResParams<double>&, int, double*, double*, cudaStream_t);
template cudaError_t launch_stats<double>(const ResParams<double>&, int, double*, int, cudaStream_t);

}  // namespace fftm

extern "C" int fftm_host_log_j2(const double* G, const double* params, const double* st, double* S,
                                double* st_out) {
  if (!G || !params || !st || !S) return FFTM_E_INVALID;
  fftm::log_j2_eval<double>(params, G, st, S, st_out);
  return FFTM_OK;
}
