// The residual, commit, state and statistics kernels of fftm_stencil.cuh instantiated for
// FP32 fields.
#include "fftm_stencil.cuh"

namespace fftm {

template cudaError_t launch_residual<float>(const ResParams<float>&, int, bool, cudaStream_t, int*);
template int residual_blocks<float>(const ResParams<float>&, int);
template bool residual_one_pass<float>(const ResParams<float>&);
template cudaError_t launch_commit<float>(const ResParams<float>&, int, float*, cudaStream_t);
template cudaError_t launch_state_io<float>(const ResParams<float>&, int, float*, const float*, cudaStream_t);
template cudaError_t launch_voxel_fields<float>(const ResParams<float>&, int, float*, float*, cudaStream_t);
template cudaError_t launch_stats<float>(const ResParams<float>&, int, double*, int, cudaStream_t);

}  // namespace fftm
