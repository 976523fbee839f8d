// sweep_fp32.cu — the two-sweep kernels (sweep.cuh) for FP32 elements.
#include "sweep.cuh"

namespace dsfft {

template SweepFn sweep_lookup<kFP32>(bool, bool, bool, int);
template cudaError_t sweep_prepare_ls<kFP32>(bool, int);

}  // namespace dsfft
