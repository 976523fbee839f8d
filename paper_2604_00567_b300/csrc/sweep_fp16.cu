// sweep_fp16.cu — the two-sweep kernels (sweep.cuh) for FP16 elements.
#include "sweep.cuh"

namespace dsfft {

template SweepFn sweep_lookup<kFP16>(bool, bool, bool, int);
template cudaError_t sweep_prepare_ls<kFP16>(bool, int);

}  // namespace dsfft
