// sweep_bf16.cu — the two-sweep kernels (sweep.cuh) for BF16 elements.
#include "sweep.cuh"

namespace dsfft {

template SweepFn sweep_lookup<kBF16>(bool, bool, bool, int);
template cudaError_t sweep_prepare_ls<kBF16>(bool, int);

}  // namespace dsfft
