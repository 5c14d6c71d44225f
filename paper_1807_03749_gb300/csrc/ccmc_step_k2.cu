// ccmc_step_k2.cu -- the step kernels for determinants of 2 words (65-128 spin-orbitals), FP64 and FP32 matrix elements.
#include "ccmc_kernels.cuh"

namespace ccmc {

template cudaError_t launch_phases<2, double>(const StepArgs *, int, const Shapes &, bool, cudaStream_t, i64 *,
                                                const cudaEvent_t *, const FlatPlan *);
template cudaError_t launch_phases<2, float>(const StepArgs *, int, const Shapes &, bool, cudaStream_t, i64 *,
                                                const cudaEvent_t *, const FlatPlan *);

}  // namespace ccmc
