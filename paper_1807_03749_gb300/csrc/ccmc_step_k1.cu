// ccmc_step_k1.cu -- the step kernels for determinants of 1 word (1-64 spin-orbitals), FP64 and FP32 matrix elements.
#include "ccmc_kernels.cuh"

namespace ccmc {

template cudaError_t launch_phases<1, double>(const StepArgs *, int, const Shapes &, bool, cudaStream_t, i64 *,
                                                const cudaEvent_t *, const FlatPlan *);
template cudaError_t launch_phases<1, float>(const StepArgs *, int, const Shapes &, bool, cudaStream_t, i64 *,
                                                const cudaEvent_t *, const FlatPlan *);

}  // namespace ccmc
