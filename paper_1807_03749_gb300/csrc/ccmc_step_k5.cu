// ccmc_step_k5.cu -- the step kernels for determinants of 5 words (257-320 spin-orbitals), FP64 matrix elements.
#include "ccmc_kernels.cuh"

namespace ccmc {

template cudaError_t launch_phases<5, double>(const StepArgs *, int, const Shapes &, bool, cudaStream_t, i64 *,
                                                const cudaEvent_t *, const FlatPlan *);

}  // namespace ccmc
