// ccmc_step_k4.cu -- the step kernels for determinants of 4 words (193-256 spin-orbitals), FP64 matrix elements.
#include "ccmc_kernels.cuh"

namespace ccmc {

template cudaError_t launch_phases<4, double>(const StepArgs *, int, const Shapes &, bool, cudaStream_t, i64 *,
                                                const cudaEvent_t *, const FlatPlan *);

}  // namespace ccmc
