// ccmc_step_k6.cu -- the step kernels for determinants of 6 words (321-384 spin-orbitals), FP64 matrix elements.
#include "ccmc_kernels.cuh"

namespace ccmc {

template cudaError_t launch_phases<6, double>(const StepArgs *, int, const Shapes &, bool, cudaStream_t, i64 *,
                                                const cudaEvent_t *, const FlatPlan *);

}  // namespace ccmc
