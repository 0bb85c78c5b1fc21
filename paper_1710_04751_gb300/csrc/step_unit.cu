// step_unit.cu -- the single-cavity kernels at the paper's unit higher-order rates
// (collide_unit.cuh), compiled apart from the general form (step.cu).
#include "step_kernels.cuh"

namespace lbm {

template <typename S>
cudaError_t launch_step_unit(const DevState& s, int cur, const ParamsOf<S>& p, cudaStream_t st) {
    return launch_step_as<S, true>(s, cur, p, st);
}

template cudaError_t launch_step_unit<double>(const DevState&, int, const ParamsOf<double>&, cudaStream_t);
template cudaError_t launch_step_unit<float>(const DevState&, int, const ParamsOf<float>&, cudaStream_t);
template cudaError_t launch_step_unit<__half>(const DevState&, int, const ParamsOf<__half>&, cudaStream_t);
template cudaError_t launch_step_unit<__nv_bfloat16>(const DevState&, int,
                                                     const ParamsOf<__nv_bfloat16>&, cudaStream_t);

}  // namespace lbm
