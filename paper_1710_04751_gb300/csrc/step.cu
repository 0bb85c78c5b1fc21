// step.cu -- the single-cavity step launcher: the kernels of step_kernels.cuh at general
// rates (instantiated here) or at the paper's unit higher-order rates (step_unit.cu).
#include "step_kernels.cuh"

namespace lbm {

template <typename S>
cudaError_t launch_step_unit(const DevState& s, int cur, const ParamsOf<S>& p, cudaStream_t st);

template <typename S>
cudaError_t launch_step(const DevState& s, int cur, const ParamsOf<S>& p, cudaStream_t st) {
    if (has_unit_rates(p, s.Q)) return launch_step_unit<S>(s, cur, p, st);
    return launch_step_as<S, false>(s, cur, p, st);
}

template cudaError_t launch_step<double>(const DevState&, int, const ParamsOf<double>&, cudaStream_t);
template cudaError_t launch_step<float>(const DevState&, int, const ParamsOf<float>&, cudaStream_t);
template cudaError_t launch_step<__half>(const DevState&, int, const ParamsOf<__half>&, cudaStream_t);
template cudaError_t launch_step<__nv_bfloat16>(const DevState&, int, const ParamsOf<__nv_bfloat16>&,
                                                cudaStream_t);

}  // namespace lbm
