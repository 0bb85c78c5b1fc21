// step.cu -- the single-cavity kernels of the fused stream-and-collide time step of
// arXiv:1710.04751 (the node update itself is node.cuh) and their launcher.
#include "node.cuh"

namespace lbm {

// Generic kernel: one thread per node of the flattened grid, any boundary mode.
template <typename S, int Q>
__global__ void __launch_bounds__(256) step_kernel(const S* __restrict__ Fin,
                                                   const S* __restrict__ Gin,
                                                   const float* __restrict__ Tin,
                                                   S* __restrict__ Fout, S* __restrict__ Gout,
                                                   float* __restrict__ Tout, ParamsOf<S> p) {
    using real = typename Storage<S>::real;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.ncell) return;
    const int i = (int)(c % p.nx);
    const int64_t t = c / p.nx;
    const int j = (int)(t % p.ny);
    const int k = (int)(t / p.ny);
    real f[15], g[Q];
    pull<S, Q>(Fin, Gin, Tin, p, i, j, k, c, f, g);
    collide_store<S, Q>(f, g, Fout, Gout, Tout, p, c);
}

// ---------------------------------------------------------------------------------
// Cavity kernel: one block per x-row segment (blockIdx.y = j, blockIdx.z = k), so the
// y/z wall tests are block-uniform.
// ---------------------------------------------------------------------------------
template <typename S, int Q>
__global__ void __launch_bounds__(128, (cavity_min_blocks<S, Q>()))
    step_cavity_kernel(const S* __restrict__ Fin, const S* __restrict__ Gin,
                       const float* __restrict__ Tin, S* __restrict__ Fout,
                       S* __restrict__ Gout, float* __restrict__ Tout, ParamsOf<S> p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= p.nx) return;
    const bool interior = j >= 1 && j + 1 < p.ny && k >= 1 && k + 1 < p.nz;
    if (interior) cavity_node<S, Q, true>(Fin, Gin, Tin, Fout, Gout, Tout, p, i, j, k);
    else cavity_node<S, Q, false>(Fin, Gin, Tin, Fout, Gout, Tout, p, i, j, k);
}

template <typename S>
cudaError_t launch_step(const DevState& s, int cur, const ParamsOf<S>& p, cudaStream_t st) {
    const S* Fin = static_cast<const S*>(s.F[cur]);
    const S* Gin = static_cast<const S*>(s.G[cur]);
    S* Fout = static_cast<S*>(s.F[cur ^ 1]);
    S* Gout = static_cast<S*>(s.G[cur ^ 1]);
    const float* Tin = static_cast<const float*>(s.T[cur]);
    float* Tout = static_cast<float*>(s.T[cur ^ 1]);
    if (p.boundary == 0 && p.ny <= 65535 && p.nz <= 65535 && 15 * p.plane < (int64_t(1) << 31)) {
        const int bx = 128;
        const dim3 grid((p.nx + bx - 1) / bx, p.ny, p.nz);
        if (s.Q == 15)
            step_cavity_kernel<S, 15><<<grid, bx, 0, st>>>(Fin, Gin, Tin, Fout, Gout, Tout, p);
        else
            step_cavity_kernel<S, 7><<<grid, bx, 0, st>>>(Fin, Gin, Tin, Fout, Gout, Tout, p);
        return cudaGetLastError();
    }
    const int threads = 256;
    const int64_t blocks = (p.ncell + threads - 1) / threads;
    if (s.Q == 15)
        step_kernel<S, 15><<<(unsigned)blocks, threads, 0, st>>>(Fin, Gin, Tin, Fout, Gout, Tout, p);
    else
        step_kernel<S, 7><<<(unsigned)blocks, threads, 0, st>>>(Fin, Gin, Tin, Fout, Gout, Tout, p);
    return cudaGetLastError();
}

template cudaError_t launch_step<double>(const DevState&, int, const ParamsOf<double>&, cudaStream_t);
template cudaError_t launch_step<float>(const DevState&, int, const ParamsOf<float>&, cudaStream_t);
template cudaError_t launch_step<__half>(const DevState&, int, const ParamsOf<__half>&, cudaStream_t);
template cudaError_t launch_step<__nv_bfloat16>(const DevState&, int, const ParamsOf<__nv_bfloat16>&,
                                                cudaStream_t);

}  // namespace lbm
