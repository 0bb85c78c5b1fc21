// equilibrium.cu -- a context's populations set to the equilibria of given fields: for
// the flow the populations whose central moments are the equilibria of the flow
// collision (App. A: Maxwellian, c_s^2 = 1/3) at (rho, u); for the scalar those whose
// central moments are the equilibria of Eq. (15) at (T, u).
//
// Each node starts from populations with the right conserved moments -- rho w_a
// (1 + e_a.u / c_s^2) for the flow (sum rho, first moment rho u) and w^phi_a T
// (1 + e_a.u / c_sphi^2) for the scalar (sum T, first moment T u) -- and takes one
// collision with every relaxation rate 1, no force and no source: every non-conserved
// central moment then equals its equilibrium and the conserved ones are unchanged.
#include "collide.cuh"
#include "internal.h"
#include "lattice.cuh"

namespace lbm {

template <typename S, int Q>
__global__ void set_fields_kernel(S* __restrict__ F, S* __restrict__ G, float* __restrict__ Tn,
                                  ParamsOf<S> p, const double* __restrict__ rho,
                                  const double* __restrict__ ux, const double* __restrict__ uy,
                                  const double* __restrict__ uz, const double* __restrict__ T) {
    using real = typename Storage<S>::real;
    using St = Storage<S>;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.ncell) return;
    ParamsOf<S> q = p;  // every rate 1, no force, no source
#pragma unroll
    for (int b = 0; b < 15; ++b) {
        q.om_f[b] = real(1);
        q.om_g[b] = real(1);
    }
    q.heat_source = real(0);
    const real r = rho ? (real)rho[c] : real(1);
    const real u[3] = {(real)ux[c], (real)uy[c], (real)uz[c]};
    const real t = (real)T[c];
    real f[15], g[Q];
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        const real eu = ex(a) * u[0] + ey(a) * u[1] + ez(a) * u[2];
        f[a] = r * p.wf[a] * (real(1) + real(3) * eu);  // wf: the flow rest weights
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const real eu = ex(a) * u[0] + ey(a) * u[1] + ez(a) * u[2];
        g[a] = t * p.wg[a] * (real(1) + eu / p.cs2_phi);
    }
    real vx, vy, vz;
    collide_flow<real>(f, real(0), real(0), real(0), q, vx, vy, vz);
    if constexpr (Q == 15) collide_thermal15<real>(g, u[0], u[1], u[2], q);
    else collide_thermal7<real>(g, u[0], u[1], u[2], q);
#pragma unroll
    for (int a = 0; a < 15; ++a) F[a * p.plane + c] = St::store_f(f[a], p.wf[a]);
    if constexpr (St::deviation) Tn[c] = (float)t;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        real off = real(0);
        if constexpr (St::deviation) off = p.wg[a] * t;
        G[a * p.plane + c] = St::store(g[a], off);
    }
}

// Equilibria (f, g) at (rho, u, T) into f_out, g_out: the construction of the file comment.
template <typename real, int Q>
__device__ __forceinline__ void equilibria(const DevParams<real>& unit, real r, const real (&u)[3],
                                           real t, real (&f)[15], real (&g)[Q]) {
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        const real eu = ex(a) * u[0] + ey(a) * u[1] + ez(a) * u[2];
        f[a] = r * unit.wf[a] * (real(1) + real(3) * eu);
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const real eu = ex(a) * u[0] + ey(a) * u[1] + ez(a) * u[2];
        g[a] = t * unit.wg[a] * (real(1) + eu / unit.cs2_phi);
    }
    real vx, vy, vz;
    collide_flow<real>(f, real(0), real(0), real(0), unit, vx, vy, vz);
    if constexpr (Q == 15) collide_thermal15<real>(g, u[0], u[1], u[2], unit);
    else collide_thermal7<real>(g, u[0], u[1], u[2], unit);
}

// Moves the macroscopic u and T of every node back to the targets and keeps each node's
// departure from equilibrium: p <- p - p_eq(current fields) + p_eq(target fields), with
// rho unchanged (the current rho; u and T as lbm_fields defines them).  Repeated after
// steps of the solver, this lets the non-equilibrium parts (stresses, heat fluxes) adapt
// to the imposed fields -- the iterative consistent initialisation of Mei, Luo, Lallemand
// & d'Humieres (Computers & Fluids 35, 2006), applied to u and T.
template <typename S, int Q>
__global__ void reimpose_kernel(S* __restrict__ F, S* __restrict__ G, float* __restrict__ Tn,
                                ParamsOf<S> p, const double* __restrict__ ux,
                                const double* __restrict__ uy, const double* __restrict__ uz,
                                const double* __restrict__ T) {
    using real = typename Storage<S>::real;
    using St = Storage<S>;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.ncell) return;
    ParamsOf<S> q = p;
#pragma unroll
    for (int b = 0; b < 15; ++b) {
        q.om_f[b] = real(1);
        q.om_g[b] = real(1);
    }
    q.heat_source = real(0);
    real f[15], g[Q];
    real r = 0, jx = 0, jy = 0, jz = 0, t = 0;
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        f[a] = St::load_f(F[a * p.plane + c], p.wf[a]);
        r += f[a];
        jx += ex(a) * f[a];
        jy += ey(a) * f[a];
        jz += ez(a) * f[a];
    }
    const real Tref = St::deviation ? (real)Tn[c] : real(0);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        g[a] = St::load(G[a * p.plane + c], p.wg[a] * Tref);
        t += g[a];
    }
    t -= real(0.5) * p.heat_source;
    const real Fz = p.ext_fz + p.gbeta * (t - p.T0);
    const real uc[3] = {(jx - real(0.5) * p.ext_fx) / r, (jy - real(0.5) * p.ext_fy) / r,
                        (jz - real(0.5) * Fz) / r};
    const real ut[3] = {(real)ux[c], (real)uy[c], (real)uz[c]};
    const real tt = (real)T[c];
    real fc[15], gc[Q], ft[15], gt[Q];
    equilibria<real, Q>(q, r, uc, t, fc, gc);
    equilibria<real, Q>(q, r, ut, tt, ft, gt);
#pragma unroll
    for (int a = 0; a < 15; ++a) F[a * p.plane + c] = St::store_f(f[a] - fc[a] + ft[a], p.wf[a]);
    if constexpr (St::deviation) Tn[c] = (float)tt;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        real off = real(0);
        if constexpr (St::deviation) off = p.wg[a] * tt;
        G[a * p.plane + c] = St::store(g[a] - gc[a] + gt[a], off);
    }
}

template <typename S>
cudaError_t launch_reimpose(const DevState& s, int cur, const ParamsOf<S>& p, const double* ux,
                            const double* uy, const double* uz, const double* T, cudaStream_t st) {
    const int threads = 128;
    const unsigned blocks = (unsigned)((p.ncell + threads - 1) / threads);
    S* F = static_cast<S*>(s.F[cur]);
    S* G = static_cast<S*>(s.G[cur]);
    float* Tn = static_cast<float*>(s.T[cur]);
    if (s.Q == 15)
        reimpose_kernel<S, 15><<<blocks, threads, 0, st>>>(F, G, Tn, p, ux, uy, uz, T);
    else
        reimpose_kernel<S, 7><<<blocks, threads, 0, st>>>(F, G, Tn, p, ux, uy, uz, T);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_set_fields(const DevState& s, int cur, const ParamsOf<S>& p, const double* rho,
                              const double* ux, const double* uy, const double* uz,
                              const double* T, cudaStream_t st) {
    const int threads = 128;
    const unsigned blocks = (unsigned)((p.ncell + threads - 1) / threads);
    S* F = static_cast<S*>(s.F[cur]);
    S* G = static_cast<S*>(s.G[cur]);
    float* Tn = static_cast<float*>(s.T[cur]);
    if (s.Q == 15)
        set_fields_kernel<S, 15><<<blocks, threads, 0, st>>>(F, G, Tn, p, rho, ux, uy, uz, T);
    else
        set_fields_kernel<S, 7><<<blocks, threads, 0, st>>>(F, G, Tn, p, rho, ux, uy, uz, T);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE_SET(S)                                                                  \
    template cudaError_t launch_set_fields<S>(const DevState&, int, const ParamsOf<S>&,          \
                                              const double*, const double*, const double*,      \
                                              const double*, const double*, cudaStream_t);      \
    template cudaError_t launch_reimpose<S>(const DevState&, int, const ParamsOf<S>&,            \
                                            const double*, const double*, const double*,        \
                                            const double*, cudaStream_t);
LBM_INSTANTIATE_SET(double)
LBM_INSTANTIATE_SET(float)
LBM_INSTANTIATE_SET(__half)
LBM_INSTANTIATE_SET(__nv_bfloat16)

}  // namespace lbm
