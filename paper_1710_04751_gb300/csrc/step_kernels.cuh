// step_kernels.cuh -- the single-cavity kernels of the fused stream-and-collide time step
// of arXiv:1710.04751 (the node update itself is node.cuh / pair.cuh) and their launcher,
// templated on UNIT: the update at the paper's unit higher-order rates (collide_unit.cuh)
// or at general rates.  step.cu instantiates the general form and chooses between the
// two; step_unit.cu instantiates the unit-rate form (two translation units compile in
// parallel).
#pragma once

#include <type_traits>

#include "node.cuh"
#include "pair.cuh"

namespace lbm {

// Programmatic dependent launch of the step kernels (LBM_PDL): a step kernel is launched
// so that its blocks may be scheduled while the kernel before it on the stream drains its
// last wave; every block first waits (griddepcontrol.wait) for that kernel's completion
// and memory -- before it reads or writes anything -- and then allows the next step's
// launch to begin (griddepcontrol.launch_dependents).  Launched without the attribute
// (the batched and slab paths) both instructions do nothing.
#ifndef LBM_PDL
#define LBM_PDL 1
#endif
__device__ __forceinline__ void pdl_begin() {
    if (LBM_PDL) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }
}

template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = LBM_PDL ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Generic kernel: one thread per node of the flattened grid, any boundary mode.
// The step number of the 16-bit forms' rounding dither: read from the counter of the
// source buffer's parity; the launch's first thread writes the next value into the other
// parity's counter, which no thread of this launch reads (the next launch, in stream
// order, does).
template <typename S>
__device__ __forceinline__ uint32_t step_of(const unsigned* __restrict__ ctr_in,
                                            unsigned* __restrict__ ctr_out) {
    if constexpr (Storage<S>::deviation) {
        const uint32_t step = *ctr_in;
        if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0)
            *ctr_out = step + 1;
        return step;
    } else {
        return 0;
    }
}

template <typename S, int Q, bool UNIT>
__global__ void __launch_bounds__(256) step_kernel(const S* __restrict__ Fin,
                                                   const S* __restrict__ Gin,
                                                   const float* __restrict__ Tin,
                                                   S* __restrict__ Fout, S* __restrict__ Gout,
                                                   float* __restrict__ Tout, ParamsOf<S> p,
                                                   const unsigned* __restrict__ ctr_in,
                                                   unsigned* __restrict__ ctr_out) {
    using real = typename Storage<S>::real;
    pdl_begin();
    const uint32_t step = step_of<S>(ctr_in, ctr_out);
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.ncell) return;
    const int i = (int)(c % p.nx);
    const int64_t t = c / p.nx;
    const int j = (int)(t % p.ny);
    const int k = (int)(t / p.ny);
    real f[15], g[Q];
    pull<S, Q>(Fin, Gin, Tin, p, i, j, k, c, f, g);
    uint32_t seed = 0;
    if constexpr (Storage<S>::deviation) seed = dither_seed((uint32_t)(p.cell0 + c), step);
    collide_store<S, Q, UNIT>(f, g, Fout, Gout, Tout, p, c, seed);
}

// ---------------------------------------------------------------------------------
// Cavity kernel: one block per x-row segment (blockIdx.y = j, blockIdx.z = k), so the
// y/z wall tests are block-uniform.
// ---------------------------------------------------------------------------------
template <typename S, int Q, bool UNIT>
__global__ void __launch_bounds__(128, (cavity_min_blocks<S, Q>()))
    step_cavity_kernel(const S* __restrict__ Fin, const S* __restrict__ Gin,
                       const float* __restrict__ Tin, S* __restrict__ Fout,
                       S* __restrict__ Gout, float* __restrict__ Tout, ParamsOf<S> p,
                       const unsigned* __restrict__ ctr_in, unsigned* __restrict__ ctr_out) {
    pdl_begin();
    const uint32_t step = step_of<S>(ctr_in, ctr_out);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= p.nx) return;
    const bool interior = j >= 1 && j + 1 < p.ny && k >= 1 && k + 1 < p.nz;
    if (interior) cavity_node<S, Q, true, UNIT>(Fin, Gin, Tin, Fout, Gout, Tout, p, i, j, k, step);
    else cavity_node<S, Q, false, UNIT>(Fin, Gin, Tin, Fout, Gout, Tout, p, i, j, k, step);
}

// ---------------------------------------------------------------------------------
// Pair kernel of the 16-bit forms: one thread per pair of nodes (2t, 2t+1) of an x-row
// (blockIdx.y = j, blockIdx.z = k), nx even.  Rows away from the y and z walls take the
// packed pair update (pair.cuh); rows at a y or z wall update the two nodes one after
// the other with the general pull.
// ---------------------------------------------------------------------------------
constexpr int kPairThreads = 64;

// Resident blocks per SM the pair kernel is built for (sets its register budget: 128 for
// 7 or 8 blocks of 64 threads).  Measured: 7-8 beat 5-6 (168-204 registers, fewer warps)
// and 10 (96 registers, spills) at 128^3.
#ifndef LBM_PAIR_MIN_BLOCKS_Q15
#define LBM_PAIR_MIN_BLOCKS_Q15 7
#endif
#ifndef LBM_PAIR_MIN_BLOCKS_Q7
#define LBM_PAIR_MIN_BLOCKS_Q7 8
#endif
// The unit-rate pair update (fewer live values): D3Q15 measured best at 8 blocks of 64
// (128 registers; 10 and 14 blocks were 4% and 7% slower at 128^3), D3Q7 at 14 (72
// registers; 10% faster than 8 at 128^3 and 256^3).  FP16 D3Q15 with every load issued
// ahead of the arithmetic (pair_node_unit_early) needs 106 registers, and at 10 blocks it
// is 4.5% faster than the compiler's order at 8 (68.4 against 71.6 us at 128^3, 426 against
// 443 us at 256^3); BF16 measured 2% slower that way and keeps the compiler's order.
#ifndef LBM_PAIR_UNIT_MIN_BLOCKS_Q15
#define LBM_PAIR_UNIT_MIN_BLOCKS_Q15 8
#endif
#ifndef LBM_PAIR_UNIT_MIN_BLOCKS_Q7
#define LBM_PAIR_UNIT_MIN_BLOCKS_Q7 14
#endif
#ifndef LBM_PAIR_EARLY_MIN_BLOCKS
#define LBM_PAIR_EARLY_MIN_BLOCKS 10
#endif
#ifndef LBM_PAIR_EARLY_LOADS
#define LBM_PAIR_EARLY_LOADS 1
#endif
#ifndef LBM_PAIR_EARLY_Q7
#define LBM_PAIR_EARLY_Q7 0
#endif
#ifndef LBM_PAIR_EARLY_BF16
#define LBM_PAIR_EARLY_BF16 0
#endif
#ifndef LBM_PAIR_EARLY_MIN_BLOCKS_Q7
#define LBM_PAIR_EARLY_MIN_BLOCKS_Q7 14
#endif
template <typename S, int Q, bool UNIT>
constexpr bool pair_early_loads() {
    return LBM_PAIR_EARLY_LOADS && UNIT && (Q == 15 || LBM_PAIR_EARLY_Q7) &&
           (std::is_same<S, __half>::value || LBM_PAIR_EARLY_BF16);
}

template <typename S, int Q, bool UNIT>
constexpr int pair_min_blocks() {
    return pair_early_loads<S, Q, UNIT>() ? (Q == 15 ? LBM_PAIR_EARLY_MIN_BLOCKS : LBM_PAIR_EARLY_MIN_BLOCKS_Q7)
           : UNIT ? (Q == 15 ? LBM_PAIR_UNIT_MIN_BLOCKS_Q15 : LBM_PAIR_UNIT_MIN_BLOCKS_Q7)
                  : (Q == 15 ? LBM_PAIR_MIN_BLOCKS_Q15 : LBM_PAIR_MIN_BLOCKS_Q7);
}

template <typename S, int Q, bool UNIT>
__device__ __forceinline__ void pair_row(const S* __restrict__ Fin, const S* __restrict__ Gin,
                                         const float* __restrict__ Tin, S* __restrict__ Fout,
                                         S* __restrict__ Gout, float* __restrict__ Tout, const ParamsOf<S>& p,
                                         const PairParams& q, int t, int j, int k, uint32_t step) {
    const int npair = p.nx >> 1;
    if (t >= npair) return;
    if (j >= 1 && j + 1 < p.ny && k >= 1 && k + 1 < p.nz) {
        const int nx = p.nx, nxy = nx * p.ny;
        const int c0 = k * nxy + j * nx + 2 * t;
        const uint32_t seed = dither_weyl((uint32_t)(p.cell0 + c0), step);  // the pair hashes it
        if constexpr (UNIT) {
            if constexpr (pair_early_loads<S, Q, UNIT>())
                pair_node_unit_early<S, Q>(Fin, Gin, Tin, Fout, Gout, Tout, q, nx, nxy, (int)p.plane, c0,
                                           t == 0, t == npair - 1, seed);
            else
                pair_node_unit<S, Q>(Fin, Gin, Tin, Fout, Gout, Tout, q, nx, nxy, (int)p.plane, c0,
                                     t == 0, t == npair - 1, seed);
        }
        else
            pair_node<S, Q>(Fin, Gin, Tin, Fout, Gout, Tout, q, nx, nxy, (int)p.plane, c0,
                            t == 0, t == npair - 1, seed);
    } else {
#pragma unroll 1
        for (int e = 0; e < 2; ++e)
            cavity_node<S, Q, false, UNIT>(Fin, Gin, Tin, Fout, Gout, Tout, p, 2 * t + e, j, k, step);
    }
}

template <typename S, int Q, bool UNIT>
__global__ void __launch_bounds__(kPairThreads, (pair_min_blocks<S, Q, UNIT>()))
    step_pair_kernel(const S* __restrict__ Fin, const S* __restrict__ Gin,
                     const float* __restrict__ Tin, S* __restrict__ Fout,
                     S* __restrict__ Gout, float* __restrict__ Tout, ParamsOf<S> p,
                     PairParams q, const unsigned* __restrict__ ctr_in,
                     unsigned* __restrict__ ctr_out) {
    pdl_begin();
    const uint32_t step = step_of<S>(ctr_in, ctr_out);
    pair_row<S, Q, UNIT>(Fin, Gin, Tin, Fout, Gout, Tout, p, q, blockIdx.x * blockDim.x + threadIdx.x,
                         blockIdx.y, blockIdx.z, step);
}

// The pair parameters of a context's FP32 parameters, every value broadcast to both lanes.
inline PairParams make_pair_params(const DevParams<float>& p, int Q) {
    auto b = [](float v) { return make_float2(v, v); };
    PairParams q;
    for (int a = 0; a < 15; ++a) {
        q.wf[a] = b(p.wf[a]);
        q.wg[a] = b(p.wg[a]);
        q.nwg[a] = b(-p.wg[a]);
        q.wTc2[a] = 2.0f * p.wg[a] * p.T_cold;
        q.wTh2[a] = 2.0f * p.wg[a] * p.T_hot;
        q.nomf[a] = b(-p.om_f[a]);
        q.nomg[a] = b(-p.om_g[a]);
    }
    const float cs2 = 1.0f / 3.0f;
    q.omf9 = b(p.om_f[9]);
    q.omf14 = b(p.om_f[14]);
    for (int i = 0; i < 3; ++i) q.cf3[i] = b((1.0f - p.om_f[10 + i]) * cs2);
    const float cp = p.cs2_phi;
    q.omg_tr = b(p.om_g[Q == 15 ? 9 : 6] * (3.0f * cp));
    q.omg_4 = b(p.om_g[14] * (cp * cp));
    q.cs2 = b(cp);
    q.cs4 = b(cp * cp);
    q.R = b(p.heat_source);
    q.halfR = b(0.5f * p.heat_source);
    q.gbeta = b(p.gbeta);
    q.T0 = b(p.T0);
    q.fx = b(p.ext_fx);
    q.fy = b(p.ext_fy);
    q.fz = b(p.ext_fz);
    q.halffx = b(0.5f * p.ext_fx);
    q.halffy = b(0.5f * p.ext_fy);
    q.e4_mode = p.e4_mode;
    UnitRates<Pair>& u = q.ur;
    auto P = [](double v) { return Pair{make_float2((float)v, (float)v)}; };
    for (int i = 0; i < 3; ++i) {
        u.om1[i] = P(1.0 - (double)p.om_f[4 + i]);
        u.omg[i] = P(1.0 - (double)p.om_g[1 + i]);
    }
    u.omA = P(1.0 - (double)p.om_f[7]);
    u.omB = P(1.0 - (double)p.om_f[8]);
    u.cs2 = P((double)p.cs2_phi);
    u.cs4 = P((double)p.cs2_phi * (double)p.cs2_phi);
    u.R = P((double)p.heat_source);
    u.halfR = P(0.5 * (double)p.heat_source);
    u.e4_mode = p.e4_mode;
    return q;
}

template <typename S, bool UNIT>
bool launch_pair(const DevState& s, int cur, const ParamsOf<S>& p, cudaStream_t st) {
    if constexpr (!Storage<S>::deviation) {
        return false;
    } else {
        if (p.boundary != 0 || (p.nx & 1) || p.ny > 65535 || p.nz > 65535 ||
            15 * p.plane >= (int64_t(1) << 31))
            return false;
        const S* Fin = static_cast<const S*>(s.F[cur]);
        const S* Gin = static_cast<const S*>(s.G[cur]);
        S* Fout = static_cast<S*>(s.F[cur ^ 1]);
        S* Gout = static_cast<S*>(s.G[cur ^ 1]);
        const float* Tin = static_cast<const float*>(s.T[cur]);
        float* Tout = static_cast<float*>(s.T[cur ^ 1]);
        const PairParams q = make_pair_params(p, s.Q);
        const int npair = p.nx / 2;
        const int bx = npair <= 32 ? 32 : kPairThreads;
        const dim3 grid((npair + bx - 1) / bx, p.ny, p.nz);
        if (s.Q == 15)
            launch_pdl(step_pair_kernel<S, 15, UNIT>, grid, dim3(bx), st, Fin, Gin, Tin, Fout, Gout, Tout, p, q,
                       (const unsigned*)(s.step_ctr + cur), s.step_ctr + (cur ^ 1));
        else
            launch_pdl(step_pair_kernel<S, 7, UNIT>, grid, dim3(bx), st, Fin, Gin, Tin, Fout, Gout, Tout, p, q,
                       (const unsigned*)(s.step_ctr + cur), s.step_ctr + (cur ^ 1));
        return true;
    }
}


template <typename S, bool UNIT>
cudaError_t launch_step_as(const DevState& s, int cur, const ParamsOf<S>& p, cudaStream_t st) {
    const S* Fin = static_cast<const S*>(s.F[cur]);
    const S* Gin = static_cast<const S*>(s.G[cur]);
    S* Fout = static_cast<S*>(s.F[cur ^ 1]);
    S* Gout = static_cast<S*>(s.G[cur ^ 1]);
    const float* Tin = static_cast<const float*>(s.T[cur]);
    float* Tout = static_cast<float*>(s.T[cur ^ 1]);
    if (launch_pair<S, UNIT>(s, cur, p, st)) return cudaGetLastError();
    const unsigned* ctr_in = s.step_ctr ? s.step_ctr + cur : nullptr;
    unsigned* ctr_out = s.step_ctr ? s.step_ctr + (cur ^ 1) : nullptr;
    if (p.boundary == 0 && p.ny <= 65535 && p.nz <= 65535 && 15 * p.plane < (int64_t(1) << 31)) {
        const int bx = 128;
        const dim3 grid((p.nx + bx - 1) / bx, p.ny, p.nz);
        if (s.Q == 15)
            return launch_pdl(step_cavity_kernel<S, 15, UNIT>, grid, dim3(bx), st, Fin, Gin, Tin, Fout, Gout,
                              Tout, p, ctr_in, ctr_out);
        return launch_pdl(step_cavity_kernel<S, 7, UNIT>, grid, dim3(bx), st, Fin, Gin, Tin, Fout, Gout, Tout,
                          p, ctr_in, ctr_out);
    }
    const int threads = 256;
    const int64_t blocks = (p.ncell + threads - 1) / threads;
    if (s.Q == 15)
        return launch_pdl(step_kernel<S, 15, UNIT>, dim3((unsigned)blocks), dim3(threads), st, Fin, Gin, Tin,
                          Fout, Gout, Tout, p, ctr_in, ctr_out);
    return launch_pdl(step_kernel<S, 7, UNIT>, dim3((unsigned)blocks), dim3(threads), st, Fin, Gin, Tin, Fout,
                      Gout, Tout, p, ctr_in, ctr_out);
}

}  // namespace lbm
