// node.cuh -- the update of one lattice node in the fused stream-and-collide step of
// arXiv:1710.04751, shared by the single-cavity kernels (step.cu) and the batched
// kernel (batch.cu).
//
// A thread pulls its 15 flow and Q thermal populations from the post-collision arrays
// of the previous step (Eqs. 2b, 13b), substitutes the wall rules for links whose source
// node lies outside the cavity (Sec. 3), computes T (Eq. 25), the Boussinesq force
// (Sec. 3) and u (Eq. 3), runs the flow collision (App. A) and the thermal collision
// (Sec. 2.2 or App. C) in registers and writes the post-collision populations of its
// own node to the other buffer.
//
// Memory layout: structure of arrays, population a of node c at a * plane + c with
// c = (k * ny + j) * nx + i; consecutive threads own consecutive x, so every load and
// store of a warp is one contiguous run (shifted by at most one element for e_x != 0).
// S is the storage type (storage.cuh); arithmetic is Storage<S>::real.  In the 16-bit
// forms a thermal population is stored as its deviation from w^phi_a T_node, where
// T_node is the temperature of the node that holds it (kept in an FP32 plane, Tin /
// Tout): the pull adds w^phi_a T of the source node back, the store subtracts
// w^phi_a T of this node.
#pragma once

#include "collide.cuh"
#include "collide_unit.cuh"
#include "internal.h"
#include "lattice.cuh"

namespace lbm {

// Source coordinate along one axis with periodic wrap when the axis is periodic.
__device__ __forceinline__ int wrap_axis(int s, int n, bool periodic) {
    if (periodic) {
        if (s < 0) s += n;
        else if (s >= n) s -= n;
    }
    return s;
}

// Offset a stored thermal population of node `node` decodes with (16-bit forms).
template <typename S>
__device__ __forceinline__ typename Storage<S>::real thermal_offset(const float* __restrict__ Tin,
                                                                    const ParamsOf<S>& p, int a,
                                                                    int64_t node) {
    if constexpr (Storage<S>::deviation) return p.wg[a] * Tin[node];
    else return typename Storage<S>::real(0);
}

// Pull of every link with the general wall rules (any boundary mode).
template <typename S, int Q>
__device__ __forceinline__ void pull(const S* __restrict__ Fin, const S* __restrict__ Gin,
                                     const float* __restrict__ Tin,
                                     const ParamsOf<S>& p, int i, int j, int k, int64_t c,
                                     typename Storage<S>::real (&f)[15],
                                     typename Storage<S>::real (&g)[Q]) {
    using real = typename Storage<S>::real;
    using St = Storage<S>;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int64_t P = p.plane;
    const bool px = p.boundary & 1, py = p.boundary & 2, pz = p.boundary & 4;
    const bool x_dirichlet = !(p.boundary & 8);
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        const int si = wrap_axis(i - ex(a), nx, px);
        const int sj = wrap_axis(j - ey(a), ny, py);
        const int sk = wrap_axis(k - ez(a), nz, pz);
        const bool in_x = (unsigned)si < (unsigned)nx;
        const bool in_y = (unsigned)sj < (unsigned)ny;
        const bool in_z = (unsigned)sk < (unsigned)nz;
        const int64_t s = ((int64_t)sk * ny + sj) * nx + si;
        // opposite / mirrored directions have the same rest weight as a
        if (in_x && in_y && in_z) {
            f[a] = St::load_f(Fin[a * P + s], p.wf[a]);
        } else {
            f[a] = St::load_f(Fin[opp(a) * P + c], p.wf[a]);  // no-slip: half-way bounce-back
        }
        if (a < Q) {
            if (in_x && in_y && in_z) {
                g[a] = St::load(Gin[a * P + s], thermal_offset<S>(Tin, p, a, s));
            } else if (x_dirichlet && !in_x) {
                // Dirichlet T: anti-bounce-back with the face temperature
                const real Tw = si < 0 ? p.T_cold : p.T_hot;
                g[a] = -St::load(Gin[opp(a) * P + c], thermal_offset<S>(Tin, p, a, c)) +
                       real(2) * p.wg[a] * Tw;
            } else if (p.adiabatic_mode == 1) {
                // adiabatic, specular: mirror the crossed components; the population is
                // the one that left toward the wall from the mirrored source node
                int di = ex(a), dj = ey(a), dk = ez(a), ri = si, rj = sj, rk = sk;
                if (!in_x) { di = -di; ri = i; }
                if (!in_y) { dj = -dj; rj = j; }
                if (!in_z) { dk = -dk; rk = k; }
                const int b = dir_index(di, dj, dk);
                const int64_t r = ((int64_t)rk * ny + rj) * nx + ri;
                g[a] = St::load(Gin[b * P + r], thermal_offset<S>(Tin, p, a, r));
            } else {
                // adiabatic, bounce-back
                g[a] = St::load(Gin[opp(a) * P + c], thermal_offset<S>(Tin, p, a, c));
            }
        }
    }
}

// Macroscopic variables, both collisions and the store of one node.  UNIT: the paper's
// unit higher-order rates (collide_unit.cuh), for which the post-collision state needs
// only the low-order moments of the pulled populations.
// seed: the node's rounding dither (dither_seed of its global index and the step) for
// the stochastically rounded flow stores of the 16-bit forms; unused otherwise.
template <typename S, int Q, bool UNIT = false>
__device__ __forceinline__ void collide_store(typename Storage<S>::real (&f)[15],
                                              typename Storage<S>::real (&g)[Q],
                                              S* __restrict__ Fout, S* __restrict__ Gout,
                                              float* __restrict__ Tout,
                                              const ParamsOf<S>& p, int64_t c, uint32_t seed = 0) {
    using real = typename Storage<S>::real;
    using St = Storage<S>;
    const int64_t P = p.plane;
    if constexpr (UNIT) {
        const UnitRates<real> r = unit_rates<real>(p);
        real m0, mx, my, mz;
        raw_first<real, Q>(g, m0, mx, my, mz);  // all the scalar collision needs of g
        const real T = m0 + r.halfR;             // Eq. (25)
        const real Fx = p.ext_fx, Fy = p.ext_fy, Fz = p.ext_fz + p.gbeta * (T - p.T0);
        Low10<real> dm = raw_low15<real>(f);     // moments of f - w_a: the rest state's are
        dm.m0 -= real(1);                        // 1 (zeroth) and 1/3 (xx, yy, zz)
        dm.xx -= real(1.0 / 3.0);
        dm.yy -= real(1.0 / 3.0);
        dm.zz -= real(1.0 / 3.0);
        const real inv_rho = real(1) / (real(1) + dm.m0);
        UPow<real> u;
        Raw15<real> D;
        flow_unit<real>(dm, Fx, Fy, Fz, r, inv_rho, u, D);
        populations15<real>(D, f);  // f~ - w_a: the 16-bit forms store it as it is
#pragma unroll
        for (int a = 0; a < 15; ++a) {
            if constexpr (St::deviation) Fout[a * P + c] = store16<S, St::sr_flow, true>(f[a], dither_of(seed, a));
            else Fout[a * P + c] = St::store(f[a] + p.wf[a], real(0));
        }
        if constexpr (Q == 15) {
            thermal15_unit<real>(T, m0, mx, my, mz, u, r, D);
            populations15<real>(D, g);
        } else {
            thermal7_unit<real>(T, m0, mx, my, mz, u, r, g);
        }
        if constexpr (St::deviation) Tout[c] = T;  // the reference of the stored deviations
#pragma unroll
        for (int a = 0; a < Q; ++a) {  // g~ - w^phi_a T: the 16-bit forms' stored value
            if constexpr (St::deviation)
                Gout[a * P + c] = store16<S, St::sr_thermal>(g[a], dither_of(seed, 15 + a));
            else
                Gout[a * P + c] = St::store(fmad(p.wg[a], T, g[a]), real(0));
        }
        return;
    }
    real T = real(0);
#pragma unroll
    for (int a = 0; a < Q; ++a) T += g[a];
    T += real(0.5) * p.heat_source;  // Eq. (25)
    const real Fz = p.ext_fz + p.gbeta * (T - p.T0);
    real ux, uy, uz;
    collide_flow<real>(f, p.ext_fx, p.ext_fy, Fz, p, ux, uy, uz);
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        if constexpr (St::deviation)
            Fout[a * P + c] = store16<S, St::sr_flow, true>(f[a] - p.wf[a], dither_of(seed, a));
        else
            Fout[a * P + c] = St::store_f(f[a], p.wf[a]);
    }
    if constexpr (Q == 15) collide_thermal15<real>(g, ux, uy, uz, p);
    else collide_thermal7<real>(g, ux, uy, uz, p);
    if constexpr (St::deviation) Tout[c] = T;  // collision conserves T: the node's reference
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        real off = real(0);
        if constexpr (St::deviation) off = p.wg[a] * T;
        Gout[a * P + c] = St::store(g[a], off);
    }
}

// ---------------------------------------------------------------------------------
// Cavity node update.  Nodes away from the y and z walls (all but ~4/n of the rows) take
// the interior body, where the only missing links are those through the x faces: one
// select of the load address per link, plus the anti-bounce-back transform of the
// thermal value.  Loads use one base pointer and per-link offsets that are the same for
// every thread.  Nodes touching a y or z wall run the generic pull.  The interior body
// needs boundary == 0 (the cavity) and 15 * plane < 2^31 (32-bit node indices).
// ---------------------------------------------------------------------------------
template <typename S, int Q, bool INTERIOR, bool UNIT = false>
__device__ __forceinline__ void cavity_node(const S* __restrict__ Fin, const S* __restrict__ Gin,
                                            const float* __restrict__ Tin, S* __restrict__ Fout,
                                            S* __restrict__ Gout, float* __restrict__ Tout,
                                            const ParamsOf<S>& p, int i, int j, int k,
                                            uint32_t step = 0) {
    using real = typename Storage<S>::real;
    using St = Storage<S>;
    const int nx = p.nx;
    const int64_t nxy = (int64_t)nx * p.ny;
    const int64_t c = k * nxy + (int64_t)j * nx + i;
    const int64_t P = p.plane;
    real f[15], g[Q];
    if constexpr (INTERIOR) {
        const bool lo = i == 0, hi = i == nx - 1;
        // 32-bit node indices from per-population base pointers (the launcher takes this
        // kernel only when 15 * plane < 2^31); measured 2% faster in FP32 and 19% in FP16
        const int ci = (int)c;
        const int nxi = nx, nxyi = (int)nxy, Pi = (int)P;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int shift = ex(a) + ey(a) * nxi + ez(a) * nxyi;
            const bool out = (ex(a) > 0 && lo) || (ex(a) < 0 && hi);
            const S* Ga = Gin + (int64_t)a * P - shift;
            const int idx = out ? ci + shift + (opp(a) - a) * Pi : ci;
            real off = real(0);
            if constexpr (St::deviation) {
                const float* Ta = Tin - shift;
                off = p.wg[a] * Ta[out ? ci + shift : ci];
            }
            const real v = St::load(Ga[idx], off);
            // Dirichlet face: anti-bounce-back with the face temperature
            const real Tw = ex(a) > 0 ? p.T_cold : p.T_hot;
            g[a] = out ? (real(2) * p.wg[a] * Tw - v) : v;
        }
#pragma unroll
        for (int a = 0; a < 15; ++a) {
            const int shift = ex(a) + ey(a) * nxi + ez(a) * nxyi;
            const bool out = (ex(a) > 0 && lo) || (ex(a) < 0 && hi);
            const S* Fa = Fin + (int64_t)a * P - shift;
            f[a] = St::load_f(Fa[out ? ci + shift + (opp(a) - a) * Pi : ci], p.wf[a]);
        }
    } else {
        pull<S, Q>(Fin, Gin, Tin, p, i, j, k, c, f, g);
    }
    uint32_t seed = 0;
    if constexpr (St::deviation) seed = dither_seed((uint32_t)(p.cell0 + c), step);
    collide_store<S, Q, UNIT>(f, g, Fout, Gout, Tout, p, c, seed);
}

// Blocks per SM the single-precision kernels are built for: 7 for D3Q15 (at most 72
// registers, no spills; measured 1.8% faster than the unconstrained 80 registers at
// 128^3) and 8 for D3Q7 (64 registers).  FP64 is left unconstrained.
template <typename S, int Q>
constexpr int cavity_min_blocks() {
    return sizeof(typename Storage<S>::real) == 8 ? 1 : (Q == 15 ? 7 : 8);
}

}  // namespace lbm
