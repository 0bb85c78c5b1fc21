// storage.cuh -- how populations are stored in HBM.
//
// FP64 and FP32 store the populations themselves.  The 16-bit forms (FP16, BF16) store
// each population minus its rest-state value -- w_a for the flow, w^phi_a T_node for the
// scalar -- so that the few significant bits of the 16-bit format carry the deviation,
// which is small, rather than the value, which is not.  Arithmetic is FP32 in all three
// single-precision forms: a load adds the offset back in FP32, a store subtracts it in
// FP32 and rounds -- to nearest for the scalar, stochastically for the flow (below).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

template <typename S>
struct Storage {
    using real = S;
    static constexpr bool deviation = false;
    __host__ __device__ __forceinline__ static real load(S v, real) { return v; }
    __host__ __device__ __forceinline__ static S store(real x, real) { return x; }
};

// Stochastic rounding of FP32 values to a 16-bit format (the 16-bit forms' flow stores).
// Rounding to nearest makes the storage error a fixed function of the stored value: in a
// steady state every node stores the same values step after step, so the errors act as a
// constant spurious source and shift the steady state (FP16 at 48^3, Ra = 1e4: +0.5% in
// the mid-plane Nu).  Rounding up with probability equal to the distance to the lower
// neighbour, in units of the spacing, makes the error zero-mean in time instead.  It is
// done on the bit pattern: the discarded low bits of |x| plus a dither d, uniform over the
// discarded range, carry into the kept bits, which are then truncated (round toward
// zero) -- exact for every value whose result is a normal number of the 16-bit format; in
// FP16's subnormal range (|x| < 2^-14) the result is truncated toward zero.  The dither is
// the top bits of a Weyl sequence over (global node, population, step) (dither_of, with
// the golden-ratio step increment 0x9E3779B9): deterministic, the same for a node whatever
// decomposition holds it, and for a fixed node and population equidistributed over the
// steps with low discrepancy.
__device__ __forceinline__ uint32_t dither_seed(uint32_t node, uint32_t step) {
    return node * 0x2C1B3C6Du + step * 0x9E3779B9u;
}
__device__ __forceinline__ uint32_t dither_of(uint32_t seed, int a) {
    return seed + (uint32_t)a * 0x632BE5ABu;
}

// Which stores of the 16-bit forms round stochastically (the others round to nearest).
// Measured on the 48^3, Ra = 1e4 cavity from rest (steady mid-plane / hot-wall Nu against
// FP32): FP16 with stochastic flow stores -0.09% / -0.08% (to nearest: +0.56% / +0.46%);
// BF16, whose 8 significant bits make the stochastic noise itself bias the state, is best
// to nearest in both (+0.32% / +0.56%; stochastic flow -1.18% / -0.91%, both stochastic
// -1.05% / -0.80%, stochastic scalar only +0.46% / +0.71%).
#ifndef LBM_SR_FLOW_FP16
#define LBM_SR_FLOW_FP16 1
#endif
#ifndef LBM_SR_THERMAL_FP16
#define LBM_SR_THERMAL_FP16 0
#endif
#ifndef LBM_SR_FLOW_BF16
#define LBM_SR_FLOW_BF16 0
#endif
#ifndef LBM_SR_THERMAL_BF16
#define LBM_SR_THERMAL_BF16 0
#endif

template <>
struct Storage<__half> {
    using real = float;
    static constexpr bool deviation = true;
    static constexpr bool sr_flow = LBM_SR_FLOW_FP16, sr_thermal = LBM_SR_THERMAL_FP16;
    __device__ __forceinline__ static float load(__half v, float off) { return __half2float(v) + off; }
    __device__ __forceinline__ static __half store(float x, float off) { return __float2half_rn(x - off); }
    // x rounded stochastically with the dither taken from the top 13 bits of d
    __device__ __forceinline__ static __half store_sr(float x, uint32_t d) {
        return __float2half_rz(__uint_as_float(__float_as_uint(x) + (d >> 19)));
    }
};

template <>
struct Storage<__nv_bfloat16> {
    using real = float;
    static constexpr bool deviation = true;
    static constexpr bool sr_flow = LBM_SR_FLOW_BF16, sr_thermal = LBM_SR_THERMAL_BF16;
    __device__ __forceinline__ static float load(__nv_bfloat16 v, float off) {
        return __bfloat162float(v) + off;
    }
    __device__ __forceinline__ static __nv_bfloat16 store(float x, float off) {
        return __float2bfloat16_rn(x - off);
    }
    // x rounded stochastically with the dither taken from the top 16 bits of d
    __device__ __forceinline__ static __nv_bfloat16 store_sr(float x, uint32_t d) {
        return __float2bfloat16_rz(__uint_as_float(__float_as_uint(x) + (d >> 16)));
    }
};

// The 16-bit store of x: stochastic (dither d) when SR, else to nearest.
template <typename S, bool SR>
__device__ __forceinline__ S store16(float x, uint32_t d) {
    if constexpr (SR) return Storage<S>::store_sr(x, d);
    else return Storage<S>::store(x, 0.f);
}

}  // namespace lbm
