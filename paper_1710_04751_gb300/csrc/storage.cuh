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
    // flow populations (the 16-bit forms scale their flow deviations, below)
    __host__ __device__ __forceinline__ static real load_f(S v, real) { return v; }
    __host__ __device__ __forceinline__ static S store_f(real x, real) { return x; }
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
// FP16's subnormal range (|x| < 2^-14, which the scaling of the flow deviations below keeps
// clear of) the result is truncated toward zero.  The dither of a node is a 32-bit hash of
// a Weyl value of (global node, step), plus a fixed odd offset per population (dither_of),
// of which the top bits are used: deterministic, the same for a node whatever
// decomposition holds it.  The hash (LBM_DITHER_HASH) is the "lowbias32" integer hash of
// C. Wellons' hash-prospector search (xor-shifts by 16, 15, 16 and two odd multipliers).
// Without it the dither is the Weyl value itself, which is equidistributed over the steps
// of a node but forms a regular lattice over the nodes of a step, a pattern that the
// streaming carries along.
constexpr uint32_t kDitherNodeStep = 0x2C1B3C6Du;
__device__ __forceinline__ uint32_t dither_weyl(uint32_t node, uint32_t step) {
    return node * kDitherNodeStep + step * 0x9E3779B9u;
}
#ifndef LBM_DITHER_HASH
#define LBM_DITHER_HASH 1
#endif
// The seed of a Weyl value: hashed, or the Weyl value itself.
__device__ __forceinline__ uint32_t dither_from_weyl(uint32_t w) {
    if (LBM_DITHER_HASH) {
        w ^= w >> 16;
        w *= 0x7FEB352Du;
        w ^= w >> 15;
        w *= 0x846CA68Bu;
        w ^= w >> 16;
    }
    return w;
}
__device__ __forceinline__ uint32_t dither_seed(uint32_t node, uint32_t step) {
    return dither_from_weyl(dither_weyl(node, step));
}
__device__ __forceinline__ uint32_t dither_of(uint32_t seed, int a) {
    return seed + (uint32_t)a * 0x632BE5ABu;
}

// Which stores of the 16-bit forms round stochastically (the others round to nearest):
// FP16's flow deviations.  Measured against FP32 at the FP32 steady state's step count
// (mid-plane / hot-wall Nu, u_max): FP16 at 128^3, Ra = 1e5: +0.019% / +0.021% / +0.006%;
// at 256^3, Ra = 1e6: -0.15% / -0.17% / -0.55% (to nearest: -0.98% / +0.44% / +15.7%).
// BF16, 8 significant bits, to nearest: +4.5% / +2.9% / +35% at 128^3, +1.9% / +1.0% / +104%
// at 256^3; with stochastic flow stores it is within 0.1% at 48^3 and 128^3 but -2.5% at
// 64^3 (against FP64) and drifts away at 256^3, Ra = 1e6 (-12% / -9% after 288 000 steps,
// still falling): its rounding noise, eight times FP16's, stirs the low-viscosity flow.
// BF16 therefore rounds to nearest, a bias that does not grow.
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

// FP16 stores its flow deviations times 2^LBM_FP16_FLOW_EXP.  The deviations of a cavity
// flow are small (the density and corner-population deviations are a few 1e-5 over much of
// the box), and FP16 is subnormal below 2^-14 = 6.1e-5: there its spacing is a fixed 2^-24,
// so the value keeps few significant bits and the stochastic rounding above degenerates
// into truncation toward zero, a systematic pull of the slow flow toward rest.  Scaling by
// 2^12 moves the subnormal range below 1.5e-8 and caps the stored deviation at
// 65504 / 2^12 = 16, far above any deviation of a stable flow (a larger one, or a
// non-finite one, still reads back as non-finite or saturated and fails the residual
// check).  The scalar deviations are rounded to nearest and left unscaled.
#ifndef LBM_FP16_FLOW_EXP
#define LBM_FP16_FLOW_EXP 12
#endif

template <>
struct Storage<__half> {
    using real = float;
    static constexpr bool deviation = true;
    static constexpr bool sr_flow = LBM_SR_FLOW_FP16, sr_thermal = LBM_SR_THERMAL_FP16;
    static constexpr int flow_exp = LBM_FP16_FLOW_EXP;
    static constexpr float fup = (float)(1u << flow_exp), fdown = 1.f / fup;
    __device__ __forceinline__ static float load(__half v, float off) { return __half2float(v) + off; }
    __device__ __forceinline__ static __half store(float x, float off) { return __float2half_rn(x - off); }
    __device__ __forceinline__ static float load_f(__half v, float off) {
        return fmaf(__half2float(v), fdown, off);
    }
    __device__ __forceinline__ static __half store_f(float x, float off) {
        return __float2half_rn((x - off) * fup);
    }
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
    static constexpr int flow_exp = 0;  // BF16's exponent range needs no scaling
    static constexpr float fup = 1.f, fdown = 1.f;
    __device__ __forceinline__ static float load_f(__nv_bfloat16 v, float off) { return load(v, off); }
    __device__ __forceinline__ static __nv_bfloat16 store_f(float x, float off) { return store(x, off); }
    // x rounded stochastically with the dither taken from the top 16 bits of d
    __device__ __forceinline__ static __nv_bfloat16 store_sr(float x, uint32_t d) {
        return __float2bfloat16_rz(__uint_as_float(__float_as_uint(x) + (d >> 16)));
    }
};

// The 16-bit store of the deviation x: stochastic (dither d) when SR, else to nearest; a
// flow deviation (FLOW) is scaled first.
template <typename S, bool SR, bool FLOW = false>
__device__ __forceinline__ S store16(float x, uint32_t d) {
    if constexpr (FLOW && Storage<S>::flow_exp != 0) x *= Storage<S>::fup;
    if constexpr (SR) return Storage<S>::store_sr(x, d);
    else return Storage<S>::store(x, 0.f);
}

}  // namespace lbm
