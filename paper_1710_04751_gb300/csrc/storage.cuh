// storage.cuh -- how populations are stored in HBM.
//
// FP64 and FP32 store the populations themselves.  The 16-bit forms (FP16, BF16) store
// each population minus its rest-state value -- w_a for the flow, w^phi_a T0 for the
// scalar -- so that the few significant bits of the 16-bit format carry the deviation,
// which is small, rather than the value, which is not.  Arithmetic is FP32 in all three
// single-precision forms: a load adds the offset back in FP32, a store subtracts it in
// FP32 and rounds to nearest.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace lbm {

template <typename S>
struct Storage {
    using real = S;
    static constexpr bool deviation = false;
    __host__ __device__ __forceinline__ static real load(S v, real) { return v; }
    __host__ __device__ __forceinline__ static S store(real x, real) { return x; }
};

template <>
struct Storage<__half> {
    using real = float;
    static constexpr bool deviation = true;
    __device__ __forceinline__ static float load(__half v, float off) { return __half2float(v) + off; }
    __device__ __forceinline__ static __half store(float x, float off) { return __float2half_rn(x - off); }
};

template <>
struct Storage<__nv_bfloat16> {
    using real = float;
    static constexpr bool deviation = true;
    __device__ __forceinline__ static float load(__nv_bfloat16 v, float off) {
        return __bfloat162float(v) + off;
    }
    __device__ __forceinline__ static __nv_bfloat16 store(float x, float off) {
        return __float2bfloat16_rn(x - off);
    }
};

}  // namespace lbm
