// pair.cuh -- the fused stream-and-collide update of two x-neighbouring nodes at once,
// for the 16-bit storage forms (FP16 / BF16 deviations from the rest state, FP32
// arithmetic), with packed FP32 pair arithmetic (add / sub / mul / fma on .f32x2, one
// instruction for both lanes on the sm_100 family).
//
// It computes what node.cuh computes for each of the two nodes -- pull (Eqs. 2b, 13b)
// with the x-face rules of Sec. 3, T (Eq. 25), the Boussinesq force, u (Eq. 3), the flow
// collision of App. A and the scalar collision of Sec. 2.2 / App. C in central moments
// (collide.cuh's increments, or the lean form below), the store of both populations'
// deviations -- with about 40% fewer instructions per node (713 against ~1150 measured for
// the one-node 16-bit update): every floating-point operation covers two nodes, the
// populations of the x-aligned links (e_x = 0) and every store move two 16-bit values in
// one 32-bit access, and the node temperatures of a source row come as one aligned
// float2 plus the two x-neighbours.  Lane .x is node i = 2t, lane .y is node 2t + 1.
//
// Used for rows away from the y and z walls of the cavity with an even nx (the pair
// (2t, 2t+1) then starts at an even node index, so the 32-bit and 64-bit accesses are
// aligned); the kernel falls back to node.cuh's update for the other rows.  At the paper's
// unit higher-order rates the update is pair_node_unit (collide_unit.cuh), for FP16 D3Q15
// with every load issued ahead of the arithmetic (pair_node_unit_early).  The `seed` of a
// pair is the Weyl value of its first node (dither_weyl of the global node index and the
// step); the stores hash it into each node's rounding dither (storage.cuh), the same
// dither node.cuh draws for the node.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "collide.cuh"
#include "collide_unit.cuh"
#include "internal.h"
#include "lattice.cuh"

// Which form of the two-node update each scalar lattice uses: the lean form (moments of
// the deviations, pair_collide_store_lean) or the increment form (pair_collide_store).
// Measured at 128^3 and 256^3 (FP16): lean is faster for D3Q15 (0.0825 / 0.511 ms against
// 0.0863 / 0.540 ms per step), the increment form for D3Q7 (0.0533 against 0.0552 ms).
#ifndef LBM_PAIR_LEAN_Q15
#define LBM_PAIR_LEAN_Q15 1
#endif
#ifndef LBM_PAIR_LEAN_Q7
#define LBM_PAIR_LEAN_Q7 0
#endif

namespace lbm {

// ---------------------------------------------------------------------------------
// packed FP32 pairs, round to nearest: each lane is rounded as the scalar operation
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 o;
    asm("{\n\t.reg .b64 x, y, r;\n\t"
        "mov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\t"
        "sub.rn.f32x2 r, x, y;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(o.x), "=f"(o.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return o;
}
__device__ __forceinline__ float2 neg2(float2 a) { return sub2(make_float2(0.f, 0.f), a); }

// Two adjacent 16-bit values as one 32-bit word.
template <typename S>
struct Pack;
template <>
struct Pack<__half> {
    using two = __half2;
    __device__ __forceinline__ static float2 to_float2(two v) { return __half22float2(v); }
    __device__ __forceinline__ static two from_float2(float2 v) { return __float22half2_rn(v); }
    __device__ __forceinline__ static float to_float(__half v) { return __half2float(v); }
    // both lanes rounded stochastically (storage.cuh), lane .x with dither dx, .y with dy
    __device__ __forceinline__ static two from_float2_sr(float2 v, uint32_t dx, uint32_t dy) {
        return __halves2half2(Storage<__half>::store_sr(v.x, dx), Storage<__half>::store_sr(v.y, dy));
    }
    template <bool SR>
    __device__ __forceinline__ static two store2(float2 v, uint32_t dx, uint32_t dy) {
        if constexpr (SR) return from_float2_sr(v, dx, dy);
        else return from_float2(v);
    }
    // from raw bits: a 32-bit word holding two values, or two 16-bit values
    __device__ __forceinline__ static float2 word2(uint32_t w) {
        return __half22float2(__halves2half2(__ushort_as_half((unsigned short)(w & 0xFFFFu)),
                                             __ushort_as_half((unsigned short)(w >> 16))));
    }
    __device__ __forceinline__ static float2 bits2(unsigned short x, unsigned short y) {
        return make_float2(__half2float(__ushort_as_half(x)), __half2float(__ushort_as_half(y)));
    }
    // flow deviations: stored times 2^flow_exp (storage.cuh)
    static constexpr float up = Storage<__half>::fup, down = Storage<__half>::fdown;
    __device__ __forceinline__ static float2 flow2(two v) {
        return mul2(__half22float2(v), make_float2(down, down));
    }
    __device__ __forceinline__ static float2 flow2(__half x, __half y) {
        return mul2(make_float2(__half2float(x), __half2float(y)), make_float2(down, down));
    }
    template <bool SR>
    __device__ __forceinline__ static two store2f(float2 v, uint32_t dx, uint32_t dy) {
        return store2<SR>(mul2(v, make_float2(up, up)), dx, dy);
    }
};
template <>
struct Pack<__nv_bfloat16> {
    using two = __nv_bfloat162;
    __device__ __forceinline__ static float2 to_float2(two v) { return __bfloat1622float2(v); }
    __device__ __forceinline__ static two from_float2(float2 v) { return __float22bfloat162_rn(v); }
    __device__ __forceinline__ static float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ __forceinline__ static two from_float2_sr(float2 v, uint32_t dx, uint32_t dy) {
        return __halves2bfloat162(Storage<__nv_bfloat16>::store_sr(v.x, dx),
                                  Storage<__nv_bfloat16>::store_sr(v.y, dy));
    }
    template <bool SR>
    __device__ __forceinline__ static two store2(float2 v, uint32_t dx, uint32_t dy) {
        if constexpr (SR) return from_float2_sr(v, dx, dy);
        else return from_float2(v);
    }
    __device__ __forceinline__ static float2 word2(uint32_t w) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
    }
    __device__ __forceinline__ static float2 bits2(unsigned short x, unsigned short y) {
        return make_float2(__uint_as_float((uint32_t)x << 16), __uint_as_float((uint32_t)y << 16));
    }
    static constexpr float up = 1.f, down = 1.f;
    // flow deviations: stored as they are
    __device__ __forceinline__ static float2 flow2(two v) { return to_float2(v); }
    __device__ __forceinline__ static float2 flow2(__nv_bfloat16 x, __nv_bfloat16 y) {
        return make_float2(to_float(x), to_float(y));
    }
    template <bool SR>
    __device__ __forceinline__ static two store2f(float2 v, uint32_t dx, uint32_t dy) {
        return store2<SR>(v, dx, dy);
    }
};


// Two lanes of FP32 as one arithmetic value (the unit-rate collisions of
// collide_unit.cuh are templates over it): every operator is one packed instruction.
struct Pair {
    float2 v;
};
__device__ __forceinline__ Pair operator+(Pair a, Pair b) { return {add2(a.v, b.v)}; }
__device__ __forceinline__ Pair operator-(Pair a, Pair b) { return {sub2(a.v, b.v)}; }
__device__ __forceinline__ Pair operator*(Pair a, Pair b) { return {mul2(a.v, b.v)}; }
__device__ __forceinline__ Pair& operator+=(Pair& a, Pair b) { a = a + b; return a; }
__device__ __forceinline__ Pair& operator-=(Pair& a, Pair b) { a = a - b; return a; }
__device__ __forceinline__ Pair fmad(Pair a, Pair b, Pair c) { return {fma2(a.v, b.v, c.v)}; }
template <>
__device__ __forceinline__ Pair cst<Pair>(double v) {
    return {make_float2((float)v, (float)v)};
}

// Parameters of the pair update, each broadcast to both lanes (host: make_pair_params).
struct PairParams {
    float2 wf[15];     // flow rest values w_a: the offsets of the stored flow deviations
    float2 wg[15];     // thermal rest weights w^phi_a
    float2 nwg[15];    // -w^phi_a
    float wTc2[15];    // 2 w^phi_a T_cold: anti-bounce-back at the cold face (i = 0)
    float wTh2[15];    // 2 w^phi_a T_hot: anti-bounce-back at the hot face (i = nx - 1)
    float2 nomf[15];   // -omega_b of the flow moments
    float2 omf9;       // omega_9 (bulk): relaxes the trace toward 3 c_s^2 rho
    float2 omf14;      // omega_14: relaxes xxyy toward its equilibrium E
    float2 cf3[3];     // (1 - omega_b) c_s^2, b = 10, 11, 12: third-order source moments
    float2 nomg[15];   // -omega_b of the scalar moments
    float2 omg_tr;     // omega of the trace (b = 9, or 6 for D3Q7) times 3 c_sphi^2
    float2 omg_4;      // omega_14 c_sphi^4 (D3Q15)
    float2 cs2, cs4;   // c_sphi^2, c_sphi^4: moments of the scalar rest weights
    float2 R, halfR;   // uniform source R (Eq. 4) and R/2 (Eq. 25)
    float2 gbeta, T0;  // Boussinesq force gbeta (T - T0)
    float2 fx, fy, fz; // uniform body force
    float2 halffx, halffy;
    int e4_mode;
    UnitRates<Pair> ur; // the rates of the unit-rate update (pair_node_unit)
};

// Powers of one velocity (lane-wise) that the binomial shifts need.
struct Vel2 {
    float2 x, y, z, x2, y2, z2;             // v, 2v
    float2 xx, yy, zz, xy, xz, yz;          // second order
    float2 xy2, xz2, xy4;                   // 2 v_x v_y, 2 v_x v_z, 4 v_x v_y
    float2 xyy, xxy, xxz, xyz, xyy2, xxy2;  // third order (and doubled)
    float2 xxyy;
};

__device__ __forceinline__ Vel2 vel2(float2 x, float2 y, float2 z) {
    Vel2 v;
    v.x = x; v.y = y; v.z = z;
    v.x2 = add2(x, x); v.y2 = add2(y, y); v.z2 = add2(z, z);
    v.xx = mul2(x, x); v.yy = mul2(y, y); v.zz = mul2(z, z);
    v.xy = mul2(x, y); v.xz = mul2(x, z); v.yz = mul2(y, z);
    v.xy2 = add2(v.xy, v.xy); v.xz2 = add2(v.xz, v.xz); v.xy4 = add2(v.xy2, v.xy2);
    v.xyy = mul2(x, v.yy); v.xxy = mul2(v.xx, y); v.xxz = mul2(v.xx, z); v.xyz = mul2(v.xy, z);
    v.xyy2 = add2(v.xyy, v.xyy); v.xxy2 = add2(v.xxy, v.xxy);
    v.xxyy = mul2(v.xx, v.yy);
    return v;
}

// The powers of -v from those of v: the odd ones change sign.
__device__ __forceinline__ Vel2 vel2_negated(const Vel2& v) {
    Vel2 n = v;
    n.x = neg2(v.x); n.y = neg2(v.y); n.z = neg2(v.z);
    n.x2 = neg2(v.x2); n.y2 = neg2(v.y2); n.z2 = neg2(v.z2);
    n.xyy = neg2(v.xyy); n.xxy = neg2(v.xxy); n.xxz = neg2(v.xxz); n.xyz = neg2(v.xyz);
    n.xyy2 = neg2(v.xyy2); n.xxy2 = neg2(v.xxy2);
    return n;
}

// Raw moments of a D3Q15 pair of population vectors (the sign transform of raw15).
__device__ __forceinline__ Raw15<float2> raw15_2(const float2 (&p)[15]) {
    const float2 a0 = add2(p[7], p[8]), b0 = sub2(p[7], p[8]);
    const float2 a1 = add2(p[9], p[10]), b1 = sub2(p[9], p[10]);
    const float2 a2 = add2(p[11], p[12]), b2 = sub2(p[11], p[12]);
    const float2 a3 = add2(p[13], p[14]), b3 = sub2(p[13], p[14]);
    const float2 c0 = add2(a0, a1), c1 = sub2(a0, a1), c2 = add2(a2, a3), c3 = sub2(a2, a3);
    const float2 e0 = add2(b0, b1), e1 = sub2(b0, b1), e2 = add2(b2, b3), e3 = sub2(b2, b3);
    const float2 H0 = add2(c0, c2), Hz = sub2(c0, c2), Hy = add2(c1, c3), Hyz = sub2(c1, c3);
    const float2 Hx = add2(e0, e2), Hxz = sub2(e0, e2), Hxy = add2(e1, e3), Hxyz = sub2(e1, e3);
    const float2 px = add2(p[1], p[2]), qx = sub2(p[1], p[2]);
    const float2 py = add2(p[3], p[4]), qy = sub2(p[3], p[4]);
    const float2 pz = add2(p[5], p[6]), qz = sub2(p[5], p[6]);
    Raw15<float2> m;
    m.m0 = add2(add2(add2(add2(p[0], px), py), pz), H0);
    m.x = add2(qx, Hx);
    m.y = add2(qy, Hy);
    m.z = add2(qz, Hz);
    m.xy = Hxy;
    m.xz = Hxz;
    m.yz = Hyz;
    m.xx = add2(px, H0);
    m.yy = add2(py, H0);
    m.zz = add2(pz, H0);
    m.xyy = Hx;
    m.xxy = Hy;
    m.xxz = Hz;
    m.xyz = Hxyz;
    m.xxyy = H0;
    return m;
}

// Moments about a point moved by v (binomial theorem): with v = -u the central moments
// of raw moments m (Eq. 14); with v = +u the raw moments of central moments m (the
// inverse shift).  D0 = false drops the terms of the zeroth moment (taken as zero).
template <bool D0>
__device__ __forceinline__ Raw15<float2> shift15_2(const Raw15<float2>& m, const Vel2& v) {
    Raw15<float2> c;
    c.m0 = m.m0;
    c.x = m.x;
    c.y = m.y;
    c.z = m.z;
    c.xy = fma2(v.x, m.y, fma2(v.y, m.x, m.xy));
    c.xz = fma2(v.x, m.z, fma2(v.z, m.x, m.xz));
    c.yz = fma2(v.y, m.z, fma2(v.z, m.y, m.yz));
    c.xx = fma2(v.x2, m.x, m.xx);
    c.yy = fma2(v.y2, m.y, m.yy);
    c.zz = fma2(v.z2, m.z, m.zz);
    c.xyy = fma2(v.xy2, m.y, fma2(v.yy, m.x, fma2(v.x, m.yy, fma2(v.y2, m.xy, m.xyy))));
    c.xxy = fma2(v.xy2, m.x, fma2(v.xx, m.y, fma2(v.y, m.xx, fma2(v.x2, m.xy, m.xxy))));
    c.xxz = fma2(v.xz2, m.x, fma2(v.xx, m.z, fma2(v.z, m.xx, fma2(v.x2, m.xz, m.xxz))));
    c.xyz = fma2(v.yz, m.x,
                 fma2(v.xz, m.y, fma2(v.xy, m.z, fma2(v.z, m.xy, fma2(v.y, m.xz, fma2(v.x, m.yz, m.xyz))))));
    c.xxyy = fma2(v.xxy2, m.y,
                  fma2(v.xyy2, m.x,
                       fma2(v.xy4, m.xy,
                            fma2(v.xx, m.yy, fma2(v.yy, m.xx, fma2(v.x2, m.xyy, fma2(v.y2, m.xxy, m.xxyy)))))));
    if constexpr (D0) {
        const float2 m0 = m.m0;
        c.x = fma2(v.x, m0, c.x);
        c.y = fma2(v.y, m0, c.y);
        c.z = fma2(v.z, m0, c.z);
        c.xy = fma2(v.xy, m0, c.xy);
        c.xz = fma2(v.xz, m0, c.xz);
        c.yz = fma2(v.yz, m0, c.yz);
        c.xx = fma2(v.xx, m0, c.xx);
        c.yy = fma2(v.yy, m0, c.yy);
        c.zz = fma2(v.zz, m0, c.zz);
        c.xyy = fma2(v.xyy, m0, c.xyy);
        c.xxy = fma2(v.xxy, m0, c.xxy);
        c.xxz = fma2(v.xxz, m0, c.xxz);
        c.xyz = fma2(v.xyz, m0, c.xyz);
        c.xxyy = fma2(v.xxyy, m0, c.xxyy);
    }
    return c;
}

// p += the populations whose raw moments are r (inverse of raw15_2).
__device__ __forceinline__ void add_populations15_2(float2 (&p)[15], const Raw15<float2>& r) {
    const float2 G0 = r.xxyy, Gx = r.xyy, Gy = r.xxy, Gz = r.xxz;
    const float2 P0 = add2(G0, Gz), P0m = sub2(G0, Gz), Px = add2(Gx, r.xz), Pxm = sub2(Gx, r.xz);
    const float2 Py = add2(Gy, r.yz), Pym = sub2(Gy, r.yz);
    const float2 Pxy = add2(r.xy, r.xyz), Pxym = sub2(r.xy, r.xyz);
    const float2 Q0 = add2(P0, Py), Q1 = sub2(P0, Py), X0 = add2(Px, Pxy), X1 = sub2(Px, Pxy);
    const float2 Q2 = add2(P0m, Pym), Q3 = sub2(P0m, Pym), X2 = add2(Pxm, Pxym), X3 = sub2(Pxm, Pxym);
    const float2 e = make_float2(0.125f, 0.125f), h = make_float2(0.5f, 0.5f);
    p[7] = fma2(e, add2(Q0, X0), p[7]);
    p[8] = fma2(e, sub2(Q0, X0), p[8]);
    p[9] = fma2(e, add2(Q1, X1), p[9]);
    p[10] = fma2(e, sub2(Q1, X1), p[10]);
    p[11] = fma2(e, add2(Q2, X2), p[11]);
    p[12] = fma2(e, sub2(Q2, X2), p[12]);
    p[13] = fma2(e, add2(Q3, X3), p[13]);
    p[14] = fma2(e, sub2(Q3, X3), p[14]);
    const float2 px = sub2(r.xx, G0), qx = sub2(r.x, Gx);
    const float2 py = sub2(r.yy, G0), qy = sub2(r.y, Gy);
    const float2 pz = sub2(r.zz, G0), qz = sub2(r.z, Gz);
    p[1] = fma2(h, add2(px, qx), p[1]);
    p[2] = fma2(h, sub2(px, qx), p[2]);
    p[3] = fma2(h, add2(py, qy), p[3]);
    p[4] = fma2(h, sub2(py, qy), p[4]);
    p[5] = fma2(h, add2(pz, qz), p[5]);
    p[6] = fma2(h, sub2(pz, qz), p[6]);
    p[0] = add2(p[0], sub2(sub2(sub2(sub2(r.m0, px), py), pz), G0));
}

// Second-order increments from the relaxed combinations xx-yy, xx+yy-2zz, xx+yy+zz.
__device__ __forceinline__ void split_second_order2(float2 d1, float2 d2, float2 dtr, float2& dxx,
                                                    float2& dyy, float2& dzz) {
    dzz = mul2(sub2(dtr, d2), make_float2(1.0f / 3.0f, 1.0f / 3.0f));
    const float2 s = sub2(dtr, dzz);
    const float2 h = make_float2(0.5f, 0.5f);
    dxx = mul2(h, add2(s, d1));
    dyy = mul2(h, sub2(s, d1));
}

// Flow collision of App. A for a pair (collide_flow's increments): f becomes f~; the
// velocity powers of u are returned for the scalar collision.
__device__ __forceinline__ void collide_flow2(float2 (&f)[15], float2 Fz, const PairParams& q,
                                              Vel2& vu) {
    const Raw15<float2> m = raw15_2(f);
    const float2 rho = m.m0;
    const float2 inv_rho = make_float2(1.0f / rho.x, 1.0f / rho.y);
    const float2 ux = mul2(add2(m.x, q.halffx), inv_rho);
    const float2 uy = mul2(add2(m.y, q.halffy), inv_rho);
    const float2 uz = mul2(fma2(make_float2(0.5f, 0.5f), Fz, m.z), inv_rho);
    vu = vel2(ux, uy, uz);
    const Raw15<float2> k = shift15_2<true>(m, vel2_negated(vu));
    Raw15<float2> d;
    d.m0 = make_float2(0.f, 0.f);
    d.x = q.fx;
    d.y = q.fy;
    d.z = Fz;
    d.xy = mul2(q.nomf[4], k.xy);
    d.xz = mul2(q.nomf[5], k.xz);
    d.yz = mul2(q.nomf[6], k.yz);
    const float2 sxy = add2(k.xx, k.yy);
    const float2 d1 = mul2(q.nomf[7], sub2(k.xx, k.yy));
    const float2 d2 = mul2(q.nomf[8], fma2(make_float2(-2.f, -2.f), k.zz, sxy));
    const float2 tr = add2(sxy, k.zz);
    const float2 dtr = fma2(q.omf9, rho, mul2(q.nomf[9], tr));  // equilibrium trace 3 c_s^2 rho
    split_second_order2(d1, d2, dtr, d.xx, d.yy, d.zz);
    d.xyy = fma2(q.nomf[10], k.xyy, mul2(q.cf3[0], q.fx));
    d.xxy = fma2(q.nomf[11], k.xxy, mul2(q.cf3[1], q.fy));
    d.xxz = fma2(q.nomf[12], k.xxz, mul2(q.cf3[2], Fz));
    d.xyz = mul2(q.nomf[13], k.xyz);
    const float2 E = q.e4_mode == 1 ? mul2(rho, make_float2(1.0f / 9.0f, 1.0f / 9.0f))
                                    : mul2(mul2(add2(k.xx, d.xx), add2(k.yy, d.yy)), inv_rho);
    d.xxyy = fma2(q.omf14, E, mul2(q.nomf[14], k.xxyy));
    add_populations15_2(f, shift15_2<false>(d, vu));
}

// Scalar D3Q15 collision of Sec. 2.2 for a pair (collide_thermal15's increments).
__device__ __forceinline__ void collide_thermal15_2(float2 (&g)[15], const Vel2& vu,
                                                    const PairParams& q) {
    const Raw15<float2> m = raw15_2(g);
    const float2 phi = add2(m.m0, q.halfR);
    const Raw15<float2> k = shift15_2<true>(m, vel2_negated(vu));
    Raw15<float2> d;
    d.m0 = q.R;
    d.x = mul2(q.nomg[1], k.x);
    d.y = mul2(q.nomg[2], k.y);
    d.z = mul2(q.nomg[3], k.z);
    d.xy = mul2(q.nomg[4], k.xy);
    d.xz = mul2(q.nomg[5], k.xz);
    d.yz = mul2(q.nomg[6], k.yz);
    const float2 sxy = add2(k.xx, k.yy);
    const float2 d1 = mul2(q.nomg[7], sub2(k.xx, k.yy));
    const float2 d2 = mul2(q.nomg[8], fma2(make_float2(-2.f, -2.f), k.zz, sxy));
    const float2 tr = add2(sxy, k.zz);
    const float2 dtr = fma2(q.omg_tr, phi, mul2(q.nomg[9], tr));
    split_second_order2(d1, d2, dtr, d.xx, d.yy, d.zz);
    d.xyy = mul2(q.nomg[10], k.xyy);
    d.xxy = mul2(q.nomg[11], k.xxy);
    d.xxz = mul2(q.nomg[12], k.xxz);
    d.xyz = mul2(q.nomg[13], k.xyz);
    d.xxyy = fma2(q.omg_4, phi, mul2(q.nomg[14], k.xxyy));
    add_populations15_2(g, shift15_2<true>(d, vu));
}

// Scalar D3Q7 collision of App. C for a pair (collide_thermal7's increments).
__device__ __forceinline__ void collide_thermal7_2(float2 (&g)[7], const Vel2& v,
                                                   const PairParams& q) {
    const float2 px = add2(g[1], g[2]), qx = sub2(g[1], g[2]);
    const float2 py = add2(g[3], g[4]), qy = sub2(g[3], g[4]);
    const float2 pz = add2(g[5], g[6]), qz = sub2(g[5], g[6]);
    const float2 m0 = add2(add2(add2(g[0], px), py), pz);
    const float2 phi = add2(m0, q.halfR);
    // central moments about u: shift by -u
    const float2 kx = fma2(neg2(v.x), m0, qx), ky = fma2(neg2(v.y), m0, qy), kz = fma2(neg2(v.z), m0, qz);
    const float2 kxx = fma2(v.xx, m0, fma2(neg2(v.x2), qx, px));
    const float2 kyy = fma2(v.yy, m0, fma2(neg2(v.y2), qy, py));
    const float2 kzz = fma2(v.zz, m0, fma2(neg2(v.z2), qz, pz));
    const float2 dx = mul2(q.nomg[1], kx), dy = mul2(q.nomg[2], ky), dz = mul2(q.nomg[3], kz);
    const float2 sxy = add2(kxx, kyy);
    const float2 d1 = mul2(q.nomg[4], sub2(kxx, kyy));
    const float2 d2 = mul2(q.nomg[5], fma2(make_float2(-2.f, -2.f), kzz, sxy));
    const float2 dtr = fma2(q.omg_tr, phi, mul2(q.nomg[6], add2(sxy, kzz)));
    float2 dxx, dyy, dzz;
    split_second_order2(d1, d2, dtr, dxx, dyy, dzz);
    // raw increments (zeroth: R) and populations
    const float2 R = q.R;
    const float2 rx = fma2(v.x, R, dx), ry = fma2(v.y, R, dy), rz = fma2(v.z, R, dz);
    const float2 rxx = fma2(v.xx, R, fma2(v.x2, dx, dxx));
    const float2 ryy = fma2(v.yy, R, fma2(v.y2, dy, dyy));
    const float2 rzz = fma2(v.zz, R, fma2(v.z2, dz, dzz));
    const float2 h = make_float2(0.5f, 0.5f);
    g[1] = fma2(h, add2(rxx, rx), g[1]);
    g[2] = fma2(h, sub2(rxx, rx), g[2]);
    g[3] = fma2(h, add2(ryy, ry), g[3]);
    g[4] = fma2(h, sub2(ryy, ry), g[4]);
    g[5] = fma2(h, add2(rzz, rz), g[5]);
    g[6] = fma2(h, sub2(rzz, rz), g[6]);
    g[0] = add2(g[0], sub2(R, add2(add2(rxx, ryy), rzz)));
}

// T (Eq. 25), the Boussinesq force, both collisions and the store of the pair of nodes
// c0, c0 + 1 (their 16-bit deviations and the FP32 node temperature).
template <typename S, int Q>
__device__ __forceinline__ void pair_collide_store(float2 (&f)[15], float2 (&g)[Q],
                                                   S* __restrict__ Fout, S* __restrict__ Gout,
                                                   float* __restrict__ Tout, const PairParams& q,
                                                   int P, int c0, uint32_t seed) {
    using Pk = Pack<S>;
    using two = typename Pk::two;
    float2 T = g[0];
#pragma unroll
    for (int a = 1; a < Q; ++a) T = add2(T, g[a]);
    T = add2(T, q.halfR);
    const float2 Fz = fma2(q.gbeta, sub2(T, q.T0), q.fz);
    Vel2 vu;
    collide_flow2(f, Fz, q, vu);
    const uint32_t seed0 = dither_from_weyl(seed), seed1 = dither_from_weyl(seed + kDitherNodeStep);
#pragma unroll
    for (int a = 0; a < 15; ++a)
        *reinterpret_cast<two*>(Fout + a * P + c0) =
            Pk::template store2f<Storage<S>::sr_flow>(sub2(f[a], q.wf[a]), dither_of(seed0, a),
                                                     dither_of(seed1, a));
    if constexpr (Q == 15) collide_thermal15_2(g, vu, q);
    else collide_thermal7_2(g, vu, q);
    // the collision conserves T: it is the reference of this node's stored deviations
    *reinterpret_cast<float2*>(Tout + c0) = T;
#pragma unroll
    for (int a = 0; a < Q; ++a)
        *reinterpret_cast<two*>(Gout + a * P + c0) = Pk::from_float2(fma2(q.nwg[a], T, g[a]));
}


// ---------------------------------------------------------------------------------
// Lean form of pair_collide_store (LBM_PAIR_LEAN_Q15 / _Q7): the post-collision populations
// are formed from post-collision raw moments (moments + raw increment) instead of being
// added to the pulled populations, so a pulled vector is dead once its raw moments are
// taken; the scalar collision runs before the flow collision.  Same state up to rounding.
// ---------------------------------------------------------------------------------

// The populations whose raw moments are r (the inverse of raw15_2).
__device__ __forceinline__ void populations15_2(const Raw15<float2>& r, float2 (&p)[15]) {
    const float2 G0 = r.xxyy, Gx = r.xyy, Gy = r.xxy, Gz = r.xxz;
    const float2 P0 = add2(G0, Gz), P0m = sub2(G0, Gz), Px = add2(Gx, r.xz), Pxm = sub2(Gx, r.xz);
    const float2 Py = add2(Gy, r.yz), Pym = sub2(Gy, r.yz);
    const float2 Pxy = add2(r.xy, r.xyz), Pxym = sub2(r.xy, r.xyz);
    const float2 Q0 = add2(P0, Py), Q1 = sub2(P0, Py), X0 = add2(Px, Pxy), X1 = sub2(Px, Pxy);
    const float2 Q2 = add2(P0m, Pym), Q3 = sub2(P0m, Pym), X2 = add2(Pxm, Pxym), X3 = sub2(Pxm, Pxym);
    const float2 e = make_float2(0.125f, 0.125f), h = make_float2(0.5f, 0.5f);
    p[7] = mul2(e, add2(Q0, X0));
    p[8] = mul2(e, sub2(Q0, X0));
    p[9] = mul2(e, add2(Q1, X1));
    p[10] = mul2(e, sub2(Q1, X1));
    p[11] = mul2(e, add2(Q2, X2));
    p[12] = mul2(e, sub2(Q2, X2));
    p[13] = mul2(e, add2(Q3, X3));
    p[14] = mul2(e, sub2(Q3, X3));
    const float2 px = sub2(r.xx, G0), qx = sub2(r.x, Gx);
    const float2 py = sub2(r.yy, G0), qy = sub2(r.y, Gy);
    const float2 pz = sub2(r.zz, G0), qz = sub2(r.z, Gz);
    p[1] = mul2(h, add2(px, qx));
    p[2] = mul2(h, sub2(px, qx));
    p[3] = mul2(h, add2(py, qy));
    p[4] = mul2(h, sub2(py, qy));
    p[5] = mul2(h, add2(pz, qz));
    p[6] = mul2(h, sub2(pz, qz));
    p[0] = sub2(sub2(sub2(sub2(r.m0, px), py), pz), G0);
}

__device__ __forceinline__ Raw15<float2> add15_2(const Raw15<float2>& a, const Raw15<float2>& b) {
    Raw15<float2> c;
    c.m0 = add2(a.m0, b.m0); c.x = add2(a.x, b.x); c.y = add2(a.y, b.y); c.z = add2(a.z, b.z);
    c.xy = add2(a.xy, b.xy); c.xz = add2(a.xz, b.xz); c.yz = add2(a.yz, b.yz);
    c.xx = add2(a.xx, b.xx); c.yy = add2(a.yy, b.yy); c.zz = add2(a.zz, b.zz);
    c.xyy = add2(a.xyy, b.xyy); c.xxy = add2(a.xxy, b.xxy); c.xxz = add2(a.xxz, b.xxz);
    c.xyz = add2(a.xyz, b.xyz); c.xxyy = add2(a.xxyy, b.xxyy);
    return c;
}

// Flow increments in raw moments (collide_flow2's d, shifted back by u).
__device__ __forceinline__ Raw15<float2> flow_increment2(const Raw15<float2>& m, float2 inv_rho,
                                                         float2 Fz, const PairParams& q,
                                                         const Vel2& vu) {
    const float2 rho = m.m0;
    const Raw15<float2> k = shift15_2<true>(m, vel2_negated(vu));
    Raw15<float2> d;
    d.m0 = make_float2(0.f, 0.f);
    d.x = q.fx;
    d.y = q.fy;
    d.z = Fz;
    d.xy = mul2(q.nomf[4], k.xy);
    d.xz = mul2(q.nomf[5], k.xz);
    d.yz = mul2(q.nomf[6], k.yz);
    const float2 sxy = add2(k.xx, k.yy);
    const float2 d1 = mul2(q.nomf[7], sub2(k.xx, k.yy));
    const float2 d2 = mul2(q.nomf[8], fma2(make_float2(-2.f, -2.f), k.zz, sxy));
    const float2 dtr = fma2(q.omf9, rho, mul2(q.nomf[9], add2(sxy, k.zz)));
    split_second_order2(d1, d2, dtr, d.xx, d.yy, d.zz);
    d.xyy = fma2(q.nomf[10], k.xyy, mul2(q.cf3[0], q.fx));
    d.xxy = fma2(q.nomf[11], k.xxy, mul2(q.cf3[1], q.fy));
    d.xxz = fma2(q.nomf[12], k.xxz, mul2(q.cf3[2], Fz));
    d.xyz = mul2(q.nomf[13], k.xyz);
    const float2 E = q.e4_mode == 1 ? mul2(rho, make_float2(1.0f / 9.0f, 1.0f / 9.0f))
                                    : mul2(mul2(add2(k.xx, d.xx), add2(k.yy, d.yy)), inv_rho);
    d.xxyy = fma2(q.omf14, E, mul2(q.nomf[14], k.xxyy));
    return shift15_2<false>(d, vu);
}

// Scalar D3Q15 increments in raw moments (collide_thermal15_2's d, shifted back by u).
__device__ __forceinline__ Raw15<float2> thermal15_increment2(const Raw15<float2>& m, const Vel2& vu,
                                                              const PairParams& q) {
    const float2 phi = add2(m.m0, q.halfR);
    const Raw15<float2> k = shift15_2<true>(m, vel2_negated(vu));
    Raw15<float2> d;
    d.m0 = q.R;
    d.x = mul2(q.nomg[1], k.x);
    d.y = mul2(q.nomg[2], k.y);
    d.z = mul2(q.nomg[3], k.z);
    d.xy = mul2(q.nomg[4], k.xy);
    d.xz = mul2(q.nomg[5], k.xz);
    d.yz = mul2(q.nomg[6], k.yz);
    const float2 sxy = add2(k.xx, k.yy);
    const float2 d1 = mul2(q.nomg[7], sub2(k.xx, k.yy));
    const float2 d2 = mul2(q.nomg[8], fma2(make_float2(-2.f, -2.f), k.zz, sxy));
    const float2 dtr = fma2(q.omg_tr, phi, mul2(q.nomg[9], add2(sxy, k.zz)));
    split_second_order2(d1, d2, dtr, d.xx, d.yy, d.zz);
    d.xyy = mul2(q.nomg[10], k.xyy);
    d.xxy = mul2(q.nomg[11], k.xxy);
    d.xxz = mul2(q.nomg[12], k.xxz);
    d.xyz = mul2(q.nomg[13], k.xyz);
    d.xxyy = fma2(q.omg_4, phi, mul2(q.nomg[14], k.xxyy));
    return shift15_2<true>(d, vu);
}

// Raw moments of the rest state times `scale`, added to m: zeroth 1, xx = yy = zz = cs2,
// xxyy = cs2^2, the rest 0 (the moments of the weights w_a, or w^phi_a at c_sphi^2).
__device__ __forceinline__ Raw15<float2> plus_rest15_2(Raw15<float2> m, float2 scale, float2 cs2s,
                                                       float2 cs4s) {
    m.m0 = add2(m.m0, scale);
    m.xx = add2(m.xx, cs2s);
    m.yy = add2(m.yy, cs2s);
    m.zz = add2(m.zz, cs2s);
    m.xxyy = add2(m.xxyy, cs4s);
    return m;
}

// The lean pair update.  f holds the pulled flow deviations f - w_a (the stored values, not
// offset); g the pulled scalar populations.  Both collisions work on the raw moments of the
// deviations from the node's own rest state (f - w_a, g - w^phi_a T), adding the rest
// state's moments back where the central moments need them, and form the post-collision
// deviations -- the values stored -- from the deviations' post-collision moments; the
// numbers stay small, so the FP32 rounding stays far below the 16-bit resolution.
template <typename S, int Q>
__device__ __forceinline__ void pair_collide_store_lean(float2 (&f)[15], float2 (&g)[Q],
                                                        S* __restrict__ Fout, S* __restrict__ Gout,
                                                        float* __restrict__ Tout,
                                                        const PairParams& q, int P, int c0,
                                                        uint32_t seed) {
    using Pk = Pack<S>;
    using two = typename Pk::two;
    float2 T = g[0];
#pragma unroll
    for (int a = 1; a < Q; ++a) T = add2(T, g[a]);
    T = add2(T, q.halfR);
    const float2 Fz = fma2(q.gbeta, sub2(T, q.T0), q.fz);
    const Raw15<float2> df = raw15_2(f);  // moments of f - w_a
    const Raw15<float2> mf = plus_rest15_2(df, make_float2(1.f, 1.f), make_float2(1.f / 3.f, 1.f / 3.f),
                                           make_float2(1.f / 9.f, 1.f / 9.f));
    const float2 inv_rho = make_float2(1.0f / mf.m0.x, 1.0f / mf.m0.y);
    const Vel2 vu = vel2(mul2(add2(mf.x, q.halffx), inv_rho), mul2(add2(mf.y, q.halffy), inv_rho),
                         mul2(fma2(make_float2(0.5f, 0.5f), Fz, mf.z), inv_rho));
    *reinterpret_cast<float2*>(Tout + c0) = T;  // the reference of this node's stored deviations
    if constexpr (Q == 15) {
#pragma unroll
        for (int a = 0; a < 15; ++a) g[a] = fma2(q.nwg[a], T, g[a]);  // g - w^phi_a T
        const Raw15<float2> dg = raw15_2(g);
        const Raw15<float2> mg = plus_rest15_2(dg, T, mul2(q.cs2, T), mul2(q.cs4, T));
        populations15_2(add15_2(dg, thermal15_increment2(mg, vu, q)), g);
#pragma unroll
        for (int a = 0; a < 15; ++a)
            *reinterpret_cast<two*>(Gout + a * P + c0) = Pk::from_float2(g[a]);
    } else {
        collide_thermal7_2(g, vu, q);
#pragma unroll
        for (int a = 0; a < Q; ++a)
            *reinterpret_cast<two*>(Gout + a * P + c0) = Pk::from_float2(fma2(q.nwg[a], T, g[a]));
    }
    populations15_2(add15_2(df, flow_increment2(mf, inv_rho, Fz, q, vu)), f);
    const uint32_t seed0 = dither_from_weyl(seed), seed1 = dither_from_weyl(seed + kDitherNodeStep);
#pragma unroll
    for (int a = 0; a < 15; ++a)
        *reinterpret_cast<two*>(Fout + a * P + c0) =
            Pk::template store2f<Storage<S>::sr_flow>(f[a], dither_of(seed0, a), dither_of(seed1, a));
}

// The pair update after the pull: f holds the pulled flow deviations (f - w_a), g the pulled
// scalar populations; the lean or the increment form per lattice (LBM_PAIR_LEAN_*).
template <typename S, int Q>
__device__ __forceinline__ void pair_finish(float2 (&f)[15], float2 (&g)[Q], S* __restrict__ Fout,
                                            S* __restrict__ Gout, float* __restrict__ Tout,
                                            const PairParams& q, int P, int c0, uint32_t seed) {
    if constexpr (Q == 15 ? LBM_PAIR_LEAN_Q15 : LBM_PAIR_LEAN_Q7) {
        pair_collide_store_lean<S, Q>(f, g, Fout, Gout, Tout, q, P, c0, seed);
    } else {
#pragma unroll
        for (int a = 0; a < 15; ++a) f[a] = add2(f[a], q.wf[a]);
        pair_collide_store<S, Q>(f, g, Fout, Gout, Tout, q, P, c0, seed);
    }
}

// ---------------------------------------------------------------------------------
// The update of nodes c0 (i = 2t) and c0 + 1 of a row away from the y and z walls.
// lo: i = 0 is the first node (its +x links come through the cold face); hi: i + 1 is
// the last node (its -x links come through the hot face).  Indices are 32-bit (the
// launcher takes this kernel only when 15 * plane < 2^31).
//
// Source of link a for node i is i - e_x(a) in row r_a = e_y nx + e_z nxy below:
//   e_x =  0: nodes (2t, 2t+1)   -- one aligned 32-bit load of two 16-bit values;
//   e_x = +1: nodes (2t-1, 2t)   -- lane .x through the cold face when lo;
//   e_x = -1: nodes (2t+1, 2t+2) -- lane .y through the hot face when hi.
// A link through an x face reads the node's own opposite population (bounce-back,
// flow; anti-bounce-back with the face temperature, scalar), selected by index so that
// every thread issues the same loads.
// ---------------------------------------------------------------------------------
template <typename S, int Q>
__device__ __forceinline__ void pair_node(const S* __restrict__ Fin, const S* __restrict__ Gin,
                                          const float* __restrict__ Tin, S* __restrict__ Fout,
                                          S* __restrict__ Gout, float* __restrict__ Tout,
                                          const PairParams& q, int nx, int nxy, int P, int c0,
                                          bool lo, bool hi, uint32_t seed) {
    using Pk = Pack<S>;
    using two = typename Pk::two;
    float2 g[Q], f[15];
    // scalar populations: the stored deviation plus w^phi_a T of the node that holds it
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int r = ey(a) * nx + ez(a) * nxy;
        const S* Ga = Gin + a * P;
        // node temperatures (2t, 2t+1) of the source row, shared by the links of that row
        const float2 Tp = *reinterpret_cast<const float2*>(Tin + c0 - r);
        if (ex(a) == 0) {
            const float2 v = Pk::to_float2(*reinterpret_cast<const two*>(Ga + c0 - r));
            g[a] = fma2(q.wg[a], Tp, v);
        } else if (ex(a) > 0) {
            const S* Gs = Ga - r - 1;
            const int i0 = lo ? c0 + r + 1 + (opp(a) - a) * P : c0;
            const float* Ts = Tin - r - 1;
            const float T0 = Ts[lo ? c0 + r + 1 : c0];
            float2 v = make_float2(Pk::to_float(Gs[i0]), Pk::to_float(Gs[c0 + 1]));
            v = fma2(q.wg[a], make_float2(T0, Tp.x), v);
            v.x = lo ? q.wTc2[a] - v.x : v.x;
            g[a] = v;
        } else {
            const S* Gs = Ga - r + 1;
            const int i1 = hi ? c0 + r + (opp(a) - a) * P : c0 + 1;
            const float* Ts = Tin - r + 1;
            const float T1 = Ts[hi ? c0 + r : c0 + 1];
            float2 v = make_float2(Pk::to_float(Gs[c0]), Pk::to_float(Gs[i1]));
            v = fma2(q.wg[a], make_float2(Tp.y, T1), v);
            v.y = hi ? q.wTh2[a] - v.y : v.y;
            g[a] = v;
        }
    }
    // flow populations: the stored deviations f - w_a (w_a is added back by the caller)
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        const int r = ey(a) * nx + ez(a) * nxy;
        const S* Fa = Fin + a * P;
        if (ex(a) == 0) {
            f[a] = Pk::flow2(*reinterpret_cast<const two*>(Fa + c0 - r));
        } else if (ex(a) > 0) {
            const S* Fs = Fa - r - 1;
            const int i0 = lo ? c0 + r + 1 + (opp(a) - a) * P : c0;
            f[a] = Pk::flow2(Fs[i0], Fs[c0 + 1]);
        } else {
            const S* Fs = Fa - r + 1;
            const int i1 = hi ? c0 + r + (opp(a) - a) * P : c0 + 1;
            f[a] = Pk::flow2(Fs[c0], Fs[i1]);
        }
    }
    pair_finish<S, Q>(f, g, Fout, Gout, Tout, q, P, c0, seed);
}

// ---------------------------------------------------------------------------------
// The pair update at the paper's unit higher-order rates (collide_unit.cuh): the scalar
// collision needs only phi and the first moments of the pulled g, so the thermal pull is
// reduced to those four pairs at once and the flow update runs with no scalar population
// held in registers.  Pull addressing and wall rules as pair_node.
// ---------------------------------------------------------------------------------
template <typename S, int Q>
__device__ __forceinline__ void pair_unit_update(Pair m0, Pair mx, Pair my, Pair mz, Pair (&f)[15],
                                                 S* __restrict__ Fout, S* __restrict__ Gout,
                                                 float* __restrict__ Tout, const PairParams& q,
                                                 int P, int c0, uint32_t seed);

template <typename S, int Q>
__device__ __forceinline__ void pair_node_unit(const S* __restrict__ Fin, const S* __restrict__ Gin,
                                               const float* __restrict__ Tin, S* __restrict__ Fout,
                                               S* __restrict__ Gout, float* __restrict__ Tout,
                                               const PairParams& q, int nx, int nxy, int P, int c0,
                                               bool lo, bool hi, uint32_t seed) {
    using Pk = Pack<S>;
    using two = typename Pk::two;
    Pair m0, mx, my, mz;
    {
        Pair g[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int r = ey(a) * nx + ez(a) * nxy;
            const S* Ga = Gin + a * P;
            const float2 Tp = *reinterpret_cast<const float2*>(Tin + c0 - r);
            if (ex(a) == 0) {
                const float2 v = Pk::to_float2(*reinterpret_cast<const two*>(Ga + c0 - r));
                g[a].v = fma2(q.wg[a], Tp, v);
            } else if (ex(a) > 0) {
                const S* Gs = Ga - r - 1;
                const int i0 = lo ? c0 + r + 1 + (opp(a) - a) * P : c0;
                const float* Ts = Tin - r - 1;
                const float T0 = Ts[lo ? c0 + r + 1 : c0];
                float2 v = make_float2(Pk::to_float(Gs[i0]), Pk::to_float(Gs[c0 + 1]));
                v = fma2(q.wg[a], make_float2(T0, Tp.x), v);
                v.x = lo ? q.wTc2[a] - v.x : v.x;
                g[a].v = v;
            } else {
                const S* Gs = Ga - r + 1;
                const int i1 = hi ? c0 + r + (opp(a) - a) * P : c0 + 1;
                const float* Ts = Tin - r + 1;
                const float T1 = Ts[hi ? c0 + r : c0 + 1];
                float2 v = make_float2(Pk::to_float(Gs[c0]), Pk::to_float(Gs[i1]));
                v = fma2(q.wg[a], make_float2(Tp.y, T1), v);
                v.y = hi ? q.wTh2[a] - v.y : v.y;
                g[a].v = v;
            }
        }
        raw_first<Pair, Q>(g, m0, mx, my, mz);
    }
    Pair f[15];  // the stored flow deviations f - w_a
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        const int r = ey(a) * nx + ez(a) * nxy;
        const S* Fa = Fin + a * P;
        if (ex(a) == 0) {
            f[a].v = Pk::flow2(*reinterpret_cast<const two*>(Fa + c0 - r));
        } else if (ex(a) > 0) {
            const S* Fs = Fa - r - 1;
            const int i0 = lo ? c0 + r + 1 + (opp(a) - a) * P : c0;
            f[a].v = Pk::flow2(Fs[i0], Fs[c0 + 1]);
        } else {
            const S* Fs = Fa - r + 1;
            const int i1 = hi ? c0 + r + (opp(a) - a) * P : c0 + 1;
            f[a].v = Pk::flow2(Fs[c0], Fs[i1]);
        }
    }
    pair_unit_update<S, Q>(m0, mx, my, mz, f, Fout, Gout, Tout, q, P, c0, seed);
}

// Read-only global loads as volatile statements: they keep their program order, so a
// block of them is issued before the arithmetic that follows it.
__device__ __forceinline__ uint32_t ldnc_b32(const void* p) {
    uint32_t v;
    asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned short ldnc_b16(const void* p) {
    unsigned short v;
    asm volatile("ld.global.nc.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float2 ldnc_f2(const float* p) {
    float2 v;
    asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ float ldnc_f(const float* p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// Whether the lattice of Q scalar directions has a link with these y, z components and an
// x component of the given sign (sx = 0: any).
template <int Q>
__host__ __device__ constexpr bool has_link(int sx, int dy, int dz) {
    for (int a = 0; a < Q; ++a)
        if (ey(a) == dy && ez(a) == dz && (sx == 0 || ex(a) == sx)) return true;
    return false;
}

// pair_node_unit with every load of the pair -- the raw 16-bit scalar and flow words and
// the node temperatures, one pair per source row and one value per shifted source -- issued
// in one block before any arithmetic, so that a warp waits for memory once per pair rather
// than once per batch the compiler would otherwise form.  The same values as
// pair_node_unit, bit for bit.
template <typename S, int Q>
__device__ __forceinline__ void pair_node_unit_early(const S* __restrict__ Fin, const S* __restrict__ Gin,
                                                     const float* __restrict__ Tin, S* __restrict__ Fout,
                                                     S* __restrict__ Gout, float* __restrict__ Tout,
                                                     const PairParams& q, int nx, int nxy, int P, int c0,
                                                     bool lo, bool hi, uint32_t seed) {
    using Pk = Pack<S>;
    uint32_t gw[Q], fw[15];
    unsigned short gx[Q], gy[Q], fx[15], fy[15];
    float2 Tp[9];
    float T0[9], T1[9];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int r = ey(a) * nx + ez(a) * nxy;
        const S* Ga = Gin + a * P;
        if (ex(a) == 0) {
            gw[a] = ldnc_b32(Ga + c0 - r);
        } else if (ex(a) > 0) {
            const S* Gs = Ga - r - 1;
            gx[a] = ldnc_b16(Gs + (lo ? c0 + r + 1 + (opp(a) - a) * P : c0));
            gy[a] = ldnc_b16(Gs + c0 + 1);
        } else {
            const S* Gs = Ga - r + 1;
            gx[a] = ldnc_b16(Gs + c0);
            gy[a] = ldnc_b16(Gs + (hi ? c0 + r + (opp(a) - a) * P : c0 + 1));
        }
    }
#pragma unroll
    for (int sl = 0; sl < 9; ++sl) {
        const int dy = sl / 3 - 1, dz = sl % 3 - 1;
        if (!has_link<Q>(0, dy, dz)) continue;
        const int r = dy * nx + dz * nxy;
        Tp[sl] = ldnc_f2(Tin + c0 - r);
        if (has_link<Q>(1, dy, dz)) T0[sl] = ldnc_f(lo ? Tin + c0 : Tin + c0 - r - 1);
        if (has_link<Q>(-1, dy, dz)) T1[sl] = ldnc_f(hi ? Tin + c0 + 1 : Tin + c0 - r + 2);
    }
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        const int r = ey(a) * nx + ez(a) * nxy;
        const S* Fa = Fin + a * P;
        if (ex(a) == 0) {
            fw[a] = ldnc_b32(Fa + c0 - r);
        } else if (ex(a) > 0) {
            const S* Fs = Fa - r - 1;
            fx[a] = ldnc_b16(Fs + (lo ? c0 + r + 1 + (opp(a) - a) * P : c0));
            fy[a] = ldnc_b16(Fs + c0 + 1);
        } else {
            const S* Fs = Fa - r + 1;
            fx[a] = ldnc_b16(Fs + c0);
            fy[a] = ldnc_b16(Fs + (hi ? c0 + r + (opp(a) - a) * P : c0 + 1));
        }
    }
    Pair m0, mx, my, mz;
    {
        Pair g[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int sl = (ey(a) + 1) * 3 + (ez(a) + 1);
            if (ex(a) == 0) {
                g[a].v = fma2(q.wg[a], Tp[sl], Pk::word2(gw[a]));
            } else if (ex(a) > 0) {
                float2 v = fma2(q.wg[a], make_float2(T0[sl], Tp[sl].x), Pk::bits2(gx[a], gy[a]));
                v.x = lo ? q.wTc2[a] - v.x : v.x;
                g[a].v = v;
            } else {
                float2 v = fma2(q.wg[a], make_float2(Tp[sl].y, T1[sl]), Pk::bits2(gx[a], gy[a]));
                v.y = hi ? q.wTh2[a] - v.y : v.y;
                g[a].v = v;
            }
        }
        raw_first<Pair, Q>(g, m0, mx, my, mz);
    }
    Pair f[15];  // the stored flow deviations f - w_a
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        f[a].v = ex(a) == 0 ? Pk::word2(fw[a]) : Pk::bits2(fx[a], fy[a]);
        if constexpr (Pk::down != 1.f) f[a].v = mul2(f[a].v, make_float2(Pk::down, Pk::down));
    }
    pair_unit_update<S, Q>(m0, mx, my, mz, f, Fout, Gout, Tout, q, P, c0, seed);
}

// The unit-rate pair update from the pulled scalar sums (phi and the first moments of g)
// and the pulled flow deviations f - w_a: collision, then the stores of both nodes.
template <typename S, int Q>
__device__ __forceinline__ void pair_unit_update(Pair m0, Pair mx, Pair my, Pair mz, Pair (&f)[15],
                                                 S* __restrict__ Fout, S* __restrict__ Gout,
                                                 float* __restrict__ Tout, const PairParams& q,
                                                 int P, int c0, uint32_t seed) {
    using Pk = Pack<S>;
    using two = typename Pk::two;
    const UnitRates<Pair>& ur = q.ur;
    const Pair T = m0 + ur.halfR;  // Eq. (25)
    const Pair Fz = {fma2(q.gbeta, sub2(T.v, q.T0), q.fz)};
    const Pair Fx = {q.fx}, Fy = {q.fy};
    const Low10<Pair> dm = raw_low15<Pair>(f);
    const Pair inv_rho = {make_float2(1.0f / (1.0f + dm.m0.v.x), 1.0f / (1.0f + dm.m0.v.y))};
    UPow<Pair> u;
    Raw15<Pair> D;
    flow_unit<Pair>(dm, Fx, Fy, Fz, ur, inv_rho, u, D);
    populations15<Pair>(D, f);
    const uint32_t seed0 = dither_from_weyl(seed), seed1 = dither_from_weyl(seed + kDitherNodeStep);
#pragma unroll
    for (int a = 0; a < 15; ++a)
        *reinterpret_cast<two*>(Fout + a * P + c0) =
            Pk::template store2f<Storage<S>::sr_flow>(f[a].v, dither_of(seed0, a), dither_of(seed1, a));
    *reinterpret_cast<float2*>(Tout + c0) = T.v;  // the reference of this node's stored deviations
    Pair g[Q];
    if constexpr (Q == 15) {
        thermal15_unit<Pair>(T, m0, mx, my, mz, u, ur, D);
        populations15<Pair>(D, g);
    } else {
        thermal7_unit<Pair>(T, m0, mx, my, mz, u, ur, g);
    }
#pragma unroll
    for (int a = 0; a < Q; ++a)
        *reinterpret_cast<two*>(Gout + a * P + c0) = Pk::template store2<Storage<S>::sr_thermal>(
            g[a].v, dither_of(seed0, 15 + a), dither_of(seed1, 15 + a));
}

}  // namespace lbm
