// collide_unit.cuh -- the collisions of arXiv:1710.04751 at the paper's own choice of the
// higher-order rates, computed directly from the few moments that choice leaves alive.
//
// The paper sets every relaxation rate it does not tie to a transport coefficient to
// unity: for the scalar (Sec. 2.2, App. C) all but omega_1..3, which give the
// diffusivity (Eq. 23); for the flow (App. A) all but the viscous ones (read here as the
// five shear moments; the bulk moment and the third and fourth orders relax at 1).  A
// central moment relaxed at rate 1 takes its equilibrium (plus, for the flow, its source
// share (1 - omega) Gamma = 0) whatever its pre-collision value.  So the post-collision
// state depends on the pulled populations only through
//   flow:   rho, the momentum and the six second-order moments (ten raw moments);
//   scalar: phi (Eq. 25) and the three first-order moments.
// collide.cuh computes every moment and relaxes each with its own rate; for these rates
// the result is the same up to rounding (the tests hold both to the FP64 oracle, which
// runs the paper's closed-form cascades).  Here the post-collision central moments are
//   flow   c0 = rho, c_i = F_i/2, c_xy.. = (1 - omega) k_xy.., traceless second-order
//          combinations (1 - omega) k, trace rho (= 3 c_s^2 rho), third order 0,
//          c_xxyy = E (reading R1: c_xx c_yy / rho, or rho c_s^4);
//   scalar c0 = phi + R/2, c_i = (1 - omega_i)(m_i - u_i m0), c_ii = c_sphi^2 phi,
//          mixed and third order 0, c_xxyy = c_sphi^4 phi (Eq. 15);
// shifted to raw moments by the binomial theorem about u (Eqs. 14, 17) and inverted to
// populations.  Everything is written for moments taken RELATIVE TO THE REST STATE
// (f - w_a for the flow, g - w^phi_a phi for the scalar): the quantities stay small, which
// keeps the rounding of the single-precision forms far below their storage resolution.
//
// Templated on the arithmetic type: float, double, or Pair (two nodes in packed FP32
// pair instructions, pair.cuh).
#pragma once

#include "collide.cuh"

namespace lbm {

// Fused multiply-add and constants for the arithmetic types.
__device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return fma(a, b, c); }
template <typename T>
__device__ __forceinline__ T cst(double v) { return T(v); }

// The ten raw moments up to second order of a D3Q15 vector (the sign transform of raw15
// without its third- and fourth-order outputs).
template <typename T>
struct Low10 {
    T m0, x, y, z, xy, xz, yz, xx, yy, zz;
};

template <typename T>
__device__ __forceinline__ Low10<T> raw_low15(const T (&p)[15]) {
    const T a0 = p[7] + p[8], b0 = p[7] - p[8];
    const T a1 = p[9] + p[10], b1 = p[9] - p[10];
    const T a2 = p[11] + p[12], b2 = p[11] - p[12];
    const T a3 = p[13] + p[14], b3 = p[13] - p[14];
    const T c0 = a0 + a1, c1 = a0 - a1, c2 = a2 + a3, c3 = a2 - a3;
    const T e0 = b0 + b1, e1 = b0 - b1, e2 = b2 + b3, e3 = b2 - b3;
    const T H0 = c0 + c2, Hz = c0 - c2, Hy = c1 + c3, Hyz = c1 - c3;
    const T Hx = e0 + e2, Hxz = e0 - e2, Hxy = e1 + e3;
    const T px = p[1] + p[2], qx = p[1] - p[2];
    const T py = p[3] + p[4], qy = p[3] - p[4];
    const T pz = p[5] + p[6], qz = p[5] - p[6];
    Low10<T> m;
    m.m0 = p[0] + px + py + pz + H0;
    m.x = qx + Hx;
    m.y = qy + Hy;
    m.z = qz + Hz;
    m.xy = Hxy;
    m.xz = Hxz;
    m.yz = Hyz;
    m.xx = px + H0;
    m.yy = py + H0;
    m.zz = pz + H0;
    return m;
}

// Zeroth and first raw moments of a D3Q15 or D3Q7 vector.
template <typename T, int Q>
__device__ __forceinline__ void raw_first(const T (&p)[Q], T& m0, T& mx, T& my, T& mz) {
    const T px = p[1] + p[2], qx = p[1] - p[2];
    const T py = p[3] + p[4], qy = p[3] - p[4];
    const T pz = p[5] + p[6], qz = p[5] - p[6];
    if constexpr (Q == 15) {
        const T a0 = p[7] + p[8], b0 = p[7] - p[8];
        const T a1 = p[9] + p[10], b1 = p[9] - p[10];
        const T a2 = p[11] + p[12], b2 = p[11] - p[12];
        const T a3 = p[13] + p[14], b3 = p[13] - p[14];
        const T c0 = a0 + a1, c1 = a0 - a1, c2 = a2 + a3, c3 = a2 - a3;
        const T e0 = b0 + b1, e2 = b2 + b3;
        m0 = p[0] + px + py + pz + (c0 + c2);
        mx = qx + (e0 + e2);
        my = qy + (c1 + c3);
        mz = qz + (c0 - c2);
    } else {
        m0 = p[0] + px + py + pz;
        mx = qx;
        my = qy;
        mz = qz;
    }
}

// The populations whose raw moments are r (the inverse of raw15): p = K^-1 applied in the
// monomial basis, diagonal links by the inverse three-level sign transform.
template <typename T>
__device__ __forceinline__ void populations15(const Raw15<T>& r, T (&p)[15]) {
    const T G0 = r.xxyy, Gx = r.xyy, Gy = r.xxy, Gz = r.xxz;
    const T P0 = G0 + Gz, P0m = G0 - Gz, Px = Gx + r.xz, Pxm = Gx - r.xz;
    const T Py = Gy + r.yz, Pym = Gy - r.yz, Pxy = r.xy + r.xyz, Pxym = r.xy - r.xyz;
    const T Q0 = P0 + Py, Q1 = P0 - Py, X0 = Px + Pxy, X1 = Px - Pxy;
    const T Q2 = P0m + Pym, Q3 = P0m - Pym, X2 = Pxm + Pxym, X3 = Pxm - Pxym;
    const T e = cst<T>(0.125), h = cst<T>(0.5);
    p[7] = e * (Q0 + X0);
    p[8] = e * (Q0 - X0);
    p[9] = e * (Q1 + X1);
    p[10] = e * (Q1 - X1);
    p[11] = e * (Q2 + X2);
    p[12] = e * (Q2 - X2);
    p[13] = e * (Q3 + X3);
    p[14] = e * (Q3 - X3);
    const T px = r.xx - G0, qx = r.x - Gx;
    const T py = r.yy - G0, qy = r.y - Gy;
    const T pz = r.zz - G0, qz = r.z - Gz;
    p[1] = h * (px + qx);
    p[2] = h * (px - qx);
    p[3] = h * (py + qy);
    p[4] = h * (py - qy);
    p[5] = h * (pz + qz);
    p[6] = h * (pz - qz);
    p[0] = r.m0 - px - py - pz - G0;
}

// The relaxation rates and constants the unit-rate collisions use.
template <typename T>
struct UnitRates {
    T om1[3];      // 1 - omega_4, 5, 6 (flow xy, xz, yz) ...
    T omA, omB;    // 1 - omega_7, 1 - omega_8 (flow xx - yy, xx + yy - 2 zz)
    T omg[3];      // 1 - omega_1, 2, 3 (scalar first order)
    T cs2, cs4;    // c_sphi^2, c_sphi^4
    T R, halfR;    // scalar source R and R/2
    int e4_mode;
};

template <typename T, typename real>
__device__ __forceinline__ UnitRates<T> unit_rates(const DevParams<real>& p) {
    UnitRates<T> r;
    for (int i = 0; i < 3; ++i) {
        r.om1[i] = cst<T>(1.0 - (double)p.om_f[4 + i]);
        r.omg[i] = cst<T>(1.0 - (double)p.om_g[1 + i]);
    }
    r.omA = cst<T>(1.0 - (double)p.om_f[7]);
    r.omB = cst<T>(1.0 - (double)p.om_f[8]);
    r.cs2 = cst<T>((double)p.cs2_phi);
    r.cs4 = cst<T>((double)p.cs2_phi * (double)p.cs2_phi);
    r.R = cst<T>((double)p.heat_source);
    r.halfR = cst<T>(0.5 * (double)p.heat_source);
    r.e4_mode = p.e4_mode;
    return r;
}

// Powers of u shared by the binomial shifts.
template <typename T>
struct UPow {
    T x, y, z, xx, yy, zz, xy, xz, yz;
};
template <typename T>
__device__ __forceinline__ UPow<T> upow(T ux, T uy, T uz) {
    return UPow<T>{ux, uy, uz, ux * ux, uy * uy, uz * uz, ux * uy, ux * uz, uy * uz};
}

// Flow (App. A) at unit bulk / third / fourth-order rates.  dm: moments of f - w_a up to
// second order; F: the body force.  Returns u (Eq. 3) and D, the raw moments of the
// post-collision f~ - w_a.
template <typename T>
__device__ __forceinline__ void flow_unit(const Low10<T>& dm, T Fx, T Fy, T Fz, const UnitRates<T>& r,
                                          T inv_rho, UPow<T>& u, Raw15<T>& D) {
    const T h = cst<T>(0.5);
    const T delta = dm.m0;               // rho - 1
    const T rho = cst<T>(1.0) + delta;
    const T hx = h * Fx, hy = h * Fy, hz = h * Fz;  // post-collision first central moments
    u = upow<T>((dm.x + hx) * inv_rho, (dm.y + hy) * inv_rho, (dm.z + hz) * inv_rho);
    // pre-collision second-order central moments about u (the 1/3 of the rest state
    // cancels in every combination that relaxes): k_ab = m_ab - rho u_a u_b
    // + (u_a F_b + u_b F_a)/2, k_aa = m_aa - rho u_a^2 + u_a F_a
    const T kxy = fmad(u.x, hy, fmad(u.y, hx, dm.xy - rho * u.xy));
    const T kxz = fmad(u.x, hz, fmad(u.z, hx, dm.xz - rho * u.xz));
    const T kyz = fmad(u.y, hz, fmad(u.z, hy, dm.yz - rho * u.yz));
    const T sxx = fmad(u.x, Fx, dm.xx - rho * u.xx);  // k_xx - 1/3
    const T syy = fmad(u.y, Fy, dm.yy - rho * u.yy);
    const T szz = fmad(u.z, Fz, dm.zz - rho * u.zz);
    // relaxation: shear at its rates, trace to rho (its equilibrium 3 c_s^2 rho)
    const T cxy = r.om1[0] * kxy, cxz = r.om1[1] * kxz, cyz = r.om1[2] * kyz;
    const T A = r.omA * (sxx - syy);
    const T B = r.omB * (sxx + syy - cst<T>(2.0) * szz);
    const T B6 = B * cst<T>(1.0 / 6.0);
    const T txx = fmad(h, A, B6), tyy = B6 - h * A, tzz = cst<T>(-2.0) * B6;  // c_aa - rho/3
    const T d3 = delta * cst<T>(1.0 / 3.0);
    const T cxx = cst<T>(1.0 / 3.0) * rho + txx, cyy = cst<T>(1.0 / 3.0) * rho + tyy;
    // fourth-order equilibrium E (reading R1), less the rest value 1/9
    T E9 = delta * cst<T>(1.0 / 9.0);
    if (r.e4_mode == 0) E9 = fmad(txx * tyy, inv_rho, fmad(cst<T>(1.0 / 3.0), txx + tyy, E9));
    // raw moments of the post-collision state about the origin (binomial theorem with
    // third-order central moments 0), less the rest state's
    D.m0 = delta;
    D.x = fmad(rho, u.x, hx);
    D.y = fmad(rho, u.y, hy);
    D.z = fmad(rho, u.z, hz);
    D.xy = fmad(rho, u.xy, fmad(u.x, hy, fmad(u.y, hx, cxy)));
    D.xz = fmad(rho, u.xz, fmad(u.x, hz, fmad(u.z, hx, cxz)));
    D.yz = fmad(rho, u.yz, fmad(u.y, hz, fmad(u.z, hy, cyz)));
    D.xx = fmad(rho, u.xx, fmad(u.x, Fx, d3 + txx));
    D.yy = fmad(rho, u.yy, fmad(u.y, Fy, d3 + tyy));
    D.zz = fmad(rho, u.zz, fmad(u.z, Fz, d3 + tzz));
    const T ruxy = rho * u.xy;
    // xyy = u_x c_yy + 2 u_y c_xy + u_y^2 c_x + 2 u_x u_y c_y + rho u_x u_y^2
    D.xyy = fmad(ruxy, u.y, fmad(u.xy, Fy, fmad(u.yy, hx, fmad(cst<T>(2.0) * u.y, cxy, u.x * cyy))));
    D.xxy = fmad(ruxy, u.x, fmad(u.xy, Fx, fmad(u.xx, hy, fmad(cst<T>(2.0) * u.x, cxy, u.y * cxx))));
    D.xxz = fmad(rho * u.xz, u.x, fmad(u.xz, Fx, fmad(u.xx, hz, fmad(cst<T>(2.0) * u.x, cxz, u.z * cxx))));
    // xyz = u_x c_yz + u_y c_xz + u_z c_xy + u_x u_y c_z + u_x u_z c_y + u_y u_z c_x + rho u_x u_y u_z
    D.xyz = fmad(ruxy, u.z, fmad(u.xy, hz, fmad(u.xz, hy, fmad(u.yz, hx,
                 fmad(u.x, cyz, fmad(u.y, cxz, u.z * cxy))))));
    // xxyy = E + u_x^2 c_yy + u_y^2 c_xx + 4 u_x u_y c_xy + 2 u_x u_y^2 c_x + 2 u_x^2 u_y c_y
    //        + rho u_x^2 u_y^2, less 1/9
    D.xxyy = fmad(ruxy, u.xy, fmad(u.xy, fmad(u.y, Fx, u.x * Fy), fmad(cst<T>(4.0) * u.xy, cxy,
                  fmad(u.yy, cxx, fmad(u.xx, cyy, E9)))));
}

// Scalar D3Q15 (Sec. 2.2) at unit higher-order rates.  phi = sum g + R/2 (Eq. 25), m0 =
// sum g, m_i the first raw moments of the pulled g.  D: raw moments of g~ - w^phi_a phi.
template <typename T>
__device__ __forceinline__ void thermal15_unit(T phi, T m0, T mx, T my, T mz, const UPow<T>& u,
                                               const UnitRates<T>& r, Raw15<T>& D) {
    const T c0 = phi + r.halfR;  // m0 + R: the zeroth moment gains the source
    const T cx = r.omg[0] * (mx - u.x * m0);
    const T cy = r.omg[1] * (my - u.y * m0);
    const T cz = r.omg[2] * (mz - u.z * m0);
    const T C2 = r.cs2 * phi;
    const T two = cst<T>(2.0);
    D.m0 = r.halfR;
    D.x = fmad(u.x, c0, cx);
    D.y = fmad(u.y, c0, cy);
    D.z = fmad(u.z, c0, cz);
    D.xy = fmad(u.xy, c0, fmad(u.x, cy, u.y * cx));
    D.xz = fmad(u.xz, c0, fmad(u.x, cz, u.z * cx));
    D.yz = fmad(u.yz, c0, fmad(u.y, cz, u.z * cy));
    D.xx = fmad(u.xx, c0, two * u.x * cx);   // c_xx = c_sphi^2 phi cancels the rest value
    D.yy = fmad(u.yy, c0, two * u.y * cy);
    D.zz = fmad(u.zz, c0, two * u.z * cz);
    D.xyy = fmad(u.xy * u.y, c0, fmad(two * u.xy, cy, fmad(u.yy, cx, u.x * C2)));
    D.xxy = fmad(u.xy * u.x, c0, fmad(two * u.xy, cx, fmad(u.xx, cy, u.y * C2)));
    D.xxz = fmad(u.xz * u.x, c0, fmad(two * u.xz, cx, fmad(u.xx, cz, u.z * C2)));
    D.xyz = fmad(u.xy * u.z, c0, fmad(u.xy, cz, fmad(u.xz, cy, u.yz * cx)));
    D.xxyy = fmad(u.xx * u.yy, c0, fmad(two * u.xy, fmad(u.y, cx, u.x * cy), (u.xx + u.yy) * C2));
}

// Scalar D3Q7 (App. C) at unit higher-order rates: the post-collision g~ - w^phi_a phi.
template <typename T>
__device__ __forceinline__ void thermal7_unit(T phi, T m0, T mx, T my, T mz, const UPow<T>& u,
                                              const UnitRates<T>& r, T (&d)[7]) {
    const T c0 = phi + r.halfR;
    const T cx = r.omg[0] * (mx - u.x * m0);
    const T cy = r.omg[1] * (my - u.y * m0);
    const T cz = r.omg[2] * (mz - u.z * m0);
    const T two = cst<T>(2.0), h = cst<T>(0.5);
    const T Dx = fmad(u.x, c0, cx), Dy = fmad(u.y, c0, cy), Dz = fmad(u.z, c0, cz);
    const T Dxx = fmad(u.xx, c0, two * u.x * cx);
    const T Dyy = fmad(u.yy, c0, two * u.y * cy);
    const T Dzz = fmad(u.zz, c0, two * u.z * cz);
    d[1] = h * (Dxx + Dx);
    d[2] = h * (Dxx - Dx);
    d[3] = h * (Dyy + Dy);
    d[4] = h * (Dyy - Dy);
    d[5] = h * (Dzz + Dz);
    d[6] = h * (Dzz - Dz);
    d[0] = r.halfR - Dxx - Dyy - Dzz;
}

// Whether a context's rates are the paper's unit higher-order rates (host side).
template <typename real>
inline bool has_unit_rates(const DevParams<real>& p, int Q) {
    for (int b = 9; b < 15; ++b)
        if (p.om_f[b] != real(1)) return false;
    for (int b = 4; b < Q; ++b)
        if (p.om_g[b] != real(1)) return false;
    return true;
}

}  // namespace lbm
