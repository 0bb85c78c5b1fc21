// collide.cuh -- one-cell cascaded collisions of arXiv:1710.04751 in registers.
//
//   collide_flow      Appendix A: D3Q15 flow collision with the body-force source
//   collide_thermal15 Sec. 2.2: D3Q15 scalar collision with a uniform source R
//   collide_thermal7  Appendix C: D3Q7 scalar collision with a uniform source R
//
// The paper writes each cascade as closed forms for the kernel components (g^_b, h^_b)
// that, added through K, make every central moment relax toward its equilibrium at its
// own rate while the lower orders are already relaxed.  The post-collision state that
// defines is computed here in an equivalent, cheaper order (same arithmetic result up to
// rounding):
//   1. raw moments of the populations (Eq. 17 / App. A notation) with a three-level
//      sign transform of the eight diagonal links;
//   2. central moments about u (binomial theorem, Eqs. 14 and 17);
//   3. their increments delta = kappa~ - kappa: each moment relaxes with its rate toward
//      its equilibrium (Eq. 15 for the scalar; Maxwellian for the flow), plus, for the
//      flow, the central moments Gamma of the source;
//   4. the increments shifted back to raw moments and inverted to populations
//      (the inverse of step 1), so that p~ = p + increment -- Eqs. 2a and 13a.
#pragma once

#include "internal.h"
#include "lattice.cuh"

namespace lbm {

// Raw moments of a D3Q15 population vector, by moment id (Mom).
template <typename real>
struct Raw15 {
    real m0, x, y, z, xy, xz, yz, xx, yy, zz, xyy, xxy, xxz, xyz, xxyy;
};

// Diagonal links 7..14 are (+-,+-,+-) with bit 0 of (a - 7) set for e_x < 0, bit 1 for
// e_y < 0, bit 2 for e_z < 0.  Three butterfly levels give all eight signed sums
// sum_d s_x^i s_y^j s_z^k p_d in 24 additions.
template <typename real>
__device__ __forceinline__ Raw15<real> raw15(const real (&p)[15]) {
    const real a0 = p[7] + p[8], b0 = p[7] - p[8];
    const real a1 = p[9] + p[10], b1 = p[9] - p[10];
    const real a2 = p[11] + p[12], b2 = p[11] - p[12];
    const real a3 = p[13] + p[14], b3 = p[13] - p[14];
    const real c0 = a0 + a1, c1 = a0 - a1, c2 = a2 + a3, c3 = a2 - a3;
    const real e0 = b0 + b1, e1 = b0 - b1, e2 = b2 + b3, e3 = b2 - b3;
    const real H0 = c0 + c2, Hz = c0 - c2, Hy = c1 + c3, Hyz = c1 - c3;
    const real Hx = e0 + e2, Hxz = e0 - e2, Hxy = e1 + e3, Hxyz = e1 - e3;
    const real px = p[1] + p[2], qx = p[1] - p[2];
    const real py = p[3] + p[4], qy = p[3] - p[4];
    const real pz = p[5] + p[6], qz = p[5] - p[6];
    Raw15<real> m;
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
    m.xyy = Hx;
    m.xxy = Hy;
    m.xxz = Hz;
    m.xyz = Hxyz;
    m.xxyy = H0;
    return m;
}

// Central moments of the 15 monomials about u (binomial theorem).  The zeroth and
// first orders are not needed by the callers beyond m0, x, y, z below.
template <typename real>
__device__ __forceinline__ Raw15<real> central15(const Raw15<real>& m, real ux, real uy, real uz) {
    const real uxx = ux * ux, uyy = uy * uy, uxy = ux * uy, uxz = ux * uz, uyz = uy * uz;
    Raw15<real> c;
    c.m0 = m.m0;
    c.x = m.x - ux * m.m0;
    c.y = m.y - uy * m.m0;
    c.z = m.z - uz * m.m0;
    c.xy = m.xy - ux * m.y - uy * m.x + uxy * m.m0;
    c.xz = m.xz - ux * m.z - uz * m.x + uxz * m.m0;
    c.yz = m.yz - uy * m.z - uz * m.y + uyz * m.m0;
    c.xx = m.xx - real(2) * ux * m.x + uxx * m.m0;
    c.yy = m.yy - real(2) * uy * m.y + uyy * m.m0;
    c.zz = m.zz - real(2) * uz * m.z + uz * uz * m.m0;
    c.xyy = m.xyy - real(2) * uy * m.xy - ux * m.yy + uyy * m.x + real(2) * uxy * m.y - ux * uyy * m.m0;
    c.xxy = m.xxy - real(2) * ux * m.xy - uy * m.xx + uxx * m.y + real(2) * uxy * m.x - uxx * uy * m.m0;
    c.xxz = m.xxz - real(2) * ux * m.xz - uz * m.xx + uxx * m.z + real(2) * uxz * m.x - uxx * uz * m.m0;
    c.xyz = m.xyz - ux * m.yz - uy * m.xz - uz * m.xy + uxy * m.z + uxz * m.y + uyz * m.x -
            uxy * uz * m.m0;
    c.xxyy = m.xxyy - real(2) * uy * m.xxy - real(2) * ux * m.xyy + uyy * m.xx + uxx * m.yy +
             real(4) * uxy * m.xy - real(2) * ux * uyy * m.x - real(2) * uxx * uy * m.y +
             uxx * uyy * m.m0;
    return c;
}

// Raw moments of a central-moment increment d about u: the inverse binomial shift.  With
// D0 = false the zeroth-order increment is zero (the flow) and its terms are dropped.
template <bool D0, typename real>
__device__ __forceinline__ Raw15<real> raw_of_central_increment(const Raw15<real>& d, real ux,
                                                                real uy, real uz) {
    const real uxx = ux * ux, uyy = uy * uy, uxy = ux * uy, uxz = ux * uz, uyz = uy * uz;
    Raw15<real> r;
    r.m0 = real(0);
    r.x = d.x;
    r.y = d.y;
    r.z = d.z;
    r.xy = d.xy + ux * d.y + uy * d.x;
    r.xz = d.xz + ux * d.z + uz * d.x;
    r.yz = d.yz + uy * d.z + uz * d.y;
    r.xx = d.xx + real(2) * ux * d.x;
    r.yy = d.yy + real(2) * uy * d.y;
    r.zz = d.zz + real(2) * uz * d.z;
    r.xyy = d.xyy + real(2) * uy * d.xy + ux * d.yy + uyy * d.x + real(2) * uxy * d.y;
    r.xxy = d.xxy + real(2) * ux * d.xy + uy * d.xx + uxx * d.y + real(2) * uxy * d.x;
    r.xxz = d.xxz + real(2) * ux * d.xz + uz * d.xx + uxx * d.z + real(2) * uxz * d.x;
    r.xyz = d.xyz + ux * d.yz + uy * d.xz + uz * d.xy + uxy * d.z + uxz * d.y + uyz * d.x;
    r.xxyy = d.xxyy + real(2) * uy * d.xxy + real(2) * ux * d.xyy + uyy * d.xx + uxx * d.yy +
             real(4) * uxy * d.xy + real(2) * ux * uyy * d.x + real(2) * uxx * uy * d.y;
    if constexpr (D0) {
        const real d0 = d.m0;
        r.m0 = d0;
        r.x += ux * d0;
        r.y += uy * d0;
        r.z += uz * d0;
        r.xy += uxy * d0;
        r.xz += uxz * d0;
        r.yz += uyz * d0;
        r.xx += uxx * d0;
        r.yy += uyy * d0;
        r.zz += uz * uz * d0;
        r.xyy += ux * uyy * d0;
        r.xxy += uxx * uy * d0;
        r.xxz += uxx * uz * d0;
        r.xyz += uxy * uz * d0;
        r.xxyy += uxx * uyy * d0;
    }
    return r;
}

// p += the populations whose raw moments are r (inverse of raw15).
template <typename real>
__device__ __forceinline__ void add_populations15(real (&p)[15], const Raw15<real>& r) {
    // diagonal links: inverse of the three-level sign transform (divided by 8)
    const real G0 = r.xxyy, Gx = r.xyy, Gy = r.xxy, Gz = r.xxz;
    const real P0 = G0 + Gz, P0m = G0 - Gz, Px = Gx + r.xz, Pxm = Gx - r.xz;
    const real Py = Gy + r.yz, Pym = Gy - r.yz, Pxy = r.xy + r.xyz, Pxym = r.xy - r.xyz;
    const real Q0 = P0 + Py, Q1 = P0 - Py, X0 = Px + Pxy, X1 = Px - Pxy;
    const real Q2 = P0m + Pym, Q3 = P0m - Pym, X2 = Pxm + Pxym, X3 = Pxm - Pxym;
    const real e = real(0.125);
    p[7] += e * (Q0 + X0);
    p[8] += e * (Q0 - X0);
    p[9] += e * (Q1 + X1);
    p[10] += e * (Q1 - X1);
    p[11] += e * (Q2 + X2);
    p[12] += e * (Q2 - X2);
    p[13] += e * (Q3 + X3);
    p[14] += e * (Q3 - X3);
    // axis links and rest
    const real px = r.xx - G0, qx = r.x - Gx;
    const real py = r.yy - G0, qy = r.y - Gy;
    const real pz = r.zz - G0, qz = r.z - Gz;
    p[1] += real(0.5) * (px + qx);
    p[2] += real(0.5) * (px - qx);
    p[3] += real(0.5) * (py + qy);
    p[4] += real(0.5) * (py - qy);
    p[5] += real(0.5) * (pz + qz);
    p[6] += real(0.5) * (pz - qz);
    p[0] += r.m0 - px - py - pz - G0;
}

// Second-order increments from the relaxed combinations xx-yy, xx+yy-2zz, xx+yy+zz.
template <typename real>
__device__ __forceinline__ void split_second_order(real d1, real d2, real dtr, real& dxx,
                                                   real& dyy, real& dzz) {
    dzz = (dtr - d2) * real(1.0 / 3.0);
    const real s = dtr - dzz;
    dxx = real(0.5) * (s + d1);
    dyy = real(0.5) * (s - d1);
}

// Flow collision (Appendix A).  f: pulled populations fbar, replaced by f~.  F: the body
// force (Boussinesq + uniform).  Returns u of Eq. (3).
//
// The moments that relax are those of (fbar + S) (the expansion of App. A's brackets).
// S, whose central moments are those of the Maxwellian forcing term (first order F,
// xyy/xxy/xxz = c_s^2 F, the rest zero -- the reading of the source the paper takes from
// its prior work), enters only through those central moments Gamma:
//   increment = (1 - omega) Gamma - omega (kappa(fbar) - kappa^eq)   for relaxed moments,
//   increment = Gamma                                                 for mass and momentum.
template <typename real>
__device__ __forceinline__ void collide_flow(real (&f)[15], real Fx, real Fy, real Fz,
                                             const DevParams<real>& p, real& ux, real& uy,
                                             real& uz) {
    const real cs2 = real(1.0 / 3.0);
    const Raw15<real> m = raw15<real>(f);
    const real rho = m.m0;
    const real inv_rho = real(1) / rho;
    ux = (m.x + real(0.5) * Fx) * inv_rho;
    uy = (m.y + real(0.5) * Fy) * inv_rho;
    uz = (m.z + real(0.5) * Fz) * inv_rho;
    const Raw15<real> k = central15<real>(m, ux, uy, uz);
    const real* om = p.om_f;
    Raw15<real> d;
    d.m0 = real(0);
    d.x = Fx;
    d.y = Fy;
    d.z = Fz;
    d.xy = -om[4] * k.xy;
    d.xz = -om[5] * k.xz;
    d.yz = -om[6] * k.yz;
    const real d1 = -om[7] * (k.xx - k.yy);
    const real d2 = -om[8] * (k.xx + k.yy - real(2) * k.zz);
    const real dtr = om[9] * (rho - (k.xx + k.yy + k.zz));  // equilibrium trace 3 c_s^2 rho
    split_second_order(d1, d2, dtr, d.xx, d.yy, d.zz);
    d.xyy = (real(1) - om[10]) * cs2 * Fx - om[10] * k.xyy;
    d.xxy = (real(1) - om[11]) * cs2 * Fy - om[11] * k.xxy;
    d.xxz = (real(1) - om[12]) * cs2 * Fz - om[12] * k.xxz;
    d.xyz = -om[13] * k.xyz;
    // 4th-order equilibrium: factorised from the post-collision second-order central
    // moments (mode 0), or Maxwellian rho c_s^4 (mode 1)
    const real E = p.e4_mode == 1 ? rho * real(1.0 / 9.0)
                                  : (k.xx + d.xx) * (k.yy + d.yy) * inv_rho;
    d.xxyy = om[14] * (E - k.xxyy);
    add_populations15<real>(f, raw_of_central_increment<false, real>(d, ux, uy, uz));
}

// Thermal D3Q15 collision (Sec. 2.2) with the uniform source R = p.heat_source: g becomes
// g~; u from the flow.  phi = sum gbar + R/2 (Eq. 25).  The source's only central moment
// is the zeroth, so the zeroth moment gains R and every other moment of gbar relaxes
// toward its equilibrium at phi (Eq. 15: c_sphi^2 phi on the diagonal second order,
// c_sphi^4 phi for xxyy, zero otherwise).
template <typename real>
__device__ __forceinline__ void collide_thermal15(real (&g)[15], real ux, real uy, real uz,
                                                  const DevParams<real>& p) {
    const Raw15<real> m = raw15<real>(g);
    const real R = p.heat_source;
    const real phi = m.m0 + real(0.5) * R;
    const Raw15<real> k = central15<real>(m, ux, uy, uz);
    const real* om = p.om_g;
    const real cs2 = p.cs2_phi;
    Raw15<real> d;
    d.m0 = R;
    d.x = -om[1] * k.x;
    d.y = -om[2] * k.y;
    d.z = -om[3] * k.z;
    d.xy = -om[4] * k.xy;
    d.xz = -om[5] * k.xz;
    d.yz = -om[6] * k.yz;
    const real d1 = -om[7] * (k.xx - k.yy);
    const real d2 = -om[8] * (k.xx + k.yy - real(2) * k.zz);
    const real dtr = om[9] * (real(3) * cs2 * phi - (k.xx + k.yy + k.zz));
    split_second_order(d1, d2, dtr, d.xx, d.yy, d.zz);
    d.xyy = -om[10] * k.xyy;
    d.xxy = -om[11] * k.xxy;
    d.xxz = -om[12] * k.xxz;
    d.xyz = -om[13] * k.xyz;
    d.xxyy = om[14] * (cs2 * cs2 * phi - k.xxyy);
    add_populations15<real>(g, raw_of_central_increment<true, real>(d, ux, uy, uz));
}

// Thermal D3Q7 collision (Appendix C) with the uniform source R: moments 0; x, y, z;
// xx-yy, xx+yy-2zz, xx+yy+zz (equilibrium 3 c_sphi^2 phi, phi = sum gbar + R/2).
template <typename real>
__device__ __forceinline__ void collide_thermal7(real (&g)[7], real ux, real uy, real uz,
                                                 const DevParams<real>& p) {
    const real px = g[1] + g[2], qx = g[1] - g[2];
    const real py = g[3] + g[4], qy = g[3] - g[4];
    const real pz = g[5] + g[6], qz = g[5] - g[6];
    const real m0 = g[0] + px + py + pz;
    const real R = p.heat_source;
    const real phi = m0 + real(0.5) * R;
    // central moments of gbar about u
    const real kx = qx - ux * m0, ky = qy - uy * m0, kz = qz - uz * m0;
    const real kxx = px - real(2) * ux * qx + ux * ux * m0;
    const real kyy = py - real(2) * uy * qy + uy * uy * m0;
    const real kzz = pz - real(2) * uz * qz + uz * uz * m0;
    const real* om = p.om_g;
    const real dx = -om[1] * kx, dy = -om[2] * ky, dz = -om[3] * kz;
    const real d1 = -om[4] * (kxx - kyy);
    const real d2 = -om[5] * (kxx + kyy - real(2) * kzz);
    const real dtr = om[6] * (real(3) * p.cs2_phi * phi - (kxx + kyy + kzz));
    real dxx, dyy, dzz;
    split_second_order(d1, d2, dtr, dxx, dyy, dzz);
    // raw increments (zeroth: R) and populations: p_{+-} = (r_xx +- r_x)/2,
    // p_0 = r_0 - (r_xx + r_yy + r_zz)
    const real rx = dx + ux * R, ry = dy + uy * R, rz = dz + uz * R;
    const real rxx = dxx + real(2) * ux * dx + ux * ux * R;
    const real ryy = dyy + real(2) * uy * dy + uy * uy * R;
    const real rzz = dzz + real(2) * uz * dz + uz * uz * R;
    g[1] += real(0.5) * (rxx + rx);
    g[2] += real(0.5) * (rxx - rx);
    g[3] += real(0.5) * (ryy + ry);
    g[4] += real(0.5) * (ryy - ry);
    g[5] += real(0.5) * (rzz + rz);
    g[6] += real(0.5) * (rzz - rz);
    g[0] += R - (rxx + ryy + rzz);
}

}  // namespace lbm
