// collide.cuh -- one-cell cascaded collisions of arXiv:1710.04751 in registers.
//
//   collide_flow      Appendix A: D3Q15 flow kernel g^_4..g^_14 with the body-force
//                     source S folded into the back-transform (Eq. 2a)
//   collide_thermal15 Sec. 2.2: D3Q15 scalar kernel h^_1..h^_14 (Eq. 13a, R = 0)
//   collide_thermal7  Appendix C: D3Q7 scalar kernel h^_1..h^_6
//
// Raw moments are accumulated with compile-time monomials (lattice.cuh), so every sum
// is a short chain of adds/subtracts; the back-transforms multiply by the integer
// entries of K only where they are non-zero.
#pragma once

#include "internal.h"
#include "lattice.cuh"

namespace lbm {

template <int M, int Q, typename real>
__device__ __forceinline__ real moment(const real (&p)[Q]) {
    real s = real(0);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        if (mono(M, a) == 1) s += p[a];
        else if (mono(M, a) == -1) s -= p[a];
    }
    return s;
}

// Flow collision (Appendix A).  f: pulled populations fbar, replaced by f~.  F: the
// body force (Boussinesq + uniform).  Returns u of Eq. (3).
//
// Source (reading of the forcing term the paper takes from its prior work): central
// moments of the Maxwellian forcing F.(xi-u)/(rho cs^2) f^M -- first order F, xyy/xxy/
// xxz = cs^2 F, the rest zero -- whose raw moments sigma' follow by the binomial theorem.
// S = K^-1 m^s is never formed: (K g^)_a + S_a = sum_b K_b(a) (g^_b + m^s_b / |K_b|^2).
template <typename real>
__device__ __forceinline__ void collide_flow(real (&f)[15], real Fx, real Fy, real Fz,
                                             const DevParams<real>& p, real& ux, real& uy,
                                             real& uz) {
    const real cs2 = real(1.0 / 3.0);
    const real half = real(0.5);
    const real rho = moment<M0>(f);
    const real jx = moment<MX>(f), jy = moment<MY>(f), jz = moment<MZ>(f);
    const real inv_rho = real(1) / rho;
    ux = (jx + half * Fx) * inv_rho;
    uy = (jy + half * Fy) * inv_rho;
    uz = (jz + half * Fz) * inv_rho;
    const real uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;

    // raw moments sigma' of the source
    const real sxy = ux * Fy + uy * Fx, sxz = ux * Fz + uz * Fx, syz = uy * Fz + uz * Fy;
    const real sxx = real(2) * ux * Fx, syy = real(2) * uy * Fy, szz = real(2) * uz * Fz;
    const real sxyy = cs2 * Fx + uyy * Fx + real(2) * ux * uy * Fy;
    const real sxxy = cs2 * Fy + uxx * Fy + real(2) * ux * uy * Fx;
    const real sxxz = cs2 * Fz + uxx * Fz + real(2) * ux * uz * Fx;
    const real sxyz = ux * uy * Fz + ux * uz * Fy + uy * uz * Fx;
    const real sxxyy = real(2) * cs2 * (ux * Fx + uy * Fy) + real(2) * ux * uyy * Fx +
                       real(2) * uxx * uy * Fy;

    // eta' = raw moments of (fbar + S)
    const real e_x = jx + Fx, e_y = jy + Fy;
    const real exy = moment<MXY>(f) + sxy, exz = moment<MXZ>(f) + sxz, eyz = moment<MYZ>(f) + syz;
    const real exx = moment<MXX>(f) + sxx, eyy = moment<MYY>(f) + syy, ezz = moment<MZZ>(f) + szz;
    const real exyy = moment<MXYY>(f) + sxyy, exxy = moment<MXXY>(f) + sxxy;
    const real exxz = moment<MXXZ>(f) + sxxz, exyz = moment<MXYZ>(f) + sxyz;
    const real exxyy = moment<MXXYY>(f) + sxxyy;

    const real* om = p.om_f;
    const real g4 = om[4] * real(0.125) * (-exy + rho * ux * uy + half * (Fx * uy + Fy * ux));
    const real g5 = om[5] * real(0.125) * (-exz + rho * ux * uz + half * (Fx * uz + Fz * ux));
    const real g6 = om[6] * real(0.125) * (-eyz + rho * uy * uz + half * (Fy * uz + Fz * uy));
    const real g7 = om[7] * real(0.25) * (-(exx - eyy) + rho * (uxx - uyy) + (Fx * ux - Fy * uy));
    const real g8 = om[8] * real(1.0 / 12.0) *
                    (-(exx + eyy - real(2) * ezz) + rho * (uxx + uyy - real(2) * uzz) +
                     (Fx * ux + Fy * uy - real(2) * Fz * uz));
    const real g9 = om[9] * real(1.0 / 18.0) *
                    (-(exx + eyy + ezz) + rho * (uxx + uyy + uzz) + (Fx * ux + Fy * uy + Fz * uz) +
                     rho);
    const real g10 = om[10] * real(0.0625) *
                         (-exyy + real(2) * uy * exy + ux * eyy - real(2) * rho * ux * uyy -
                          half * Fx * uyy - Fy * uy * ux) +
                     uy * g4 + real(0.125) * ux * (-g7 + g8 + real(3) * g9);
    const real g11 = om[11] * real(0.0625) *
                         (-exxy + real(2) * ux * exy + uy * exx - real(2) * rho * uxx * uy -
                          half * Fy * uxx - Fx * ux * uy) +
                     ux * g4 + real(0.125) * uy * (g7 + g8 + real(3) * g9);
    const real g12 = om[12] * real(0.0625) *
                         (-exxz + real(2) * ux * exz + uz * exx - real(2) * rho * uxx * uz -
                          half * Fz * uxx - Fx * ux * uz) +
                     ux * g5 + real(0.125) * uz * (g7 + g8 + real(3) * g9);
    const real g13 = om[13] * real(0.125) *
                         (-exyz + ux * eyz + uy * exz + uz * exy - real(2) * rho * ux * uy * uz -
                          half * (Fx * uy * uz + Fy * ux * uz + Fz * ux * uy)) +
                     uz * g4 + uy * g5 + ux * g6;
    // equilibrium of the 4th-order central moment: factorised from the post-collision
    // second-order central moments (mode 0) or Maxwellian rho cs^4 (mode 1)
    real E;
    if (p.e4_mode == 1) {
        E = rho * real(1.0 / 9.0);
    } else {
        const real kxx = exx - real(2) * ux * e_x + uxx * rho + real(2) * g7 + real(2) * g8 +
                         real(6) * g9;
        const real kyy = eyy - real(2) * uy * e_y + uyy * rho - real(2) * g7 + real(2) * g8 +
                         real(6) * g9;
        E = kxx * kyy * inv_rho;
    }
    const real g14 = om[14] * real(0.0625) *
                         (-exxyy + real(2) * ux * exyy + real(2) * uy * exxy - uxx * eyy -
                          uyy * exx - real(4) * ux * uy * exy + E + real(3) * rho * uxx * uyy +
                          Fx * ux * uyy + Fy * uy * uxx) -
                     real(2) * ux * uy * g4 + real(0.125) * (uxx - uyy) * g7 -
                     real(0.125) * (uxx + uyy) * g8 - (real(0.375) * (uxx + uyy) + half) * g9 +
                     real(2) * ux * g10 + real(2) * uy * g11;

    // c_b = g^_b + m^s_b / |K_b|^2 (m^s: projections of S on K; g^_0..3 = 0, m^s_0 = 0)
    real c[15];
    c[0] = real(0);
    c[1] = real(0.1) * Fx;
    c[2] = real(0.1) * Fy;
    c[3] = real(0.1) * Fz;
    c[4] = g4 + real(0.125) * sxy;
    c[5] = g5 + real(0.125) * sxz;
    c[6] = g6 + real(0.125) * syz;
    c[7] = g7 + real(0.25) * (sxx - syy);
    c[8] = g8 + real(1.0 / 12.0) * (sxx + syy - real(2) * szz);
    c[9] = g9 + real(1.0 / 18.0) * (sxx + syy + szz);
    c[10] = g10 + real(1.0 / 160.0) * (real(10) * sxyy - real(8) * Fx);
    c[11] = g11 + real(1.0 / 160.0) * (real(10) * sxxy - real(8) * Fy);
    c[12] = g12 + real(1.0 / 160.0) * (real(10) * sxxz - real(8) * Fz);
    c[13] = g13 + real(0.125) * sxyz;
    c[14] = g14 + real(1.0 / 1440.0) * (real(90) * sxxyy - real(40) * (sxx + syy + szz));
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        real acc = real(0);
#pragma unroll
        for (int b = 1; b < 15; ++b) {
            if (k15(b, a) != 0) acc += real(k15(b, a)) * c[b];
        }
        f[a] += acc;
    }
}

// Thermal D3Q15 collision (Sec. 2.2) with R = 0: g becomes g~; u from the flow.
template <typename real>
__device__ __forceinline__ void collide_thermal15(real (&g)[15], real ux, real uy, real uz,
                                                  const DevParams<real>& p) {
    const real half = real(0.5);
    const real phi = moment<M0>(g);
    const real kx = moment<MX>(g), ky = moment<MY>(g), kz = moment<MZ>(g);
    const real kxy = moment<MXY>(g), kxz = moment<MXZ>(g), kyz = moment<MYZ>(g);
    const real kxx = moment<MXX>(g), kyy = moment<MYY>(g), kzz = moment<MZZ>(g);
    const real kxyy = moment<MXYY>(g), kxxy = moment<MXXY>(g), kxxz = moment<MXXZ>(g);
    const real kxyz = moment<MXYZ>(g), kxxyy = moment<MXXYY>(g);
    const real uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
    const real cs2 = p.cs2_phi;
    const real* om = p.om_g;
    real h[15];
    h[0] = real(0);
    h[1] = om[1] * real(0.1) * (phi * ux - kx);
    h[2] = om[2] * real(0.1) * (phi * uy - ky);
    h[3] = om[3] * real(0.1) * (phi * uz - kz);
    h[4] = om[4] * real(0.125) * (-kxy + uy * kx + ux * ky - phi * ux * uy) +
           real(1.25) * (uy * h[1] + ux * h[2]);
    h[5] = om[5] * real(0.125) * (-kxz + uz * kx + ux * kz - phi * ux * uz) +
           real(1.25) * (uz * h[1] + ux * h[3]);
    h[6] = om[6] * real(0.125) * (-kyz + uz * ky + uy * kz - phi * uy * uz) +
           real(1.25) * (uz * h[2] + uy * h[3]);
    h[7] = om[7] * real(0.25) *
               (-(kxx - kyy) + real(2) * (ux * kx - uy * ky) - phi * (uxx - uyy)) +
           real(5) * (ux * h[1] - uy * h[2]);
    h[8] = om[8] * real(1.0 / 12.0) *
               (-(kxx + kyy - real(2) * kzz) + real(2) * (ux * kx + uy * ky - real(2) * uz * kz) -
                phi * (uxx + uyy - real(2) * uzz)) +
           real(5.0 / 3.0) * (ux * h[1] + uy * h[2] - real(2) * uz * h[3]);
    h[9] = om[9] * real(1.0 / 18.0) *
               (real(3) * cs2 * phi - (kxx + kyy + kzz) + real(2) * (ux * kx + uy * ky + uz * kz) -
                phi * (uxx + uyy + uzz)) +
           real(10.0 / 9.0) * (ux * h[1] + uy * h[2] + uz * h[3]);
    h[10] = om[10] * real(0.0625) *
                (-kxyy + real(2) * uy * kxy - uyy * kx + ux * kyy - real(2) * ux * uy * ky +
                 phi * ux * uyy) -
            (real(0.625) * uyy + half) * h[1] - real(1.25) * ux * uy * h[2] + uy * h[4] +
            real(0.125) * ux * (-h[7] + h[8] + real(3) * h[9]);
    h[11] = om[11] * real(0.0625) *
                (-kxxy + real(2) * ux * kxy + uy * kxx - uxx * ky - real(2) * ux * uy * kx +
                 phi * uxx * uy) -
            real(1.25) * ux * uy * h[1] - (real(0.625) * uxx + half) * h[2] + ux * h[4] +
            real(0.125) * uy * (h[7] + h[8] + real(3) * h[9]);
    h[12] = om[12] * real(0.0625) *
                (-kxxz + real(2) * ux * kxz + uz * kxx - real(2) * ux * uz * kx - uxx * kz +
                 phi * uxx * uz) -
            real(1.25) * ux * uz * h[1] - (real(0.625) * uxx + half) * h[3] + ux * h[5] +
            real(0.125) * uz * (h[7] + h[8] + real(3) * h[9]);
    h[13] = om[13] * real(0.125) *
                (-kxyz + ux * kyz + uy * kxz + uz * kxy - uy * uz * kx - ux * uz * ky -
                 ux * uy * kz + phi * ux * uy * uz) -
            real(1.25) * (uy * uz * h[1] + ux * uz * h[2] + ux * uy * h[3]) + uz * h[4] +
            uy * h[5] + ux * h[6];
    h[14] = om[14] * real(0.0625) *
                (-kxxyy + real(2) * uy * kxxy + real(2) * ux * kxyy - uyy * kxx - uxx * kyy -
                 real(4) * ux * uy * kxy + real(2) * ux * uyy * kx + real(2) * uxx * uy * ky +
                 cs2 * cs2 * phi - phi * uxx * uyy) +
            real(1.25) * (ux * uyy * h[1] + uxx * uy * h[2]) - real(2) * ux * uy * h[4] +
            real(0.125) * (uxx - uyy) * h[7] - real(0.125) * (uxx + uyy) * h[8] -
            (real(0.375) * (uxx + uyy) + half) * h[9] + real(2) * (ux * h[10] + uy * h[11]) +
            uy * h[2] + ux * h[1];
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        real acc = real(0);
#pragma unroll
        for (int b = 1; b < 15; ++b) {
            if (k15(b, a) != 0) acc += real(k15(b, a)) * h[b];
        }
        g[a] += acc;
    }
}

// Thermal D3Q7 collision (Appendix C) with R = 0.
template <typename real>
__device__ __forceinline__ void collide_thermal7(real (&g)[7], real ux, real uy, real uz,
                                                 const DevParams<real>& p) {
    const real phi = moment<M0>(g);
    const real kx = moment<MX>(g), ky = moment<MY>(g), kz = moment<MZ>(g);
    const real kxx = moment<MXX>(g), kyy = moment<MYY>(g), kzz = moment<MZZ>(g);
    const real uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
    const real* om = p.om_g;
    real h[7];
    h[0] = real(0);
    h[1] = om[1] * real(0.5) * (phi * ux - kx);
    h[2] = om[2] * real(0.5) * (phi * uy - ky);
    h[3] = om[3] * real(0.5) * (phi * uz - kz);
    h[4] = om[4] * real(0.25) *
               (-(kxx - kyy) + real(2) * (ux * kx - uy * ky) - phi * (uxx - uyy)) +
           ux * h[1] - uy * h[2];
    h[5] = om[5] * real(1.0 / 12.0) *
               (-(kxx + kyy - real(2) * kzz) + real(2) * (ux * kx + uy * ky - real(2) * uz * kz) -
                phi * (uxx + uyy - real(2) * uzz)) +
           real(1.0 / 3.0) * (ux * h[1] + uy * h[2] - real(2) * uz * h[3]);
    h[6] = om[6] * real(1.0 / 6.0) *
               (real(3) * p.cs2_phi * phi - (kxx + kyy + kzz) +
                real(2) * (ux * kx + uy * ky + uz * kz) - phi * (uxx + uyy + uzz)) +
           real(2.0 / 3.0) * (ux * h[1] + uy * h[2] + uz * h[3]);
#pragma unroll
    for (int a = 0; a < 7; ++a) {
        real acc = real(0);
#pragma unroll
        for (int b = 1; b < 7; ++b) {
            if (k7(b, a) != 0) acc += real(k7(b, a)) * h[b];
        }
        g[a] += acc;
    }
}

}  // namespace lbm
