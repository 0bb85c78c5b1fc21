/*
 * lbm_oracle.c -- FP64 CPU oracle of the cascaded central-moment thermal LBM of
 * Hajabdollahi & Premnath, "Central Moments-based Cascaded Lattice Boltzmann Method
 * for Thermal Convective Flows in Three-Dimensions" (arXiv:1710.04751).
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA library is checked against.  It
 * shares no code with the CUDA path and must never be called by the product.
 *
 * Every formula below is written from the paper in its own order and notation:
 *   - velocities, basis and collision matrix K ........ Sec. 2.2, Eqs. (5)-(6) block
 *   - flow cascade g^_4..g^_14 and post-collision ...... Appendix A
 *   - thermal D3Q15 cascade h^_1..h^_14, back-transform  Sec. 2.2 (Eq. 21 notation)
 *   - thermal D3Q7 cascade and back-transform .......... Appendix C
 *   - macroscopic variables ............................ Eq. (3), Eq. (25)
 *   - Boussinesq force, boundary conditions, Nu ........ Sec. 3
 * Where the paper is silent the oracle follows these readings (shared with the CUDA
 * library, stated again next to the code that uses them):
 *   R1  4th-order flow equilibrium E = kxx~ * kyy~ / rho (mode 0) or rho*cs^4 (mode 1)
 *   R2  flow source S: central moments of the Maxwellian forcing term, 1st order F,
 *       3rd order cs^2 F, all others zero, mapped to populations through K^-1
 *   R3  flow omega_4..omega_8 (shear) set the viscosity, omega_9..omega_14 = 1
 *   R4  thermal omega_1..omega_3 set the diffusivity, the rest = 1
 *   R5  no-slip: half-way bounce-back
 *   R6  Dirichlet T: anti-bounce-back g = -g~_opp + 2 w_a T_w
 *   R7  adiabatic: specular reflection of g (mode 1, default) or bounce-back (mode 0);
 *       a link that leaves through an x face is Dirichlet
 *   R8  F = (0, 0, g beta (T - T0)), rho0 = 1, T0 = (T_hot + T_cold)/2
 *   R9  stored arrays are post-collision; a step is pull, then collide
 *   R11 Nu from the one-sided stencil (9 T1 - T2 - 8 Tw)/3 at half-way walls
 *   R12 peak velocities on the centrelines of the symmetry plane
 *
 * Readings the paper does not fix, and what pins them: the fourth-order equilibrium E of
 * R1 is held to Table 1, the paper's only arbiter (both forms agree within the table's
 * printed digits, and the implemented one is nearer to it); the third-order source
 * moments of R2 cancel in the collision at the paper's unit third-order rates (they move
 * nothing unless those rates are changed).  Form B (oracle/formb.py) restates the same
 * readings, so the Form A == Form B tests check their transcription.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (oracle/build.py).
 * OpenMP only splits the loop over z-planes; each cell's arithmetic is unchanged.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------ */
/* Lattice tables (Sec. 2.2, D3Q15 velocity components; App. C, D3Q7 subset).      */
/* ------------------------------------------------------------------------------ */

static const int EX[15] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
static const int EY[15] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
static const int EZ[15] = {0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1};

void orc_velocities(int q, int* ex, int* ey, int* ez) {
    for (int a = 0; a < q; ++a) { ex[a] = EX[a]; ey[a] = EY[a]; ez[a] = EZ[a]; }
}

int orc_opposite(int q, int a) {
    for (int b = 0; b < q; ++b)
        if (EX[b] == -EX[a] && EY[b] == -EY[a] && EZ[b] == -EZ[a]) return b;
    return -1;
}

/* D3Q15 orthogonal collision matrix K (Sec. 2.2, the Gram-Schmidt basis K_0..K_14). */
void orc_kmatrix15(int* K) {
    for (int a = 0; a < 15; ++a) {
        int x = EX[a], y = EY[a], z = EZ[a];
        int e2 = x * x + y * y + z * z;
        K[0 * 15 + a] = 1;
        K[1 * 15 + a] = x;
        K[2 * 15 + a] = y;
        K[3 * 15 + a] = z;
        K[4 * 15 + a] = x * y;
        K[5 * 15 + a] = x * z;
        K[6 * 15 + a] = y * z;
        K[7 * 15 + a] = x * x - y * y;
        K[8 * 15 + a] = e2 - 3 * z * z;
        K[9 * 15 + a] = e2 - 2;
        K[10 * 15 + a] = 5 * x * e2 - 13 * x;
        K[11 * 15 + a] = 5 * y * e2 - 13 * y;
        K[12 * 15 + a] = 5 * z * e2 - 13 * z;
        K[13 * 15 + a] = x * y * z;
        K[14 * 15 + a] = 30 * (x * x * y * y + x * x * z * z + y * y * z * z) - 40 * e2 + 32;
    }
}

/* D3Q7 orthogonal collision matrix (Appendix C, K_0..K_6). */
void orc_kmatrix7(int* K) {
    for (int a = 0; a < 7; ++a) {
        int x = EX[a], y = EY[a], z = EZ[a];
        int e2 = x * x + y * y + z * z;
        K[0 * 7 + a] = 1;
        K[1 * 7 + a] = x;
        K[2 * 7 + a] = y;
        K[3 * 7 + a] = z;
        K[4 * 7 + a] = x * x - y * y;
        K[5 * 7 + a] = 2 * (x * x - z * z) - (x * x - y * y);
        K[6 * 7 + a] = 7 * e2 - 6;
    }
}

/* Tables derived once, when the library is loaded, from the definitions above. */
static int K15[225], K7[49], OPP[15];
static double NORM15[15], NORM7[7];
static double MONO[15][15];
static double monomial(int m, int a);

static void knorms(const int* K, int q, double* norm) {
    for (int b = 0; b < q; ++b) {
        double s = 0.0;
        for (int a = 0; a < q; ++a) s += (double)(K[b * q + a] * K[b * q + a]);
        norm[b] = s;
    }
}

/* Rest-state populations of the flow equilibrium (rho = 1, u = 0, cs^2 = 1/3): the
 * populations whose central moments are 1, 0, cs^2 (diagonal 2nd order) and cs^4
 * (xxyy).  With w0 + 6 w1 + 8 w7 = 1, 2 w1 + 8 w7 = cs^2, 8 w7 = cs^4. */
void orc_weights_flow(double w[15]) {
    const double cs2 = 1.0 / 3.0;
    double w7 = cs2 * cs2 / 8.0, w1 = (cs2 - cs2 * cs2) / 2.0;
    double w0 = 1.0 - 6.0 * w1 - 8.0 * w7;
    for (int a = 0; a < 15; ++a) w[a] = (a == 0) ? w0 : (a < 7 ? w1 : w7);
}

/* Rest-state populations of the thermal equilibrium (Eq. 15 with u = 0, phi = 1). */
void orc_weights_thermal(int q, double cs2, double* w) {
    if (q == 15) {
        double w7 = cs2 * cs2 / 8.0, w1 = (cs2 - cs2 * cs2) / 2.0;
        double w0 = 1.0 - 6.0 * w1 - 8.0 * w7;
        for (int a = 0; a < 15; ++a) w[a] = (a == 0) ? w0 : (a < 7 ? w1 : w7);
    } else {
        /* D3Q7: sum w = 1 and 2 w1 = cs^2 (the trace 3 cs^2 phi over six links). */
        double w1 = cs2 / 2.0;
        double w0 = 1.0 - 6.0 * w1;
        for (int a = 0; a < 7; ++a) w[a] = (a == 0) ? w0 : w1;
    }
}

/* The 15 raw-moment monomials used by the cascades (Eq. 17 / App. A notation). */
enum { M0, MX, MY, MZ, MXY, MXZ, MYZ, MXX, MYY, MZZ, MXYY, MXXY, MXXZ, MXYZ, MXXYY, NMOM };

static double monomial(int m, int a) {
    double x = EX[a], y = EY[a], z = EZ[a];
    switch (m) {
    case M0: return 1.0;
    case MX: return x;
    case MY: return y;
    case MZ: return z;
    case MXY: return x * y;
    case MXZ: return x * z;
    case MYZ: return y * z;
    case MXX: return x * x;
    case MYY: return y * y;
    case MZZ: return z * z;
    case MXYY: return x * y * y;
    case MXXY: return x * x * y;
    case MXXZ: return x * x * z;
    case MXYZ: return x * y * z;
    case MXXYY: return x * x * y * y;
    }
    return 0.0;
}

static void raw_moments(const double* p, int q, double* mom) {
    for (int m = 0; m < NMOM; ++m) {
        double s = 0.0;
        for (int a = 0; a < q; ++a) s += p[a] * MONO[m][a];
        mom[m] = s;
    }
}

__attribute__((constructor)) static void orc_tables_init(void) {
    orc_kmatrix15(K15);
    orc_kmatrix7(K7);
    knorms(K15, 15, NORM15);
    knorms(K7, 7, NORM7);
    for (int a = 0; a < 15; ++a) OPP[a] = orc_opposite(15, a);
    for (int m = 0; m < NMOM; ++m)
        for (int a = 0; a < 15; ++a) MONO[m][a] = monomial(m, a);
}

/* ------------------------------------------------------------------------------ */
/* Flow source S_alpha (reading R2).                                               */
/* ------------------------------------------------------------------------------ */
/* The paper defers S_alpha to its prior work.  By analogy with its own construction
 * for the scalar source (Eqs. 8, 16, 19 and Appendix B), the central moments of the
 * forcing term are those of the Maxwellian forcing F.(xi - u)/(rho cs^2) f^M:
 *   Gamma_x,y,z = F_x,y,z ; Gamma_xyy = cs^2 F_x ; Gamma_xxy = cs^2 F_y ;
 *   Gamma_xxz = cs^2 F_z ; every other central moment (0, 2nd, xyz, xxyy) = 0.
 * The binomial theorem turns them into raw moments sigma', which are projected on K
 * (m^s_b = <K_b|S>) and inverted through the orthogonality of K, as the paper does
 * for the scalar source (Appendix B). */
static void source_from_raw15(const double* s, double S[15]);

void orc_flow_source(const double F[3], const double u[3], double S[15]) {
    const double cs2 = 1.0 / 3.0;
    double Fx = F[0], Fy = F[1], Fz = F[2];
    double ux = u[0], uy = u[1], uz = u[2];
    double s[NMOM];
    s[M0] = 0.0;
    s[MX] = Fx;
    s[MY] = Fy;
    s[MZ] = Fz;
    s[MXY] = ux * Fy + uy * Fx;
    s[MXZ] = ux * Fz + uz * Fx;
    s[MYZ] = uy * Fz + uz * Fy;
    s[MXX] = 2.0 * ux * Fx;
    s[MYY] = 2.0 * uy * Fy;
    s[MZZ] = 2.0 * uz * Fz;
    s[MXYY] = cs2 * Fx + uy * uy * Fx + 2.0 * ux * uy * Fy;
    s[MXXY] = cs2 * Fy + ux * ux * Fy + 2.0 * ux * uy * Fx;
    s[MXXZ] = cs2 * Fz + ux * ux * Fz + 2.0 * ux * uz * Fx;
    s[MXYZ] = ux * uy * Fz + ux * uz * Fy + uy * uz * Fx;
    s[MXXYY] = 2.0 * cs2 * (ux * Fx + uy * Fy) + 2.0 * ux * uy * uy * Fx + 2.0 * ux * ux * uy * Fy;

    source_from_raw15(s, S);
}

/* S_a = sum_b K_b(a) m^s_b / |K_b|^2 for the raw moments s[] of S (the inversion the
 * paper uses for the scalar source, Eq. 19 and Appendix B).  The projections m^s_b use
 * the identities of the D3Q15 lattice: e_x^3 = e_x, e_x e_z^2 = e_x e_y^2, e_y e_z^2 =
 * e_x^2 e_y, e_y^2 e_z = e_x^2 e_z, and all three products e_i^2 e_j^2 coincide. */
static void source_from_raw15(const double* s, double S[15]) {
    double m[15];
    m[0] = s[M0];
    m[1] = s[MX];
    m[2] = s[MY];
    m[3] = s[MZ];
    m[4] = s[MXY];
    m[5] = s[MXZ];
    m[6] = s[MYZ];
    m[7] = s[MXX] - s[MYY];
    m[8] = s[MXX] + s[MYY] - 2.0 * s[MZZ];
    m[9] = s[MXX] + s[MYY] + s[MZZ] - 2.0 * s[M0];
    m[10] = 5.0 * (s[MX] + 2.0 * s[MXYY]) - 13.0 * s[MX];
    m[11] = 5.0 * (s[MY] + 2.0 * s[MXXY]) - 13.0 * s[MY];
    m[12] = 5.0 * (s[MZ] + 2.0 * s[MXXZ]) - 13.0 * s[MZ];
    m[13] = s[MXYZ];
    m[14] = 30.0 * 3.0 * s[MXXYY] - 40.0 * (s[MXX] + s[MYY] + s[MZZ]) + 32.0 * s[M0];

    for (int a = 0; a < 15; ++a) {
        double acc = 0.0;
        for (int b = 0; b < 15; ++b) acc += K15[b * 15 + a] * m[b] / NORM15[b];
        S[a] = acc;
    }
}

/* Raw moments of the scalar source (Sec. 2.2): its only non-zero central moment is the
 * zeroth, R (Eq. 16), so by the binomial theorem sigma'_{x^m y^n z^p} = u_x^m u_y^n u_z^p R
 * (the list printed after Eq. 17). */
static void scalar_source_raw(double R, const double u[3], double* s) {
    double ux = u[0], uy = u[1], uz = u[2];
    s[M0] = R;
    s[MX] = ux * R;
    s[MY] = uy * R;
    s[MZ] = uz * R;
    s[MXY] = ux * uy * R;
    s[MXZ] = ux * uz * R;
    s[MYZ] = uy * uz * R;
    s[MXX] = ux * ux * R;
    s[MYY] = uy * uy * R;
    s[MZZ] = uz * uz * R;
    s[MXYY] = ux * uy * uy * R;
    s[MXXY] = ux * ux * uy * R;
    s[MXXZ] = ux * ux * uz * R;
    s[MXYZ] = ux * uy * uz * R;
    s[MXXYY] = ux * ux * uy * uy * R;
}

/* Scalar source in velocity space, D3Q15 (Appendix B, S^phi = K^-1 m^s) and D3Q7
 * (Appendix C, rows 3 and 4 with m^s_2 as K^-1 gives, m^s_6 = (7 u^2 - 6) R). */
void orc_scalar_source(int q, double R, const double u[3], double* S) {
    double s[NMOM];
    scalar_source_raw(R, u, s);
    if (q == 15) {
        source_from_raw15(s, S);
    } else {
        double m[7];
        m[0] = s[M0];
        m[1] = s[MX];
        m[2] = s[MY];
        m[3] = s[MZ];
        m[4] = s[MXX] - s[MYY];
        m[5] = s[MXX] + s[MYY] - 2.0 * s[MZZ];
        m[6] = 7.0 * (s[MXX] + s[MYY] + s[MZZ]) - 6.0 * s[M0];
        for (int a = 0; a < 7; ++a) {
            double acc = 0.0;
            for (int b = 0; b < 7; ++b) acc += K7[b * 7 + a] * m[b] / NORM7[b];
            S[a] = acc;
        }
    }
}

/* ------------------------------------------------------------------------------ */
/* Flow collision: Appendix A (Eq. 2a with the kernel g^_0..g^_14).                */
/* ------------------------------------------------------------------------------ */
void orc_collide_flow(const double fbar[15], const double F[3], const double om[15],
                      int e4_mode, double out[15], double* rho_out, double u_out[3]) {
    /* Eq. (3): rho = sum fbar, rho u = sum fbar e + F/2. */
    double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int a = 0; a < 15; ++a) {
        rho += fbar[a];
        jx += fbar[a] * EX[a];
        jy += fbar[a] * EY[a];
        jz += fbar[a] * EZ[a];
    }
    double ux = (jx + 0.5 * F[0]) / rho;
    double uy = (jy + 0.5 * F[1]) / rho;
    double uz = (jz + 0.5 * F[2]) / rho;
    double u[3] = {ux, uy, uz};

    double S[15];
    orc_flow_source(F, u, S);

    /* kappa-bar' (raw moments of fbar), sigma' (raw moments of S), eta = kappa-bar' + sigma'. */
    double kb[NMOM], sg[NMOM], et[NMOM];
    raw_moments(fbar, 15, kb);
    raw_moments(S, 15, sg);
    for (int m = 0; m < NMOM; ++m) et[m] = kb[m] + sg[m];
    double sx = sg[MX], sy = sg[MY], sz = sg[MZ];

    double g[15];
    g[0] = g[1] = g[2] = g[3] = 0.0;
    g[4] = om[4] / 8.0 * (-et[MXY] + rho * ux * uy + 0.5 * (sx * uy + sy * ux));
    g[5] = om[5] / 8.0 * (-et[MXZ] + rho * ux * uz + 0.5 * (sx * uz + sz * ux));
    g[6] = om[6] / 8.0 * (-et[MYZ] + rho * uy * uz + 0.5 * (sy * uz + sz * uy));
    g[7] = om[7] / 4.0 *
           (-(et[MXX] - et[MYY]) + rho * (ux * ux - uy * uy) + (sx * ux - sy * uy));
    g[8] = om[8] / 12.0 *
           (-(et[MXX] + et[MYY] - 2.0 * et[MZZ]) + rho * (ux * ux + uy * uy - 2.0 * uz * uz) +
            (sx * ux + sy * uy - 2.0 * sz * uz));
    g[9] = om[9] / 18.0 *
           (-(et[MXX] + et[MYY] + et[MZZ]) + rho * (ux * ux + uy * uy + uz * uz) +
            (sx * ux + sy * uy + sz * uz) + rho);
    g[10] = om[10] / 16.0 *
                (-et[MXYY] + 2.0 * uy * et[MXY] + ux * et[MYY] - 2.0 * rho * ux * uy * uy -
                 0.5 * sx * uy * uy - sy * uy * ux) +
            uy * g[4] + 0.125 * ux * (-g[7] + g[8] + 3.0 * g[9]);
    g[11] = om[11] / 16.0 *
                (-et[MXXY] + 2.0 * ux * et[MXY] + uy * et[MXX] - 2.0 * rho * ux * ux * uy -
                 0.5 * sy * ux * ux - sx * ux * uy) +
            ux * g[4] + 0.125 * uy * (g[7] + g[8] + 3.0 * g[9]);
    g[12] = om[12] / 16.0 *
                (-et[MXXZ] + 2.0 * ux * et[MXZ] + uz * et[MXX] - 2.0 * rho * ux * ux * uz -
                 0.5 * sz * ux * ux - sx * ux * uz) +
            ux * g[5] + 0.125 * uz * (g[7] + g[8] + 3.0 * g[9]);
    g[13] = om[13] / 8.0 *
                (-et[MXYZ] + ux * et[MYZ] + uy * et[MXZ] + uz * et[MXY] -
                 2.0 * rho * ux * uy * uz - 0.5 * (sx * uy * uz + sy * ux * uz + sz * ux * uy)) +
            uz * g[4] + uy * g[5] + ux * g[6];

    /* Equilibrium of the 4th-order central moment (reading R1).  kxx~ and kyy~ are the
     * post-collision 2nd-order central moments: those of (fbar + S) about u plus the
     * contribution of K g^ (2 g7 + 2 g8 + 6 g9 and -2 g7 + 2 g8 + 6 g9, Sec. 2.2 list of
     * raw moments of K h^ applied to g^ with g^_0..3 = 0). */
    double E;
    if (e4_mode == 1) {
        E = rho / 9.0;
    } else {
        double cxx = et[MXX] - 2.0 * ux * et[MX] + ux * ux * et[M0];
        double cyy = et[MYY] - 2.0 * uy * et[MY] + uy * uy * et[M0];
        double kxx_t = cxx + 2.0 * g[7] + 2.0 * g[8] + 6.0 * g[9];
        double kyy_t = cyy - 2.0 * g[7] + 2.0 * g[8] + 6.0 * g[9];
        E = kxx_t * kyy_t / rho;
    }
    g[14] = om[14] / 16.0 *
                (-et[MXXYY] + 2.0 * ux * et[MXYY] + 2.0 * uy * et[MXXY] - ux * ux * et[MYY] -
                 uy * uy * et[MXX] - 4.0 * ux * uy * et[MXY] + E + 3.0 * rho * ux * ux * uy * uy +
                 sx * ux * uy * uy + sy * uy * ux * ux) -
            2.0 * ux * uy * g[4] + 0.125 * (ux * ux - uy * uy) * g[7] +
            0.125 * (-ux * ux - uy * uy) * g[8] +
            (0.375 * (-ux * ux - uy * uy) - 0.5) * g[9] + 2.0 * ux * g[10] + 2.0 * uy * g[11];

    /* Eq. (2a): f~ = fbar + (K g^) + S. */
    for (int a = 0; a < 15; ++a) {
        double kg = 0.0;
        for (int b = 0; b < 15; ++b) kg += K15[b * 15 + a] * g[b];
        out[a] = fbar[a] + kg + S[a];
    }
    if (rho_out) *rho_out = rho;
    if (u_out) { u_out[0] = ux; u_out[1] = uy; u_out[2] = uz; }
}

/* ------------------------------------------------------------------------------ */
/* Thermal collision, D3Q15: Sec. 2.2 (kernel h^_0..h^_14, Eq. 13a) with source R.  */
/* ------------------------------------------------------------------------------ */
void orc_collide_thermal15(const double gbar[15], const double u[3], const double om[15],
                           double cs2, double R, double out[15]) {
    double ux = u[0], uy = u[1], uz = u[2];
    double k[NMOM], sg[NMOM], e[NMOM];
    raw_moments(gbar, 15, k);      /* kappa-bar' (Eq. 17) */
    scalar_source_raw(R, u, sg);   /* sigma' */
    for (int m = 0; m < NMOM; ++m) e[m] = k[m] + sg[m]; /* eta-bar' = kappa-bar' + sigma' (Eq. 21) */
    double phi = k[M0] + 0.5 * R;  /* Eq. (25) */
    double pr = phi + 0.5 * R;     /* the (phi + R/2) of the kernel */
    double cs4 = cs2 * cs2;
    double h[15];
    h[0] = 0.0;
    h[1] = om[1] / 10.0 * (phi * ux - k[MX] - ux * 0.5 * R);
    h[2] = om[2] / 10.0 * (phi * uy - k[MY] - uy * 0.5 * R);
    h[3] = om[3] / 10.0 * (phi * uz - k[MZ] - uz * 0.5 * R);
    h[4] = om[4] / 8.0 * (-e[MXY] + uy * e[MX] + ux * e[MY] - pr * ux * uy) +
           1.25 * (uy * h[1] + ux * h[2]);
    h[5] = om[5] / 8.0 * (-e[MXZ] + uz * e[MX] + ux * e[MZ] - pr * ux * uz) +
           1.25 * (uz * h[1] + ux * h[3]);
    h[6] = om[6] / 8.0 * (-e[MYZ] + uz * e[MY] + uy * e[MZ] - pr * uy * uz) +
           1.25 * (uz * h[2] + uy * h[3]);
    h[7] = om[7] / 4.0 *
               (-(e[MXX] - e[MYY]) + 2.0 * (ux * e[MX] - uy * e[MY]) - pr * (ux * ux - uy * uy)) +
           5.0 * (ux * h[1] - uy * h[2]);
    h[8] = om[8] / 12.0 *
               (-(e[MXX] + e[MYY] - 2.0 * e[MZZ]) + 2.0 * (ux * e[MX] + uy * e[MY] - 2.0 * uz * e[MZ]) -
                pr * (ux * ux + uy * uy - 2.0 * uz * uz)) +
           (5.0 / 3.0) * (ux * h[1] + uy * h[2] - 2.0 * uz * h[3]);
    h[9] = om[9] / 18.0 *
               (3.0 * cs2 * phi - (e[MXX] + e[MYY] + e[MZZ]) +
                2.0 * (ux * e[MX] + uy * e[MY] + uz * e[MZ]) - pr * (ux * ux + uy * uy + uz * uz)) +
           (10.0 / 9.0) * (ux * h[1] + uy * h[2] + uz * h[3]);
    h[10] = om[10] / 16.0 *
                (-e[MXYY] + 2.0 * uy * e[MXY] - uy * uy * e[MX] + ux * e[MYY] -
                 2.0 * ux * uy * e[MY] + pr * ux * uy * uy) -
            (0.625 * uy * uy + 0.5) * h[1] - 1.25 * ux * uy * h[2] + uy * h[4] +
            0.125 * ux * (-h[7] + h[8] + 3.0 * h[9]);
    h[11] = om[11] / 16.0 *
                (-e[MXXY] + 2.0 * ux * e[MXY] + uy * e[MXX] - ux * ux * e[MY] -
                 2.0 * ux * uy * e[MX] + pr * ux * ux * uy) -
            1.25 * ux * uy * h[1] - (0.625 * ux * ux + 0.5) * h[2] + ux * h[4] +
            0.125 * uy * (h[7] + h[8] + 3.0 * h[9]);
    h[12] = om[12] / 16.0 *
                (-e[MXXZ] + 2.0 * ux * e[MXZ] + uz * e[MXX] - 2.0 * ux * uz * e[MX] -
                 ux * ux * e[MZ] + pr * ux * ux * uz) -
            1.25 * ux * uz * h[1] - (0.625 * ux * ux + 0.5) * h[3] + ux * h[5] +
            0.125 * uz * (h[7] + h[8] + 3.0 * h[9]);
    h[13] = om[13] / 8.0 *
                (-e[MXYZ] + ux * e[MYZ] + uy * e[MXZ] + uz * e[MXY] - uy * uz * e[MX] -
                 ux * uz * e[MY] - ux * uy * e[MZ] + pr * ux * uy * uz) -
            1.25 * (uy * uz * h[1] + ux * uz * h[2] + ux * uy * h[3]) + uz * h[4] + uy * h[5] +
            ux * h[6];
    h[14] = om[14] / 16.0 *
                (-e[MXXYY] + 2.0 * uy * e[MXXY] + 2.0 * ux * e[MXYY] - uy * uy * e[MXX] -
                 ux * ux * e[MYY] - 4.0 * ux * uy * e[MXY] + 2.0 * ux * uy * uy * e[MX] +
                 2.0 * ux * ux * uy * e[MY] + cs4 * phi - pr * ux * ux * uy * uy) +
            1.25 * (ux * uy * uy * h[1] + ux * ux * uy * h[2]) - 2.0 * ux * uy * h[4] +
            0.125 * (ux * ux - uy * uy) * h[7] - 0.125 * (ux * ux + uy * uy) * h[8] -
            (0.375 * (ux * ux + uy * uy) + 0.5) * h[9] + 2.0 * (ux * h[10] + uy * h[11]) +
            uy * h[2] + ux * h[1];

    /* Eq. (13a): g~ = gbar + (K h^) + S^phi. */
    double S[15];
    orc_scalar_source(15, R, u, S);
    for (int a = 0; a < 15; ++a) {
        double kh = 0.0;
        for (int b = 0; b < 15; ++b) kh += K15[b * 15 + a] * h[b];
        out[a] = gbar[a] + kh + S[a];
    }
}

/* ------------------------------------------------------------------------------ */
/* Thermal collision, D3Q7: Appendix C (kernel h^_0..h^_6) with source R.           */
/* ------------------------------------------------------------------------------ */
void orc_collide_thermal7(const double gbar[7], const double u[3], const double om[7],
                          double cs2, double R, double out[7]) {
    double ux = u[0], uy = u[1], uz = u[2];
    double k[NMOM], sg[NMOM], e[NMOM];
    raw_moments(gbar, 7, k);
    scalar_source_raw(R, u, sg);
    for (int m = 0; m < NMOM; ++m) e[m] = k[m] + sg[m];
    double phi = k[M0] + 0.5 * R;
    double pr = phi + 0.5 * R;
    double h[7];
    h[0] = 0.0; /* the paper prints this line as "h_1 = 0"; h_0 is meant */
    h[1] = om[1] / 2.0 * (phi * ux - k[MX] - ux * 0.5 * R);
    h[2] = om[2] / 2.0 * (phi * uy - k[MY] - uy * 0.5 * R);
    h[3] = om[3] / 2.0 * (phi * uz - k[MZ] - uz * 0.5 * R);
    h[4] = om[4] / 4.0 *
               (-(e[MXX] - e[MYY]) + 2.0 * (ux * e[MX] - uy * e[MY]) - pr * (ux * ux - uy * uy)) +
           ux * h[1] - uy * h[2];
    h[5] = om[5] / 12.0 *
               (-(e[MXX] + e[MYY] - 2.0 * e[MZZ]) + 2.0 * (ux * e[MX] + uy * e[MY] - 2.0 * uz * e[MZ]) -
                pr * (ux * ux + uy * uy - 2.0 * uz * uz)) +
           (1.0 / 3.0) * (ux * h[1] + uy * h[2] - 2.0 * uz * h[3]);
    h[6] = om[6] / 6.0 *
               (3.0 * cs2 * phi - (e[MXX] + e[MYY] + e[MZZ]) +
                2.0 * (ux * e[MX] + uy * e[MY] + uz * e[MZ]) - pr * (ux * ux + uy * uy + uz * uz)) +
           (2.0 / 3.0) * (ux * h[1] + uy * h[2] + uz * h[3]);
    double S[7];
    orc_scalar_source(7, R, u, S);
    for (int a = 0; a < 7; ++a) {
        double kh = 0.0;
        for (int b = 0; b < 7; ++b) kh += K7[b * 7 + a] * h[b];
        out[a] = gbar[a] + kh + S[a];
    }
}

/* ------------------------------------------------------------------------------ */
/* Grid operations.                                                                */
/* ------------------------------------------------------------------------------ */

/* splitmix64 (Steele, Lea & Flood 2014; constants as published by S. Vigna): the
 * output for generator state x, i.e. the finaliser applied to x + golden gamma. */
uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline size_t cidx(const orc_problem* p, int i, int j, int k) {
    return ((size_t)k * p->ny + j) * p->nx + i;
}

/* Initial state (reading R9): fluid at rest, F = w_a; T = seeded uniform noise in
 * [-amp, amp] from splitmix64(seed ^ cell) (top 53 bits), G = w^phi_a T. */
void orc_init(const orc_problem* p, uint64_t seed, double amp, double* F, double* G) {
    size_t n = (size_t)p->nx * p->ny * p->nz;
    double wf[15], wg[15];
    orc_weights_flow(wf);
    orc_weights_thermal(p->q_g, p->cs2_phi, wg);
    for (size_t c = 0; c < n; ++c) {
        uint64_t r = orc_splitmix64(seed ^ (uint64_t)c);
        double u01 = (double)(r >> 11) * (1.0 / 9007199254740992.0);
        double T = amp * (2.0 * u01 - 1.0);
        for (int a = 0; a < 15; ++a) F[a * n + c] = wf[a];
        for (int a = 0; a < p->q_g; ++a) G[a * n + c] = wg[a] * T;
    }
}

/* Pull streaming (Eqs. 2b, 13b) with the wall rules R5-R7 for links whose source
 * node lies outside the cavity. */
static void pull_cell(const orc_problem* p, const double* Fin, const double* Gin, int i, int j,
                      int k, double fb[15], double* gb) {
    size_t n = (size_t)p->nx * p->ny * p->nz;
    size_t c = cidx(p, i, j, k);
    double wg[15];
    orc_weights_thermal(p->q_g, p->cs2_phi, wg);
    for (int a = 0; a < 15; ++a) {
        int si = i - EX[a], sj = j - EY[a], sk = k - EZ[a];
        if (p->boundary & 1) si = (si + p->nx) % p->nx;
        if (p->boundary & 2) sj = (sj + p->ny) % p->ny;
        if (p->boundary & 4) sk = (sk + p->nz) % p->nz;
        int inside = si >= 0 && si < p->nx && sj >= 0 && sj < p->ny && sk >= 0 && sk < p->nz;
        int o = OPP[a];
        if (inside) {
            fb[a] = Fin[(size_t)a * n + cidx(p, si, sj, sk)];
        } else {
            fb[a] = Fin[(size_t)o * n + c]; /* R5: half-way bounce-back */
        }
        if (a < p->q_g) {
            if (inside) {
                gb[a] = Gin[(size_t)a * n + cidx(p, si, sj, sk)];
            } else if (!(p->boundary & 8) && (si < 0 || si >= p->nx)) {
                double Tw = si < 0 ? p->T_cold : p->T_hot; /* R6: anti-bounce-back */
                gb[a] = -Gin[(size_t)o * n + c] + 2.0 * wg[a] * Tw;
            } else if (p->adiabatic_mode == 1) {
                /* R7, specular form: every velocity component whose wall the link
                 * crosses is mirrored, the others keep moving; the population is the
                 * one that left for the wall one step earlier. */
                int di = EX[a], dj = EY[a], dk = EZ[a], ri = si, rj = sj, rk = sk;
                if (si < 0 || si >= p->nx) { di = -di; ri = i; }
                if (sj < 0 || sj >= p->ny) { dj = -dj; rj = j; }
                if (sk < 0 || sk >= p->nz) { dk = -dk; rk = k; }
                int b = 0;
                while (EX[b] != di || EY[b] != dj || EZ[b] != dk) ++b;
                gb[a] = Gin[(size_t)b * n + cidx(p, ri, rj, rk)];
            } else {
                gb[a] = Gin[(size_t)o * n + c]; /* R7: adiabatic wall, bounce-back form */
            }
        }
    }
}

void orc_cell_update(const orc_problem* p, const double* Fin, const double* Gin, int i, int j,
                     int k, double fout[15], double* gout) {
    double fb[15], gb[15];
    pull_cell(p, Fin, Gin, i, j, k, fb, gb);
    /* Eq. (25): T = sum gbar + R/2. */
    double T = 0.0;
    for (int a = 0; a < p->q_g; ++a) T += gb[a];
    T += 0.5 * p->heat_source;
    /* Boussinesq force (Sec. 3), reading R8. */
    double T0 = 0.5 * (p->T_hot + p->T_cold);
    double F[3] = {p->ext_force[0], p->ext_force[1], p->ext_force[2] + p->gbeta * (T - T0)};
    double rho, u[3];
    orc_collide_flow(fb, F, p->omega_f, p->e4_mode, fout, &rho, u);
    if (p->q_g == 15)
        orc_collide_thermal15(gb, u, p->omega_g, p->cs2_phi, p->heat_source, gout);
    else
        orc_collide_thermal7(gb, u, p->omega_g, p->cs2_phi, p->heat_source, gout);
}

int orc_step(const orc_problem* p, const double* Fin, const double* Gin, double* Fout,
             double* Gout) {
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || (p->q_g != 15 && p->q_g != 7)) return -1;
    size_t n = (size_t)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < p->nz; ++k) {
        for (int j = 0; j < p->ny; ++j) {
            for (int i = 0; i < p->nx; ++i) {
                double fo[15], go[15];
                orc_cell_update(p, Fin, Gin, i, j, k, fo, go);
                size_t c = cidx(p, i, j, k);
                for (int a = 0; a < 15; ++a) Fout[(size_t)a * n + c] = fo[a];
                for (int a = 0; a < p->q_g; ++a) Gout[(size_t)a * n + c] = go[a];
            }
        }
    }
    return 0;
}

int orc_run(const orc_problem* p, double* F, double* G, double* Fs, double* Gs, int64_t nsteps) {
    size_t n = (size_t)p->nx * p->ny * p->nz;
    double *fa = F, *ga = G, *fb = Fs, *gb = Gs;
    for (int64_t s = 0; s < nsteps; ++s) {
        int rc = orc_step(p, fa, ga, fb, gb);
        if (rc) return rc;
        double* t = fa; fa = fb; fb = t;
        t = ga; ga = gb; gb = t;
    }
    if (fa != F) {
        memcpy(F, fa, sizeof(double) * 15 * n);
        memcpy(G, ga, sizeof(double) * (size_t)p->q_g * n);
    }
    return 0;
}

/* Macroscopic fields of a stored (post-collision) state: rho = sum F, T = sum G - R/2 and,
 * because collision adds F to the momentum (Eq. 2a, sum S e = F), rho u = sum F e - F/2
 * reproduces Eq. (3) of the same time level. */
void orc_fields(const orc_problem* p, const double* F, const double* G, double* rho, double* ux,
                double* uy, double* uz, double* T) {
    size_t n = (size_t)p->nx * p->ny * p->nz;
    double T0 = 0.5 * (p->T_hot + p->T_cold);
    for (size_t c = 0; c < n; ++c) {
        double r = 0, jx = 0, jy = 0, jz = 0, t = 0;
        for (int a = 0; a < 15; ++a) {
            double f = F[(size_t)a * n + c];
            r += f;
            jx += f * EX[a];
            jy += f * EY[a];
            jz += f * EZ[a];
        }
        for (int a = 0; a < p->q_g; ++a) t += G[(size_t)a * n + c];
        t -= 0.5 * p->heat_source; /* collision added R: phi = sum g~ - R/2 (Eq. 25) */
        double Fx = p->ext_force[0], Fy = p->ext_force[1];
        double Fz = p->ext_force[2] + p->gbeta * (t - T0);
        if (rho) rho[c] = r;
        if (ux) ux[c] = (jx - 0.5 * Fx) / r;
        if (uy) uy[c] = (jy - 0.5 * Fy) / r;
        if (uz) uz[c] = (jz - 0.5 * Fz) / r;
        if (T) T[c] = t;
    }
}

/* Nusselt numbers and peak velocities (Sec. 3, Table 1), readings R11 and R12. */
int orc_nusselt(const orc_problem* p, const double* F, const double* G, orc_nu* out) {
    int nx = p->nx, ny = p->ny, nz = p->nz;
    if (nx < 2) return -1;
    size_t n = (size_t)nx * ny * nz;
    double* fld = (double*)malloc(sizeof(double) * 5 * n);
    if (!fld) return -2;
    double *rho = fld, *ux = fld + n, *uy = fld + 2 * n, *uz = fld + 3 * n, *T = fld + 4 * n;
    orc_fields(p, F, G, rho, ux, uy, uz, T);
    (void)uy;
    double L = (double)nx, dT = p->T_hot - p->T_cold;
    double U0 = p->U0 > 0 ? p->U0 : 1.0;

    /* local Nu on each face cell; the one-sided stencil (9 T1 - T2 - 8 Tw)/3 gives
     * dT/dn at a half-way wall exactly for quadratic profiles */
    double hot_sum = 0.0, cold_sum = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) {
            double Th1 = T[cidx(p, nx - 1, j, k)], Th2 = T[cidx(p, nx - 2, j, k)];
            double Tc1 = T[cidx(p, 0, j, k)], Tc2 = T[cidx(p, 1, j, k)];
            hot_sum += -L * (9.0 * Th1 - Th2 - 8.0 * p->T_hot) / (3.0 * dT);
            cold_sum += L * (9.0 * Tc1 - Tc2 - 8.0 * p->T_cold) / (3.0 * dT);
        }
    out->hot_wall_mean = hot_sum / ((double)ny * nz);
    out->cold_wall_mean = cold_sum / ((double)ny * nz);

    /* symmetry plane y = L/2: node (ny-1)/2, or the mean of the two straddling nodes */
    int j0 = (ny - 1) / 2, j1 = ny / 2;
    double msum = 0.0, mmax = -1e300, mmin = 1e300, zmax = 0.0, zmin = 0.0;
    for (int k = 0; k < nz; ++k) {
        double Th1 = 0.5 * (T[cidx(p, nx - 1, j0, k)] + T[cidx(p, nx - 1, j1, k)]);
        double Th2 = 0.5 * (T[cidx(p, nx - 2, j0, k)] + T[cidx(p, nx - 2, j1, k)]);
        double nu = -L * (9.0 * Th1 - Th2 - 8.0 * p->T_hot) / (3.0 * dT);
        double z = (k + 0.5) / nz;
        msum += nu;
        if (nu > mmax) { mmax = nu; zmax = z; }
        if (nu < mmin) { mmin = nu; zmin = z; }
    }
    out->mid_mean = msum / nz;
    out->mid_max = mmax;
    out->mid_max_z = zmax;
    out->mid_min = mmin;
    out->mid_min_z = zmin;

    /* u_max: |u_x| on the vertical centreline x = y = L/2; w_max: |u_z| on the
     * horizontal centreline y = z = L/2 (straddling nodes averaged for even sizes) */
    int i0 = (nx - 1) / 2, i1 = nx / 2, k0 = (nz - 1) / 2, k1 = nz / 2;
    double umax = -1.0, uz_at = 0.0;
    for (int k = 0; k < nz; ++k) {
        double v = 0.25 * (ux[cidx(p, i0, j0, k)] + ux[cidx(p, i1, j0, k)] +
                           ux[cidx(p, i0, j1, k)] + ux[cidx(p, i1, j1, k)]);
        if (fabs(v) > umax) { umax = fabs(v); uz_at = (k + 0.5) / nz; }
    }
    double wmax = -1.0, wx_at = 0.0;
    for (int i = 0; i < nx; ++i) {
        double v = 0.25 * (uz[cidx(p, i, j0, k0)] + uz[cidx(p, i, j1, k0)] +
                           uz[cidx(p, i, j0, k1)] + uz[cidx(p, i, j1, k1)]);
        if (fabs(v) > wmax) { wmax = fabs(v); wx_at = (i + 0.5) / nx; }
    }
    out->umax = umax / U0;
    out->umax_z = uz_at;
    out->wmax = wmax / U0;
    out->wmax_x = wx_at;
    free(fld);
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loop over z-planes in orc_step (1 = serial).  The result does not
 * depend on the count: every node is computed independently. */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
