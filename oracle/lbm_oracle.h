/*
 * lbm_oracle.h -- FP64 CPU oracle of the cascaded central-moment thermal lattice
 * Boltzmann method (Hajabdollahi & Premnath, arXiv:1710.04751).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct restatement of
 * the paper's equations, used to check the CUDA library.  It shares no code, header,
 * table or constant with the CUDA path.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load it.
 *
 * Layout of every population array: p[a * ncell + cell], cell = (k*ny + j)*nx + i,
 * x (index i) fastest.  x is the heated direction (cold face at i = -1/2, hot face at
 * i = nx - 1/2), z (index k) is vertical, buoyancy acts along +z.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Boundary modes.  Bits 0..2: the x, y, z directions are periodic.  Bit 3: the walls
 * that close the x direction are adiabatic instead of Dirichlet (hot/cold).  The
 * paper's cavity (Sec. 3) is 0; the others exist for the oracle's test problems. */
enum {
    ORC_BC_CAVITY = 0,          /* no-slip walls; Dirichlet x faces; adiabatic y, z faces */
    ORC_BC_PERIODIC = 7,        /* fully periodic box */
    ORC_BC_XWALLS = 6,          /* Dirichlet x walls, y and z periodic (1D conduction) */
    ORC_BC_ADIABATIC_BOX = 8    /* closed box, every face adiabatic */
};

typedef struct {
    int nx, ny, nz;
    int q_g;              /* 15 (D3Q15 thermal, Sec. 2.2) or 7 (D3Q7 thermal, App. C) */
    int boundary;         /* ORC_BC_* (bit mask, see above) */
    int e4_mode;          /* 0: E = kxx~ kyy~ / rho ; 1: E = rho cs^4 (App. A, g14) */
    int adiabatic_mode;   /* adiabatic walls for g: 0 bounce-back, 1 specular reflection */
    double omega_f[15];   /* flow relaxation rates omega_0..omega_14 (0..3 unused) */
    double omega_g[15];   /* thermal relaxation rates omega_0..omega_{q_g-1} (0 unused) */
    double gbeta;         /* g*beta in F = g beta (T - T0) k (Eq. for the Boussinesq force) */
    double T_hot, T_cold; /* Dirichlet temperatures of the x = L and x = 0 faces */
    double cs2_phi;       /* c_{s phi}^2 of the thermal equilibrium (Sec. 2.2) */
    double ext_force[3];  /* extra uniform body force (test problems only; 0 in the cavity) */
    double U0;            /* velocity scale sqrt(g beta dT L) used to report u/U0 */
    double heat_source;   /* uniform scalar source R of the CDE (Eq. 4); 0 in the cavity */
} orc_problem;

typedef struct {
    double hot_wall_mean, cold_wall_mean;
    double mid_mean, mid_max, mid_max_z, mid_min, mid_min_z;
    double umax, umax_z, wmax, wmax_x;
} orc_nu;

/* Tables written out from the paper's definitions. */
void orc_velocities(int q, int* ex, int* ey, int* ez);
void orc_kmatrix15(int* K /* [15][15], K[b*15 + a] = K_b(alpha=a) */);
void orc_kmatrix7(int* K /* [7][7] */);
void orc_weights_flow(double w[15]);
void orc_weights_thermal(int q, double cs2_phi, double* w);
int  orc_opposite(int q, int a);

/* One-cell collisions (Form A: the paper's closed-form cascades). */
void orc_flow_source(const double F[3], const double u[3], double S[15]);
void orc_collide_flow(const double fbar[15], const double F[3], const double omega[15],
                      int e4_mode, double out[15], double* rho_out, double u_out[3]);
void orc_collide_thermal15(const double gbar[15], const double u[3], const double omega[15],
                           double cs2_phi, double R, double out[15]);
void orc_collide_thermal7(const double gbar[7], const double u[3], const double omega[7],
                          double cs2_phi, double R, double out[7]);
void orc_scalar_source(int q, double R, const double u[3], double* S);

/* Whole-grid operations. */
void orc_init(const orc_problem* p, uint64_t seed, double noise_amp, double* F, double* G);
int  orc_step(const orc_problem* p, const double* Fin, const double* Gin,
              double* Fout, double* Gout);
int  orc_run(const orc_problem* p, double* F, double* G, double* Fscratch, double* Gscratch,
             int64_t nsteps);
void orc_cell_update(const orc_problem* p, const double* Fin, const double* Gin,
                     int i, int j, int k, double fout[15], double* gout);
void orc_fields(const orc_problem* p, const double* F, const double* G,
                double* rho, double* ux, double* uy, double* uz, double* T);
int  orc_nusselt(const orc_problem* p, const double* F, const double* G, orc_nu* out);
uint64_t orc_splitmix64(uint64_t x);
int  orc_num_threads(void);
void orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
