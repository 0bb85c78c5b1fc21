/*
 * lbm.h -- C ABI of the GB300 (sm_103a) library for the cascaded central-moment thermal
 * lattice Boltzmann method of Hajabdollahi & Premnath, "Central Moments-based Cascaded
 * Lattice Boltzmann Method for Thermal Convective Flows in Three-Dimensions"
 * (arXiv:1710.04751).
 *
 * One time step (lbm_step) is one fused CUDA kernel over the grid: pull streaming
 * (Eqs. 2b, 13b), macroscopic variables (Eqs. 3, 25), the Boussinesq force (Sec. 3),
 * the D3Q15 flow cascade with forcing (Appendix A, Eq. 2a), the D3Q15 (Sec. 2.2,
 * Eq. 13a) or D3Q7 (Appendix C) thermal cascade, and the cavity wall rules (Sec. 3).
 *
 * Conventions shared by every entry point
 *  - Coordinates: x (index i) is the heated direction, cold face at i = -1/2 (T_cold),
 *    hot face at i = nx - 1/2 (T_hot); z (index k) is vertical, buoyancy along +z; y is
 *    spanwise.  Walls lie half-way between the last node and its missing neighbour, so
 *    the cavity length is L = nx.  (The paper's y is this x; its x is this y.)
 *  - Host population arrays are FP64, structure-of-arrays, p[a * ncell + cell] with
 *    cell = (k * ny + j) * nx + i (x fastest) and a the paper's direction order: D3Q15
 *    rest, +-x, +-y, +-z, then (+,+,+) (-,+,+) (+,-,+) (-,-,+) (+,+,-) (-,+,-) (+,-,-)
 *    (-,-,-); D3Q7 the first seven.  Stored populations are post-collision: a step is
 *    pull, then collide.
 *  - Every host pointer is caller-owned and only read/written during the call.  Device
 *    memory is library-owned unless the caller passes an arena in lbm_options.
 *  - Return codes: LBM_OK (0) or a negative LBM_E* code; lbm_last_error(ctx) then holds a
 *    message (lbm_last_error(NULL) for failures without a context).
 *  - A context is not thread-safe.  All work runs on the context's CUDA stream; calls
 *    that return host data synchronise that stream with a bounded wait.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_EINVAL (-1)    /* invalid argument: sizes, lattice, precision, rates out of (0,2) */
#define LBM_ENOMEM (-2)    /* device or host allocation failed, or arena too small */
#define LBM_ECUDA (-3)     /* a CUDA runtime call failed (message in lbm_last_error) */
#define LBM_EDIVERGED (-4) /* a NaN or Inf temperature was detected */
#define LBM_ETIMEOUT (-5)  /* a bounded wait for the GPU ran out */

enum { LBM_THERMAL_D3Q15 = 15, LBM_THERMAL_D3Q7 = 7 };
/* Storage and arithmetic: FP64; FP32; or 16-bit storage of each population minus its
 * rest-state value (w_a for the flow; w^phi_a T_node for the scalar, T_node the temperature
 * of the node holding it, kept in an FP32 plane) with FP32 arithmetic: FP16 (11 significant
 * bits; the flow deviations stored times 2^12, rounded stochastically, so that deviations
 * down to 1.5e-8 stay normal FP16 numbers) or BF16 (8 significant bits, FP32 range,
 * rounded to nearest); the scalar deviations are rounded to nearest.  The rounding of the stored deviations
 * puts a floor under the residual of lbm_residual (max |dT| per 100 steps about 2e-5 in
 * FP16 and 2e-4 in BF16 on 64^3-256^3 cavities), so a convergence test below that floor is
 * never met in those forms. */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16_DEV = 2, LBM_BF16_DEV = 3 };

/* Boundary modes (bit mask).  Bits 0..2: x, y, z periodic.  Bit 3: the x walls are
 * adiabatic instead of Dirichlet.  LBM_BC_CAVITY is the paper's cubic cavity (Sec. 3):
 * no-slip walls everywhere, T_cold / T_hot on the x faces, adiabatic y and z faces. */
enum {
    LBM_BC_CAVITY = 0,
    LBM_BC_XWALLS = 6,       /* Dirichlet x walls, periodic y and z */
    LBM_BC_PERIODIC = 7,     /* fully periodic box */
    LBM_BC_ADIABATIC_BOX = 8 /* closed box, every face adiabatic */
};

/* Adiabatic-wall rule for the thermal populations (Sec. 3 cites a Neumann scheme
 * without giving it).  Specular reflection (default) mirrors the wall-normal velocity
 * component of every link that crosses the wall; bounce-back reverses the whole link. */
enum { LBM_ADIABATIC_BOUNCE_BACK = 0, LBM_ADIABATIC_SPECULAR = 1 };

typedef struct {
    int nx, ny, nz; /* lattice nodes per direction, each >= 1 */
} lbm_grid;

/* Physical parameters in lattice units.  lbm_derive_params fills them from (Ra, Pr, Ma)
 * as Sec. 3 defines: U0 = Ma c_s = sqrt(g beta dT L), g beta = U0^2/(dT L),
 * nu = sqrt(Pr/Ra) U0 L, alpha = nu/Pr, nu = (1/3)(1/omega - 1/2) (Appendix A) and
 * alpha = cs2_phi (1/omega - 1/2) (Eq. 23). */
typedef struct {
    double omega_f[15];   /* flow rates omega_0..omega_14 (0..3 unused); paper: 4..8 = omega_nu (shear), rest 1 */
    double omega_g[15];   /* thermal rates omega_0..omega_{Q-1} (0 unused); paper: 1..3 = omega_phi, rest 1 */
    double gbeta;         /* g beta of the Boussinesq force F_z = g beta (T - T0) */
    double T_hot, T_cold; /* Dirichlet face temperatures; T0 = (T_hot + T_cold)/2 */
    double cs2_phi;       /* c_sphi^2 of the thermal equilibrium (Sec. 2.2), in (0, 1/2] (D3Q7: (0, 1/3]) */
    double ext_force[3];  /* extra uniform body force added to F (0 for the cavity) */
    double U0;            /* velocity scale used to report u/U0 in lbm_nusselt */
    double heat_source;   /* uniform scalar source R of the CDE (Eq. 4, App. B/C); 0 in the cavity.
                             T = sum g + R/2 (Eq. 25) */
    int e4_mode;          /* App. A g^_14 equilibrium: 0 E = kxx~ kyy~ / rho, 1 E = rho c_s^4 */
    int adiabatic_mode;   /* LBM_ADIABATIC_* */
    int boundary;         /* LBM_BC_* */
} lbm_params;

typedef struct {
    int precision;            /* LBM_FP32 (default), LBM_FP64, LBM_FP16_DEV or LBM_BF16_DEV */
    uint64_t seed;            /* noise seed of the initial temperature (default 1) */
    double noise_amp;         /* initial T = uniform noise in [-amp, amp] (default 1e-6) */
    double cs2_phi;           /* c_sphi^2; 0 (default) = 1/3 for D3Q15, 1/4 for D3Q7 (at 1/3 the
                                 D3Q7 rest equilibrium phi (1 - 3 c_sphi^2 - u^2) is negative) */
    int e4_mode;              /* default 0 */
    int adiabatic_mode;       /* default LBM_ADIABATIC_SPECULAR */
    int residual_interval;    /* steps between residual / NaN checks in lbm_step (default 100, 0 = off) */
    void* cuda_stream;        /* cudaStream_t to run on; NULL = the legacy default stream */
    void* device_arena;       /* caller-owned device memory of >= lbm_arena_bytes(), or NULL */
    size_t device_arena_bytes;
    double timeout_s;         /* bound on every host wait for the GPU (default 600 s) */
} lbm_options;

typedef struct {
    double hot_wall_mean, cold_wall_mean; /* face-averaged Nu on the hot and cold walls */
    double mid_mean;                      /* mean of the local hot-wall Nu on the symmetry plane y = L/2 */
    double mid_max, mid_max_z;            /* its maximum and the height z/L where it occurs */
    double mid_min, mid_min_z;            /* its minimum and where */
    double umax, umax_z;                  /* max |u_x|/U0 on the vertical centreline x = y = L/2, at z/L */
    double wmax, wmax_x;                  /* max |u_z|/U0 on the horizontal centreline y = z = L/2, at x/L */
} lbm_nu;

typedef struct lbm_ctx lbm_ctx; /* opaque, library-owned */

/* Fill *opt with the defaults listed above. */
void lbm_default_options(lbm_options* opt);

/* Host only, no GPU.  Parameters of the differentially heated cavity (Sec. 3) for
 * L = grid->nx, dT = 1 (T_hot = 0.5, T_cold = -0.5), from Ra, Pr and Ma = U0 / c_s.
 * LBM_EINVAL if Ra, Pr or Ma <= 0, if U0 >= 0.3, or if omega_nu or omega_phi falls
 * outside (0, 2) (the bounds stated for every rate in Sec. 2.2 and Appendix A). */
int lbm_derive_params(const lbm_grid* grid, int lattice, double Ra, double Pr, double Ma,
                      const lbm_options* opt, lbm_params* out);

/* Host only.  Device bytes a context of this size needs (for lbm_options.device_arena). */
size_t lbm_arena_bytes(const lbm_grid* grid, int lattice, int precision);

/* Create a cavity: lbm_derive_params, then lbm_create_params.  The fluid starts at rest
 * (f = rest weights) with T = seeded noise (g = w^phi T), as a post-collision state. */
int lbm_create(const lbm_grid* grid, int lattice, double Ra, double Pr, double Ma,
               const lbm_options* opt /* NULL = defaults */, lbm_ctx** out);

/* Create a context with explicit parameters (every rate must lie in (0, 2)). */
int lbm_create_params(const lbm_grid* grid, int lattice, const lbm_params* params,
                      const lbm_options* opt /* NULL = defaults */, lbm_ctx** out);

/* Advance n >= 0 time steps (one fused kernel each), asynchronously on the context's
 * stream.  Every residual_interval steps a reduction records max |T - T_previous_check|
 * and flags non-finite temperatures; if any check ran, the call waits (bounded) at its
 * end and returns LBM_EDIVERGED when the flag is set. */
int lbm_step(lbm_ctx* ctx, int64_t n);

/* Macroscopic fields of the stored state into caller-owned host arrays of ncell FP64
 * each (x fastest); any pointer may be NULL.  rho = sum f, T = sum g,
 * u = (sum f e - F/2)/rho with F from T (Eq. 3 at the same time level). */
int lbm_fields(lbm_ctx* ctx, double* rho, double* ux, double* uy, double* uz, double* T);

/* Nusselt numbers and peak velocities of Table 1 (Sec. 3).  Local Nu = L |dT/dn| / dT
 * with dT/dn = (9 T_1 - T_2 - 8 T_w)/3 at a half-way wall; lines on the symmetry plane
 * average the two straddling nodes when a size is even.  Needs nx >= 2. */
int lbm_nusselt(lbm_ctx* ctx, lbm_nu* out);

/* The last residual recorded by lbm_step: max over the grid of |T - T at the previous
 * check| (a negative value if no check has run since creation or set_populations). */
int lbm_residual(lbm_ctx* ctx, double* max_dT);

/* Copy the stored populations to / from caller-owned host arrays (FP64, layout above;
 * f has 15 ncell values, g has Q ncell values).  set_populations converts to the
 * context's precision and restarts the residual snapshot. */
int lbm_get_populations(lbm_ctx* ctx, double* f, double* g);
int lbm_set_populations(lbm_ctx* ctx, const double* f, const double* g);

/* The same in the context's own storage precision, for LBM_FP32 (float arrays) and
 * LBM_FP64 (double arrays) contexts: each population plane goes straight between the
 * caller's host array and the device state, with no conversion pass (half the bytes of the
 * FP64 calls for an FP32 context).  Same layout, ownership and residual-snapshot restart as
 * above; page-locked host arrays make the copies fastest.  LBM_EINVAL for the 16-bit forms,
 * whose stored values are deviations that need their node temperatures. */
int lbm_get_populations_native(lbm_ctx* ctx, void* f, void* g);
int lbm_set_populations_native(lbm_ctx* ctx, const void* f, const void* g);

/* Set the stored populations to the equilibria of given fields: f to the populations
 * whose central moments are the flow collision's equilibria at (rho, u) (App. A:
 * Maxwellian, c_s^2 = 1/3), g to those whose central moments are the equilibria of
 * Eq. (15) at (T, u).  rho, ux, uy, uz, T: caller-owned DEVICE arrays of ncell FP64
 * values (layout above; rho NULL means rho = 1), read on the context's stream before the
 * call returns.  Restarts the residual snapshot.  Starting the solver from a predicted
 * steady state (the learned warm start, include/lbm_net.h) uses this. */
int lbm_set_fields(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy,
                   const double* uz, const double* T);

/* lbm_set_fields followed by `iterations` rounds of one time step and a re-imposition
 * of the given u and T that keeps each node's departure from equilibrium (its stresses
 * and heat fluxes) and its rho: p <- p - p_eq(current u, T) + p_eq(given u, T).  The
 * non-equilibrium parts thereby adapt to the given fields -- the iterative consistent
 * initialisation of Mei, Luo, Lallemand & d'Humieres (Computers & Fluids 35, 2006),
 * applied to u and T.  An odd count is rounded up to the next even one (the state then
 * stays in its buffer, which batch members need).  The rounds are not counted by
 * lbm_steps_done.  iterations = 0 is lbm_set_fields. */
int lbm_init_fields(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy,
                    const double* uz, const double* T, int iterations);

/* Checkpoints (the paper has none; a restartable run needs one).  lbm_save writes to the
 * file at `path`: a header (magic "LBMCKPT1", version 1, the grid, the scalar lattice, the
 * storage precision, the model parameters as lbm_params, the step count), then the 15
 * flow and the Q scalar populations as FP64 in the layout of lbm_get_populations
 * (little-endian; the host's byte order, as both build hosts are).  The file is written
 * completely or the call fails (LBM_EINVAL: cannot open or write; the partial file is
 * removed).  lbm_checkpoint_info reads a file's header, so that a caller can create the
 * matching context (lbm_create_params with the returned grid, lattice, parameters and
 * precision); lbm_restore then loads the populations and the step count into such a
 * context (LBM_EINVAL if its grid, lattice or precision differ, or the file is short or
 * not a checkpoint).  Restoring into the same precision is exact for FP64 and FP32; the
 * 16-bit forms re-encode each deviation once (within one 16-bit rounding).  Any pointer
 * of lbm_checkpoint_info may be NULL. */
int lbm_save(lbm_ctx* ctx, const char* path);
int lbm_checkpoint_info(const char* path, lbm_grid* grid, int* lattice, int* precision,
                        lbm_params* params, int64_t* steps);
int lbm_restore(lbm_ctx* ctx, const char* path);

/* Bound, in seconds (> 0), of every later host wait of this context for the GPU (the
 * lbm_options.timeout_s given at creation until changed).  A wait that runs out returns
 * LBM_ETIMEOUT and leaves the queued work running: the context stays usable, and a later
 * call (lbm_synchronize, or any call that reads results) waits again.  Every call that
 * returns data in caller memory first waits for the stream's earlier work under this
 * bound, then copies.  LBM_EINVAL for a NULL context or timeout_s <= 0. */
int lbm_set_timeout(lbm_ctx* ctx, double timeout_s);

/* Parameters in use, step counter, last error message, stream wait, destruction. */
int lbm_get_params(const lbm_ctx* ctx, lbm_params* out);
int64_t lbm_steps_done(const lbm_ctx* ctx);
const char* lbm_last_error(const lbm_ctx* ctx);
int lbm_synchronize(lbm_ctx* ctx);
void lbm_destroy(lbm_ctx* ctx);

/* Allocation-free Nusselt reduction.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- code whose device memory is owned
 * and pre-reserved by an enclosing application or framework, real-time loops that must
 * not allocate (or risk an allocation failure) once running, plug-ins forbidden to
 * allocate after start-up.  It computes exactly what lbm_nusselt computes, for
 * populations the caller holds in its own device buffers, and allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.
 *   f_dev, g_dev  device pointers to the 15 flow and `lattice` thermal population planes,
 *                 layout of the host arrays above but with `plane` elements between
 *                 consecutive planes (plane >= nx*ny*nz); FP32 or FP64 per `precision`.
 *   params        as for lbm_create_params (T_hot, T_cold, gbeta, ext_force, U0 are used).
 *   cuda_stream   cudaStream_t to run on (NULL = legacy default stream); the call waits
 *                 for that stream (bounded, 600 s) before writing *out.
 * Its scratch is a static device array of 2*1024 + 16 doubles (16.5 KB) that every GPU
 * loading the library holds until the process exits; it bounds the face count:
 * ny*nz <= 262144 (1024 blocks of 256 face cells), larger grids give LBM_EINVAL.  The
 * first call on each device, with that device current, looks up the array's device
 * address (a one-time set-up); make that first call before any stream capture.  That
 * address is cached for the life of the process: do not call this entry point after a
 * cudaDeviceReset of the device in the same process.  Every
 * call overwrites the array's partial sums before reading them, so nothing carries over
 * from the previous call; calls that overlap on the GPU (other streams, other threads)
 * share the array and race.  Errors: LBM_EINVAL (NULL pointer, sizes, lattice,
 * precision, plane), LBM_ECUDA, LBM_ETIMEOUT; message in lbm_last_error(NULL). */
int lbm_nusselt_noalloc(const void* f_dev, const void* g_dev, int64_t plane, int precision,
                        const lbm_grid* grid, int lattice, const lbm_params* params,
                        void* cuda_stream, lbm_nu* out);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
