/*
 * lbm_slabs.h -- one cavity decomposed into z-slabs with a halo exchange (C ABI).
 *
 * The grid's nz planes are split into `nslabs` slabs of whole z-planes (planes are
 * contiguous in the structure-of-arrays layout of include/lbm.h, so every population of a
 * slab is one contiguous range).  Each slab is a context of include/lbm.h on the grid
 * (nx, ny, halo_lo + nz_owned + halo_hi): its owned planes plus one halo plane for every
 * cut it touches, holding a copy of the neighbouring slab's plane.  A time step of the
 * decomposition is one step of the method (Eqs. 2b, 13b pull streaming, Appendix A and
 * Sec. 2.2 / Appendix C collisions, the Sec. 3 wall rules) on every slab, followed by the
 * exchange: each slab's first and last owned planes of the new state are copied into the
 * halo planes of its neighbours.
 *
 * Pull streaming reads only the planes z - 1, z, z + 1, so every owned node of a slab
 * reads exactly what it would read in the undivided grid: owned planes next to a cut
 * pull from the halo copy, owned planes at the grid's z faces take the wall rules there.
 * Halo planes are updated by the slab's step as well (as if a wall lay beyond them) and
 * overwritten by the exchange, so the owned nodes follow the trajectory of one context
 * on the whole grid bit for bit, in every storage precision.  With z periodic
 * (boundary bit 2) the cuts wrap around: the first and last slab exchange too.
 *
 * The exchange copies every population of the cut plane (and, in the 16-bit forms, its
 * FP32 node temperatures), so halo nodes equal their owners exactly and the residual and
 * the NaN check, taken over whole slab buffers, stay exact; the streaming itself needs
 * only the populations with e_z across the cut (5 + 5 of 30 in D3Q15 + D3Q15, 5 + 1 of 22
 * with D3Q7).  All slabs live on one GPU and one stream; on several GPUs the same plan
 * would put one slab on each device with peer copies of the halo planes.
 *
 * The paper runs one undivided grid; this is a decomposition of the same computation.
 * Errors and threading follow include/lbm.h: LBM_OK or a negative LBM_E* code with the
 * message in lbm_slabs_last_error; a decomposition is not thread-safe.
 */
#ifndef LBM_SLABS_H
#define LBM_SLABS_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_slabs lbm_slabs; /* opaque, library-owned */

/* Host only, no GPU.  The split of nz planes into nslabs slabs under boundary mode
 * `boundary` (LBM_BC_*; bit 2 = z periodic).  owned: NULL = an even split (the first
 * nz % nslabs slabs one plane more), else nslabs caller-given plane counts, each >= 1,
 * summing to nz.  Outputs (arrays of nslabs ints, each may be NULL): z0[s] the global
 * index of slab s's first owned plane, nz_owned[s], halo_lo[s] and halo_hi[s] (0 or 1:
 * a halo plane below / above the owned planes).  A single slab has no halos.  LBM_EINVAL
 * if nz < 1, nslabs < 1, nslabs > nz or the counts are invalid. */
int lbm_slabs_plan(int nz, int nslabs, int boundary, const int* owned, int* z0, int* nz_owned,
                   int* halo_lo, int* halo_hi);

/* A decomposition of the grid `grid` into slabs as lbm_slabs_plan gives them, with the
 * parameters `params` of the whole grid (lbm_derive_params with that grid: L = nx) and
 * the options of lbm_create_params (NULL = defaults; device_arena must be NULL: each
 * slab allocates its own device memory).  The initial state is the one lbm_create_params
 * gives the whole grid (fluid at rest, the seeded noise of every node drawn for its
 * global index).  LBM_EINVAL for an invalid grid, lattice, parameters, options or split;
 * LBM_ENOMEM if an allocation fails. */
int lbm_slabs_create(const lbm_grid* grid, int lattice, const lbm_params* params,
                     const lbm_options* opt, int nslabs, const int* owned, lbm_slabs** out);

/* Advance every slab n >= 0 time steps, exchanging the halo planes after each.  Whole
 * residual intervals (lbm_options.residual_interval, aligned with the step count) run as
 * one CUDA graph launch each.  Returns on enqueue, except that when a residual check fell
 * in the call it waits for the GPU (bounded) and records the residual: LBM_EDIVERGED if
 * any slab's temperature is no longer finite. */
int lbm_slabs_step(lbm_slabs* s, int64_t n);

/* max |T(t) - T(t - residual_interval)| over the grid at the last check, or -1 if none. */
int lbm_slabs_residual(lbm_slabs* s, double* max_dT);

/* Populations of the whole grid as FP64 host arrays in the layout of include/lbm.h
 * (f: 15 * nx*ny*nz, g: lattice * nx*ny*nz), gathered from the slabs' owned planes;
 * set scatters them, halo planes included.  Caller-owned; both required. */
int lbm_slabs_get_populations(lbm_slabs* s, double* f, double* g);
int lbm_slabs_set_populations(lbm_slabs* s, const double* f, const double* g);

/* Macroscopic fields of the whole grid as lbm_fields gives them (host arrays of
 * nx*ny*nz doubles, x fastest; any may be NULL). */
int lbm_slabs_fields(lbm_slabs* s, double* rho, double* ux, double* uy, double* uz, double* T);

/* Slab count, steps taken, and the bytes the exchange copies per time step. */
int lbm_slabs_count(const lbm_slabs* s);
int64_t lbm_slabs_steps_done(const lbm_slabs* s);
int64_t lbm_slabs_halo_bytes(const lbm_slabs* s);

/* ---- the message of one cut, for slabs held by different processes -------------------
 *
 * Pull streaming carries across a cut only the populations whose e_z points across it:
 * upwards (dir = +1) the D3Q15 directions 5, 7, 8, 9, 10 of the flow and of a D3Q15 scalar
 * (direction 5 alone for D3Q7), downwards (dir = -1) 6, 11, 12, 13, 14 (D3Q7: 6).  Every
 * wall rule a node next to a cut applies reads, from the plane across the cut, only
 * populations of that set (a specular reflection keeps e_z), so a slab held by another
 * process needs, each step, only these: (5 + 5) or (5 + 1) values per node of one plane,
 * a third or a quarter of the planes lbm_slabs_step copies.  Per step and cut, the slab
 * below packs the upward set of its last owned plane and the slab above unpacks it into
 * its halo plane below; the slab above packs the downward set of its first owned plane
 * and the slab below unpacks it into its halo plane above (planes as lbm_slabs_plan
 * gives them).  The other populations of a halo plane are then not those of the
 * neighbour's plane: only the owned planes follow the undivided grid.
 *
 * These calls are host only (no GPU): they move values between FP64 host arrays of a
 * slab's state, in the layout of include/lbm.h for the slab grid (nx, ny, planes of the
 * slab), and a message of lbm_slabs_cut_values doubles (the flow set, then the scalar
 * set, each population one nx * ny plane, x fastest).  The transport between processes
 * (MPI, torch.distributed, NCCL) is the caller's.  LBM_EINVAL for an invalid grid,
 * lattice, plane, direction or NULL array. */
int lbm_slabs_cut_populations(int lattice, int dir, int* flow_ids, int* n_flow,
                              int* scalar_ids, int* n_scalar);
int64_t lbm_slabs_cut_values(int nx, int ny, int lattice);
int lbm_slabs_pack_cut(const lbm_grid* slab_grid, int lattice, int plane, int dir,
                       const double* f, const double* g, double* msg);
int lbm_slabs_unpack_cut(const lbm_grid* slab_grid, int lattice, int plane, int dir,
                         const double* msg, double* f, double* g);

/* Wait (bounded) for the work queued on the decomposition's stream. */
int lbm_slabs_synchronize(lbm_slabs* s);
const char* lbm_slabs_last_error(const lbm_slabs* s);
void lbm_slabs_destroy(lbm_slabs* s);

#ifdef __cplusplus
}
#endif

#endif
