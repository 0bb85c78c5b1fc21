/*
 * lbm_batch.h -- many independent cavities advanced together (C ABI).
 *
 * A batch holds `count` cavities of the method of arXiv:1710.04751 (each a full lbm_ctx
 * of include/lbm.h with its own grid and parameters: Ra, Pr, walls, rates) that share
 * one lattice, one storage precision and one CUDA stream.  Every time step of the whole
 * batch is ONE launch of a persistent kernel: a fixed grid of blocks walks a list of
 * tiles (runs of nodes of one cavity) covering every active cavity, and updates each
 * node exactly as lbm_step does (the same per-node code, so a member's trajectory is
 * the one lbm_step would produce).  Steps are captured in a CUDA graph, one graph per
 * `residual_interval` steps, ending with a batched convergence check.  A member whose
 * residual max|dT| over one interval falls below `steady_tol` (converged), or whose
 * temperature is no longer finite (diverged), leaves the tile list and keeps its state.
 *
 * The paper has no batched form; it runs one cavity at a time.  This interface serves
 * parameter sweeps (Ra, Pr, grid) over small cavities that alone cannot fill the GPU.
 *
 * Tiling.  The tile shape and the block shape are chosen by measurement (an autotuner
 * that times every candidate on the batch itself, lbm_batch_autotune) or set by the
 * caller.  Candidates: threads per block 128 or 256, the register budget the kernel is
 * built for (min_blocks), tiles of consecutive nodes or of whole x-rows, 1, 2 or 4 nodes
 * per thread and tile, and a persistent grid (blocks_per_sm blocks per SM, taking tiles
 * from a queue) or one block per tile.
 *
 * Errors and threading follow include/lbm.h: LBM_OK or a negative LBM_E* code, the
 * message in lbm_batch_last_error; a batch is not thread-safe.
 */
#ifndef LBM_BATCH_H
#define LBM_BATCH_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_batch lbm_batch;

/* Member states (lbm_batch_status). */
enum { LBM_MEMBER_ACTIVE = 0, LBM_MEMBER_CONVERGED = 1, LBM_MEMBER_DIVERGED = 2 };
/* Tile shapes: threads * tile_factor consecutive nodes of one cavity, or whole x-rows
 * (as many as fit in that budget; a longer row is cut into segments). */
enum { LBM_TILE_LINEAR = 0, LBM_TILE_ROWS = 1 };
/* How lbm_batch_step_with launches: captured graphs of the persistent kernel (the
 * default), one persistent-kernel launch per step, or, for comparison, one lbm_step
 * kernel launch per member and step (members one after another). */
enum { LBM_BATCH_GRAPH = 0, LBM_BATCH_LAUNCH = 1, LBM_BATCH_SEQUENTIAL = 2 };

typedef struct {
    int threads;       /* threads per block: 128 or 256 */
    int min_blocks;    /* resident blocks per SM the kernel build is constrained to (its
                          register budget).  FP32, D3Q15: 5 or 6 (128 threads), 2 or 3
                          (256); FP32, D3Q7: 6 or 7 (128), 2 or 3 (256); FP64: 1 */
    int mapping;       /* LBM_TILE_LINEAR or LBM_TILE_ROWS */
    int blocks_per_sm; /* persistent blocks per SM (1 .. the build's occupancy);
                          0 = one block per tile (not persistent) */
    int tile_factor;   /* nodes per tile = threads * tile_factor (1, 2 or 4): each thread
                          updates tile_factor nodes of a tile, one after another */
} lbm_batch_tiling;

typedef struct {
    lbm_batch_tiling tiling;
    double ms_per_step; /* mean of the timed launches (CUDA events) */
} lbm_batch_trial;

typedef struct {
    int precision;             /* LBM_FP64 or LBM_FP32 */
    uint64_t seed;             /* member m starts as lbm_create with seed + m */
    double noise_amp;          /* initial temperature noise (as lbm_options) */
    int residual_interval;     /* steps per graph and per convergence check: even, >= 2 */
    double steady_tol;         /* converged when max|dT| over one interval < steady_tol;
                                  0: never stop on convergence */
    void* cuda_stream;         /* cudaStream_t or NULL (legacy default stream) */
    void* device_arena;        /* optional caller-owned device memory (256-byte aligned) of
                                  at least lbm_batch_arena_bytes; NULL = library-owned */
    size_t device_arena_bytes;
    int autotune_steps;        /* timed launches per candidate when lbm_batch_create tunes */
    lbm_batch_tiling tiling;   /* threads == 0: tune at creation; else used as given */
    double timeout_s;          /* bound on every wait for the GPU */
} lbm_batch_options;

/* Defaults: FP32, seed 1, noise 1e-6, residual_interval 100, steady_tol 0, NULL stream
 * and arena, autotune_steps 3, tiling zero (tune), timeout 600 s. */
void lbm_batch_default_options(lbm_batch_options* opt);

/* Bytes of device memory a batch of these grids needs (0 if an argument is invalid). */
size_t lbm_batch_arena_bytes(int count, const lbm_grid* grids, int lattice, int precision);

/* Creates `count` >= 1 members; member m has grids[m] and params[m] (as for
 * lbm_create_params; e.g. from lbm_derive_params) and every member starts as lbm_create
 * would start it.  Every member must have fewer than 2^31 / 15 nodes.  Tunes the tiling
 * unless opt->tiling.threads != 0.  *out receives the batch.  LBM_EINVAL for an invalid
 * argument (including precisions other than FP64 / FP32 and an odd residual_interval),
 * LBM_ENOMEM, LBM_ECUDA, LBM_ETIMEOUT. */
int lbm_batch_create(int count, const lbm_grid* grids, int lattice, const lbm_params* params,
                     const lbm_batch_options* opt, lbm_batch** out);

/* Advances every active member by up to n steps (captured graphs; residual checks after
 * every residual_interval steps of the batch).  Stops early once no member is active.
 * Members that diverge are reported by lbm_batch_status, not by the return code. */
int lbm_batch_step(lbm_batch* b, int64_t n);

/* lbm_batch_step with an explicit launch mode (LBM_BATCH_GRAPH / _LAUNCH / _SEQUENTIAL);
 * all three compute the same states. */
int lbm_batch_step_with(lbm_batch* b, int64_t n, int mode);

/* Per-member state (LBM_MEMBER_*), steps done and last residual max|dT| (-1 before the
 * first check), into caller arrays of `count` entries; NULL pointers are skipped. */
int lbm_batch_status(const lbm_batch* b, int* state, int64_t* steps, double* residual);

/* The member as an lbm_ctx for lbm_fields, lbm_nusselt, lbm_residual,
 * lbm_get_populations, lbm_set_populations, lbm_get_params and lbm_steps_done.  It is
 * owned by the batch: lbm_step refuses it and lbm_destroy ignores it.  A member that
 * stopped keeps its state; lbm_set_populations on an active member takes effect at its
 * next step. */
int lbm_batch_member(lbm_batch* b, int index, lbm_ctx** member);

int lbm_batch_count(const lbm_batch* b);
/* Steps the batch has advanced (what every still-active member has done). */
int64_t lbm_batch_steps_done(const lbm_batch* b);
/* Nodes of the active members. */
int64_t lbm_batch_active_nodes(const lbm_batch* b);

/* Times every candidate tiling on the batch's current state with `trial_steps` launches
 * each (after one warm-up launch; the state is left unchanged: each trial launch reads
 * the current buffer and writes the other), adopts the fastest, and writes up to
 * max_trials results (in candidate order) to trials[] and their number to *n_trials
 * (either may be NULL). */
int lbm_batch_autotune(lbm_batch* b, int trial_steps, lbm_batch_trial* trials, int max_trials,
                       int* n_trials);

int lbm_batch_get_tiling(const lbm_batch* b, lbm_batch_tiling* out);
/* LBM_EINVAL if the tiling is not one of the candidates of the batch's precision and
 * lattice, or blocks_per_sm exceeds the build's occupancy. */
int lbm_batch_set_tiling(lbm_batch* b, const lbm_batch_tiling* tiling);

int lbm_batch_synchronize(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);
/* Frees the batch and all its members (NULL: no-op). */
void lbm_batch_destroy(lbm_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_BATCH_H */
