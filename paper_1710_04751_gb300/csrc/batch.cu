// batch.cu -- many independent cavities advanced by one persistent kernel per step,
// captured in CUDA graphs, with a batched convergence check and a tiling autotuner
// (include/lbm_batch.h).  The node update is the one of the single-cavity kernels
// (node.cuh), so each member follows the trajectory lbm_step would give it.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "context.h"
#include "lbm_batch.h"
#include "node.cuh"

using namespace lbm;

namespace lbm {

// One member as the kernels see it: its parameters, its two population buffers and its
// residual snapshot.
template <typename S>
struct BatchMember {
    ParamsOf<S> p;
    S* F[2];
    S* G[2];
    typename Storage<S>::real* snap;
    int fast;  // the cavity interior body applies (boundary 0, 32-bit node indices)
    int pad;
    // division of node / row indices by nx and ny as a multiplication: q = (n M) >> s
    unsigned long long div_nx, div_ny;
    int shift_nx, shift_ny;
};

// Division by an invariant integer d >= 1 as a multiplication (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994).  With l = ceil(log2 d),
// M = ceil(2^(32+l) / d) and e = M d - 2^(32+l) in [0, d):
//   n M / 2^(32+l) = n / d + n e / (d 2^(32+l)).
// The fractional part of n / d is at most (d - 1) / d, and the added term stays below 1 / d
// whenever n e < 2^(32+l), which holds for every n < 2^31 since e < d <= 2^l.  So
// floor(n M / 2^(32+l)) = floor(n / d).  (M <= 2^33, so n M fits in 64 bits.)
inline void invariant_divisor(int d, unsigned long long* M, int* shift) {
    int l = 0;
    while ((1ll << l) < d) ++l;
    const unsigned long long p = 1ull << (32 + l);
    *M = p / (unsigned long long)d + (p % (unsigned long long)d != 0);
    *shift = 32 + l;
}
__device__ __forceinline__ int div_invariant(int n, unsigned long long M, int shift) {
    return (int)(((unsigned long long)(unsigned)n * M) >> shift);
}

// A run of `count` nodes of one member starting at node c0 (count <= nodes per tile).
struct BatchTile {
    int member, c0, count, pad;
};

// Copies `words` 32-bit words with the whole block (caller synchronises).
__device__ __forceinline__ void block_copy(void* dst, const void* src, int words) {
    const uint32_t* s = static_cast<const uint32_t*>(src);
    uint32_t* d = static_cast<uint32_t*>(dst);
    for (int w = threadIdx.x; w < words; w += blockDim.x) d[w] = s[w];
}

// The member table lives in shared memory: all of it when it fits (cache_all, loaded once
// per launch), else only the current tile's member, reloaded when the member changes.
template <typename S>
__device__ __forceinline__ const BatchMember<S>& member_of(BatchMember<S>* cache,
                                                          const BatchMember<S>* members, int m,
                                                          int cache_all, int& loaded) {
    if (cache_all) return cache[m];
    if (m != loaded) {  // block-uniform
        __syncthreads();
        block_copy(cache, members + m, (int)(sizeof(BatchMember<S>) / 4));
        __syncthreads();
        loaded = m;
    }
    return cache[0];
}

template <typename S, int Q, bool UNIT>
__device__ __forceinline__ void batch_node(const BatchMember<S>& m, const ParamsOf<S>& p, int c,
                                           int parity) {
    const int nx = p.nx, ny = p.ny;
    const int row = div_invariant(c, m.div_nx, m.shift_nx);
    const int i = c - row * nx;
    const int k = div_invariant(row, m.div_ny, m.shift_ny);
    const int j = row - k * ny;
    const S* Fin = m.F[parity];
    const S* Gin = m.G[parity];
    S* Fout = m.F[parity ^ 1];
    S* Gout = m.G[parity ^ 1];
    if (m.fast && j >= 1 && j + 1 < ny && k >= 1 && k + 1 < p.nz)
        cavity_node<S, Q, true, UNIT>(Fin, Gin, nullptr, Fout, Gout, nullptr, p, i, j, k);
    else
        cavity_node<S, Q, false, UNIT>(Fin, Gin, nullptr, Fout, Gout, nullptr, p, i, j, k);
}

// Parameters of a member of a sweep: every field of `base` (a kernel parameter, so it
// stays in the constant bank) except those members of a sweep differ in -- the shear
// rate omega_nu (flow moments 4..8), the scalar rate omega_phi (thermal moments 1..3),
// g beta and the grid -- which come from the member record.
template <typename S>
__device__ __forceinline__ ParamsOf<S> sweep_params(const ParamsOf<S>& base, const ParamsOf<S>& mp) {
    ParamsOf<S> p = base;
    const auto om_nu = mp.om_f[4], om_phi = mp.om_g[1];
#pragma unroll
    for (int b = 4; b <= 8; ++b) p.om_f[b] = om_nu;
#pragma unroll
    for (int b = 1; b <= 3; ++b) p.om_g[b] = om_phi;
    p.gbeta = mp.gbeta;
    p.nx = mp.nx;
    p.ny = mp.ny;
    p.nz = mp.nz;
    p.ncell = mp.ncell;
    p.plane = mp.plane;
    return p;
}

// One time step of every member in the tile list.  Blocks take tiles from a queue in
// list order (an atomic counter per step parity), so the whole grid works on
// neighbouring tiles at any moment -- the planes a pull reads again (z +- 1) are still in
// L2 -- and an SM that runs ahead takes more tiles.  Each block claims its next tile
// while it works on the current one.  The launch for parity p uses queue[p] and zeroes
// queue[p ^ 1] for the launch that follows it in the stream.
// MODE: 0 general members; 1 a sweep (the members differ only in the fields sweep_params
// takes from them); 2 a sweep at the paper's unit higher-order rates (collide_unit.cuh).
template <typename S, int Q, int THREADS, int MINB, int MODE>
__global__ void __launch_bounds__(THREADS, MINB)
    batch_step_kernel(const BatchMember<S>* __restrict__ members, int count,
                      const BatchTile* __restrict__ tiles, const int* __restrict__ n_tiles,
                      int* __restrict__ queue, int cache_all, int parity,
                      const ParamsOf<S> base) {
    extern __shared__ __align__(16) unsigned char batch_smem[];
    __shared__ int next_tile;
    BatchMember<S>* cache = reinterpret_cast<BatchMember<S>*>(batch_smem);
    if (cache_all) block_copy(cache, members, (int)(count * sizeof(BatchMember<S>) / 4));
    if (threadIdx.x == 0) {
        if (blockIdx.x == 0) queue[parity ^ 1] = 0;
        next_tile = atomicAdd(queue + parity, 1);
    }
    __syncthreads();
    const int nt = *n_tiles;
    int loaded = -1;
    for (int t = next_tile; t < nt; t = next_tile) {
        const BatchTile tile = tiles[t];
        int claim = 0;
        if (threadIdx.x == 0) claim = atomicAdd(queue + parity, 1);
        const BatchMember<S>& m = member_of<S>(cache, members, tile.member, cache_all, loaded);
        for (int c = threadIdx.x; c < tile.count; c += THREADS) {
            if constexpr (MODE > 0)
                batch_node<S, Q, MODE == 2>(m, sweep_params<S>(base, m.p), tile.c0 + c, parity);
            else
                batch_node<S, Q, false>(m, m.p, tile.c0 + c, parity);
        }
        __syncthreads();  // every thread has read next_tile for this iteration
        if (threadIdx.x == 0) next_tile = claim;
        __syncthreads();
    }
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block max of `local` into bits[m] (non-negative doubles order like their bit
// patterns) and the non-finite flag into nonfinite[m].  Called by every thread.
__device__ __forceinline__ void flush_residual(double local, int bad, int m, double* red,
                                               unsigned long long* bits, int* nonfinite) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    local = warp_max_d(local);
    const bool any_bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        red[warp] = local;
        if (any_bad) atomicOr(nonfinite + m, 1);
    }
    __syncthreads();
    if (warp == 0) {
        double v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        v = warp_max_d(v);
        if (lane == 0) atomicMax(bits + m, (unsigned long long)__double_as_longlong(v));
    }
    __syncthreads();
}

// Convergence check of every member in the tile list: max over its nodes of
// |T - T_snapshot| into bits[member], snapshot <- T, and a flag for a non-finite T.
// T = sum_a g~_a - R/2 (Eq. 25 on the post-collision populations).
template <typename S, int Q>
__global__ void __launch_bounds__(256)
    batch_residual_kernel(const BatchMember<S>* __restrict__ members, int count,
                          const BatchTile* __restrict__ tiles, const int* __restrict__ n_tiles,
                          int cache_all, int parity, unsigned long long* __restrict__ bits,
                          int* __restrict__ nonfinite) {
    using real = typename Storage<S>::real;
    extern __shared__ __align__(16) unsigned char batch_smem[];
    __shared__ double red[8];
    BatchMember<S>* cache = reinterpret_cast<BatchMember<S>*>(batch_smem);
    if (cache_all) {
        block_copy(cache, members, (int)(count * sizeof(BatchMember<S>) / 4));
        __syncthreads();
    }
    const int nt = *n_tiles;
    int loaded = -1, cur = -1, bad = 0;
    double local = 0.0;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const BatchTile tile = tiles[t];
        if (tile.member != cur) {  // block-uniform
            if (cur >= 0) flush_residual(local, bad, cur, red, bits, nonfinite);
            local = 0.0;
            bad = 0;
            cur = tile.member;
        }
        const BatchMember<S>& m = member_of<S>(cache, members, tile.member, cache_all, loaded);
        for (int n = threadIdx.x; n < tile.count; n += blockDim.x) {
            const int64_t c = tile.c0 + n;
            const S* G = m.G[parity];
            real T = real(0);
#pragma unroll
            for (int a = 0; a < Q; ++a) T += (real)G[a * m.p.plane + c];
            T -= real(0.5) * m.p.heat_source;
            if (!isfinite(T)) bad = 1;
            const double d = fabs((double)T - (double)m.snap[c]);
            if (d > local) local = d;
            m.snap[c] = T;
        }
    }
    if (cur >= 0) flush_residual(local, bad, cur, red, bits, nonfinite);
}

// The kernel builds of one storage type and lattice: (threads, register budget).
struct Variant {
    int threads, min_blocks;
    const void* fn;
};

template <typename S, int Q, int MODE>
static int step_variants(Variant* out) {
    if constexpr (sizeof(typename Storage<S>::real) == 8) {
        out[0] = {128, 1, (const void*)batch_step_kernel<S, Q, 128, 1, MODE>};
        out[1] = {256, 1, (const void*)batch_step_kernel<S, Q, 256, 1, MODE>};
        return 2;
    } else if constexpr (Q == 15 && MODE == 0) {
        // general members: D3Q15 needs 96 registers without spills (every parameter comes
        // from shared memory, none from the constant bank); 80 spills 60 bytes
        out[0] = {128, 5, (const void*)batch_step_kernel<S, Q, 128, 5, MODE>};
        out[1] = {128, 6, (const void*)batch_step_kernel<S, Q, 128, 6, MODE>};
        out[2] = {256, 2, (const void*)batch_step_kernel<S, Q, 256, 2, MODE>};
        out[3] = {256, 3, (const void*)batch_step_kernel<S, Q, 256, 3, MODE>};
        return 4;
    } else if constexpr (MODE == 2) {
        // unit higher-order rates: fewer live moments (D3Q15: 80 registers without spills
        // at 6 blocks of 128 or 3 of 256; 72 spill 8 bytes)
        out[0] = {128, 6, (const void*)batch_step_kernel<S, Q, 128, 6, MODE>};
        out[1] = {128, 7, (const void*)batch_step_kernel<S, Q, 128, 7, MODE>};
        out[2] = {256, 2, (const void*)batch_step_kernel<S, Q, 256, 2, MODE>};
        out[3] = {256, 3, (const void*)batch_step_kernel<S, Q, 256, 3, MODE>};
        return 4;
    } else {
        out[0] = {128, 6, (const void*)batch_step_kernel<S, Q, 128, 6, MODE>};
        out[1] = {128, 7, (const void*)batch_step_kernel<S, Q, 128, 7, MODE>};
        out[2] = {256, 2, (const void*)batch_step_kernel<S, Q, 256, 2, MODE>};
        out[3] = {256, 3, (const void*)batch_step_kernel<S, Q, 256, 3, MODE>};
        return 4;
    }
}

template <typename S>
using BatchStepFn = void (*)(const BatchMember<S>*, int, const BatchTile*, const int*, int*, int,
                             int, const ParamsOf<S>);

}  // namespace lbm

constexpr int kMaxVariants = 4;
constexpr size_t kCacheAllBytes = 40 * 1024;  // member tables up to this size stay in smem

struct lbm_batch {
    int count = 0, Q = 15, precision = LBM_FP32, device = 0, sm_count = 0;
    lbm_batch_options opt{};
    cudaStream_t stream = nullptr;   // caller's stream: all work runs here
    cudaStream_t capture = nullptr;  // private stream the graphs are captured on
    void* arena = nullptr;
    bool own_arena = false;
    std::vector<lbm_ctx*> members;
    std::vector<int> state;
    std::vector<DevParams<double>> params64;  // per member, for the sequential mode
    std::vector<DevParams<float>> params32;
    size_t member_bytes = 0;
    void* d_members = nullptr;
    BatchTile* d_tiles = nullptr;
    int* d_ntiles = nullptr;
    int* d_queue = nullptr;  // two tile-queue counters (one per step parity)
    unsigned long long* d_bits = nullptr;
    int* d_nonfinite = nullptr;
    int max_tiles = 0, n_tiles = 0;
    BatchTile* h_tiles = nullptr;  // pinned
    int* h_ntiles = nullptr;       // pinned
    unsigned long long* h_bits = nullptr;  // pinned, count
    int* h_nonfinite = nullptr;            // pinned, count
    lbm_batch_tiling tiling{};
    Variant variant{};
    int grid = 0, cache_all = 0;
    bool sweep = false;  // members differ only in omega_nu, omega_phi, g beta and the grid
    bool unit = false;   // ... and all relax their higher orders at the paper's unit rates
    size_t smem = 0;
    cudaGraphExec_t graph = nullptr;
    int64_t steps = 0;
    std::string err;
};

static int bfail(lbm_batch* b, int code, const char* fmt, const char* detail = nullptr) {
    return record_error(b ? &b->err : nullptr, code, fmt, detail);
}

#define BATCH_CUDA(b, call)                                                          \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return bfail((b), LBM_ECUDA, "CUDA error in " #call ": %s",              \
                         cudaGetErrorString(e_));                                    \
    } while (0)

static int bwait(lbm_batch* b) { return wait_stream_for(b->stream, b->opt.timeout_s, &b->err); }

// Nodes of a member below which 32-bit population offsets are exact (15 planes).
static bool member_fits(const lbm_grid& g) {
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    return g.nx >= 1 && g.ny >= 1 && g.nz >= 1 && 15 * ((n + 63) / 64 * 64) < (int64_t(1) << 31);
}

// Tiles of one member for a mapping and block size, appended to out (or counted).
static int64_t member_tiles(const lbm_grid& g, int member, int tile_nodes, int mapping,
                            BatchTile* out) {
    const int threads = tile_nodes;
    const int nx = g.nx;
    const int64_t ncell = (int64_t)g.nx * g.ny * g.nz, rows = (int64_t)g.ny * g.nz;
    int64_t n = 0;
    auto put = [&](int64_t c0, int64_t cnt) {
        if (out) out[n] = BatchTile{member, (int)c0, (int)cnt, 0};
        ++n;
    };
    if (mapping == LBM_TILE_LINEAR) {
        for (int64_t c0 = 0; c0 < ncell; c0 += threads) put(c0, std::min<int64_t>(threads, ncell - c0));
    } else if (nx <= threads) {
        const int64_t k = threads / nx;
        for (int64_t r = 0; r < rows; r += k) put(r * nx, std::min<int64_t>(k, rows - r) * nx);
    } else {
        for (int64_t r = 0; r < rows; ++r)
            for (int64_t s = 0; s < nx; s += threads) put(r * nx + s, std::min<int64_t>(threads, nx - s));
    }
    return n;
}

static int64_t max_tile_count(int count, const lbm_grid* grids) {
    int64_t best = 0;
    for (int threads : {128, 256})  // the smallest tiles give the most
        for (int mapping : {LBM_TILE_LINEAR, LBM_TILE_ROWS}) {
            int64_t n = 0;
            for (int m = 0; m < count; ++m) n += member_tiles(grids[m], m, threads, mapping, nullptr);
            best = std::max(best, n);
        }
    return best;
}

static size_t member_table_bytes(int precision) {
    return precision == LBM_FP64 ? sizeof(BatchMember<double>) : sizeof(BatchMember<float>);
}

struct BatchLayout {
    std::vector<size_t> member_off;
    size_t members, tiles, ntiles, bits, nonfinite, total;
};

static BatchLayout batch_layout(int count, const lbm_grid* grids, int lattice, int precision) {
    BatchLayout L;
    size_t off = 0;
    for (int m = 0; m < count; ++m) {
        L.member_off.push_back(off);
        off = align_up(off + context_arena_bytes(&grids[m], lattice, precision), 256);
    }
    L.members = off;
    off = align_up(off + count * member_table_bytes(precision), 256);
    L.tiles = off;
    off = align_up(off + max_tile_count(count, grids) * sizeof(BatchTile), 256);
    L.ntiles = off;  // the tile count, then (16 bytes on) the two queue counters
    off = align_up(off + 64, 256);
    L.bits = off;
    off = align_up(off + count * sizeof(unsigned long long), 256);
    L.nonfinite = off;
    off = align_up(off + count * sizeof(int), 256);
    L.total = off;
    return L;
}

// Kernel builds of the batch's precision and lattice.
static int batch_variants(const lbm_batch* b, Variant* out) {
    if (b->precision == LBM_FP64) {
        if (b->sweep && b->unit)
            return b->Q == 15 ? step_variants<double, 15, 2>(out) : step_variants<double, 7, 2>(out);
        if (b->sweep) return b->Q == 15 ? step_variants<double, 15, 1>(out) : step_variants<double, 7, 1>(out);
        return b->Q == 15 ? step_variants<double, 15, 0>(out) : step_variants<double, 7, 0>(out);
    }
    if (b->sweep && b->unit)
        return b->Q == 15 ? step_variants<float, 15, 2>(out) : step_variants<float, 7, 2>(out);
    if (b->sweep) return b->Q == 15 ? step_variants<float, 15, 1>(out) : step_variants<float, 7, 1>(out);
    return b->Q == 15 ? step_variants<float, 15, 0>(out) : step_variants<float, 7, 0>(out);
}

// Shared memory of a launch: the whole member table for a persistent grid when it fits
// (each block loads it once), else one member record (reloaded on member changes).
static size_t smem_for(const lbm_batch* b, int blocks_per_sm, int* cache_all) {
    const size_t all = (size_t)b->count * b->member_bytes;
    *cache_all = blocks_per_sm > 0 && all <= kCacheAllBytes;
    return *cache_all ? all : b->member_bytes;
}

// Members of a sweep differ only in omega_nu (flow moments 4..8, equal within a member),
// omega_phi (thermal moments 1..3, likewise), g beta, U0 and the grid.
static bool is_sweep(int count, const lbm_params* P) {
    for (int m = 0; m < count; ++m) {
        const lbm_params &a = P[m], &z = P[0];
        for (int b = 5; b <= 8; ++b)
            if (a.omega_f[b] != a.omega_f[4]) return false;
        for (int b = 2; b <= 3; ++b)
            if (a.omega_g[b] != a.omega_g[1]) return false;
        for (int b = 0; b < 15; ++b) {
            if ((b < 4 || b > 8) && a.omega_f[b] != z.omega_f[b]) return false;
            if ((b < 1 || b > 3) && a.omega_g[b] != z.omega_g[b]) return false;
        }
        if (a.T_hot != z.T_hot || a.T_cold != z.T_cold || a.cs2_phi != z.cs2_phi ||
            a.heat_source != z.heat_source || a.e4_mode != z.e4_mode ||
            a.adiabatic_mode != z.adiabatic_mode || a.boundary != z.boundary)
            return false;
        for (int d = 0; d < 3; ++d)
            if (a.ext_force[d] != z.ext_force[d]) return false;
    }
    return true;
}

// Rebuilds the tile list of the active members for the current tiling and uploads it.
static int rebuild_tiles(lbm_batch* b) {
    int rc = bwait(b);  // the pinned staging may still be in flight
    if (rc != LBM_OK) return rc;
    int64_t n = 0;
    for (int m = 0; m < b->count; ++m)
        if (b->state[m] == LBM_MEMBER_ACTIVE)
            n += member_tiles(b->members[m]->grid, m, b->tiling.threads * b->tiling.tile_factor,
                              b->tiling.mapping,
                              b->h_tiles + n);
    b->n_tiles = (int)n;
    *b->h_ntiles = (int)n;
    if (n > 0)
        BATCH_CUDA(b, cudaMemcpyAsync(b->d_tiles, b->h_tiles, n * sizeof(BatchTile),
                                      cudaMemcpyHostToDevice, b->stream));
    BATCH_CUDA(b, cudaMemcpyAsync(b->d_ntiles, b->h_ntiles, sizeof(int), cudaMemcpyHostToDevice,
                                  b->stream));
    return LBM_OK;
}

// Adopts a tiling: finds its kernel build, checks the occupancy, rebuilds the tiles.
static int apply_tiling(lbm_batch* b, const lbm_batch_tiling& t) {
    Variant vs[kMaxVariants];
    const int nv = batch_variants(b, vs);
    const Variant* v = nullptr;
    for (int i = 0; i < nv; ++i)
        if (vs[i].threads == t.threads && vs[i].min_blocks == t.min_blocks) v = &vs[i];
    if (!v || (t.mapping != LBM_TILE_LINEAR && t.mapping != LBM_TILE_ROWS) || t.blocks_per_sm < 0 ||
        (t.tile_factor != 1 && t.tile_factor != 2 && t.tile_factor != 4))
        return bfail(b, LBM_EINVAL, "tiling is not a candidate of this precision and lattice%s");
    int cache_all = 0;
    const size_t smem = smem_for(b, t.blocks_per_sm, &cache_all);
    int occ = 0;
    BATCH_CUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v->fn, v->threads, smem));
    if (occ < 1) return bfail(b, LBM_EINVAL, "tiling does not fit on an SM%s");
    if (t.blocks_per_sm > occ) return bfail(b, LBM_EINVAL, "blocks_per_sm exceeds the occupancy%s");
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->tiling = t;
    b->variant = *v;
    b->cache_all = cache_all;
    b->smem = smem;
    int rc = rebuild_tiles(b);
    if (rc != LBM_OK) return rc;
    b->grid = t.blocks_per_sm > 0 ? b->sm_count * t.blocks_per_sm : std::max(1, b->n_tiles);
    return LBM_OK;
}

template <typename S>
static cudaError_t launch_batch_step(const lbm_batch* b, int parity, cudaStream_t st) {
    const auto fn = reinterpret_cast<BatchStepFn<S>>(b->variant.fn);
    const ParamsOf<S>* base;
    if constexpr (sizeof(typename Storage<S>::real) == 8) base = &b->params64[0];
    else base = &b->params32[0];
    fn<<<b->grid, b->variant.threads, b->smem, st>>>(
        static_cast<const BatchMember<S>*>(b->d_members), b->count, b->d_tiles, b->d_ntiles,
        b->d_queue, b->cache_all, parity, *base);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_batch_residual(const lbm_batch* b, int parity, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b->d_bits, 0, b->count * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_nonfinite, 0, b->count * sizeof(int), st);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(b->n_tiles, b->sm_count * 4));
    const auto* mem = static_cast<const BatchMember<S>*>(b->d_members);
    if (b->Q == 15)
        batch_residual_kernel<S, 15><<<grid, b->variant.threads, b->smem, st>>>(
            mem, b->count, b->d_tiles, b->d_ntiles, b->cache_all, parity, b->d_bits, b->d_nonfinite);
    else
        batch_residual_kernel<S, 7><<<grid, b->variant.threads, b->smem, st>>>(
            mem, b->count, b->d_tiles, b->d_ntiles, b->cache_all, parity, b->d_bits, b->d_nonfinite);
    return cudaGetLastError();
}

template <typename Fn>
static int with_real(const lbm_batch* b, Fn&& fn) {
    return b->precision == LBM_FP64 ? fn(double{}) : fn(float{});
}

static int n_active(const lbm_batch* b) {
    return (int)std::count(b->state.begin(), b->state.end(), (int)LBM_MEMBER_ACTIVE);
}

// Bookkeeping after k steps of every active member.
static void advance(lbm_batch* b, int64_t k) {
    b->steps += k;
    for (int m = 0; m < b->count; ++m)
        if (b->state[m] == LBM_MEMBER_ACTIVE) {
            b->members[m]->steps += k;
            b->members[m]->cur = (int)(b->steps & 1);
        }
}

// Reads the residuals of the last check, stops converged and diverged members.
static int check(lbm_batch* b) {
    BATCH_CUDA(b, cudaMemcpyAsync(b->h_bits, b->d_bits, b->count * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(b, cudaMemcpyAsync(b->h_nonfinite, b->d_nonfinite, b->count * sizeof(int),
                                  cudaMemcpyDeviceToHost, b->stream));
    int rc = bwait(b);
    if (rc != LBM_OK) return rc;
    bool changed = false;
    for (int m = 0; m < b->count; ++m) {
        if (b->state[m] != LBM_MEMBER_ACTIVE) continue;
        double r;
        memcpy(&r, &b->h_bits[m], sizeof r);
        b->members[m]->last_residual = r;
        if (b->h_nonfinite[m]) {
            b->state[m] = LBM_MEMBER_DIVERGED;
            changed = true;
        } else if (b->opt.steady_tol > 0 && r < b->opt.steady_tol) {
            b->state[m] = LBM_MEMBER_CONVERGED;
            changed = true;
        }
    }
    if (!changed) return LBM_OK;
    rc = rebuild_tiles(b);
    if (rc != LBM_OK) return rc;
    if (b->tiling.blocks_per_sm == 0) b->grid = std::max(1, b->n_tiles);
    if (b->graph && b->tiling.blocks_per_sm == 0) {  // its grid was sized for more tiles
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return LBM_OK;
}

// Captures residual_interval steps starting at parity 0 and the check that follows.
static int capture_graph(lbm_batch* b) {
    const int I = b->opt.residual_interval;
    BATCH_CUDA(b, cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    with_real(b, [&](auto tag) {
        using S = decltype(tag);
        for (int s = 0; s < I && e == cudaSuccess; ++s) e = launch_batch_step<S>(b, s & 1, b->capture);
        if (e == cudaSuccess) e = launch_batch_residual<S>(b, I & 1, b->capture);
        return 0;
    });
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, LBM_ECUDA, "graph capture failed: %s",
                     cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return bfail(b, LBM_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

template <typename S>
static int sequential_step(lbm_batch* b, int parity) {
    for (int m = 0; m < b->count; ++m) {
        if (b->state[m] != LBM_MEMBER_ACTIVE) continue;
        const ParamsOf<S>* p;
        if constexpr (sizeof(typename Storage<S>::real) == 8) p = &b->params64[m];
        else p = &b->params32[m];
        BATCH_CUDA(b, launch_step<S>(b->members[m]->dev, parity, *p, b->stream));
    }
    return LBM_OK;
}

extern "C" void lbm_batch_default_options(lbm_batch_options* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = LBM_FP32;
    o->seed = 1;
    o->noise_amp = 1e-6;
    o->residual_interval = 100;
    o->steady_tol = 0.0;
    o->autotune_steps = 3;
    o->timeout_s = 600.0;
}

static bool valid_batch_args(int count, const lbm_grid* grids, int lattice, int precision) {
    if (count < 1 || !grids) return false;
    if (lattice != LBM_THERMAL_D3Q15 && lattice != LBM_THERMAL_D3Q7) return false;
    if (precision != LBM_FP64 && precision != LBM_FP32) return false;
    for (int m = 0; m < count; ++m)
        if (!member_fits(grids[m])) return false;
    return true;
}

extern "C" size_t lbm_batch_arena_bytes(int count, const lbm_grid* grids, int lattice, int precision) {
    if (!valid_batch_args(count, grids, lattice, precision)) return 0;
    return batch_layout(count, grids, lattice, precision).total;
}

extern "C" void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    {
        DeviceGuard g(b->device);
        bwait(b);
        if (b->graph) cudaGraphExecDestroy(b->graph);
        if (b->capture) cudaStreamDestroy(b->capture);
        for (lbm_ctx* c : b->members) destroy_context(c);
        if (b->own_arena && b->arena) cudaFree(b->arena);
        if (b->h_tiles) cudaFreeHost(b->h_tiles);
        if (b->h_bits) cudaFreeHost(b->h_bits);
    }
    delete b;
}

template <typename S>
static void fill_member_table(lbm_batch* b, std::vector<unsigned char>& table) {
    table.assign((size_t)b->count * sizeof(BatchMember<S>), 0);
    auto* t = reinterpret_cast<BatchMember<S>*>(table.data());
    for (int m = 0; m < b->count; ++m) {
        lbm_ctx* c = b->members[m];
        t[m].p = dev_params<typename Storage<S>::real>(c);
        for (int s = 0; s < 2; ++s) {
            t[m].F[s] = static_cast<S*>(c->dev.F[s]);
            t[m].G[s] = static_cast<S*>(c->dev.G[s]);
        }
        t[m].snap = static_cast<typename Storage<S>::real*>(c->dev.snap);
        t[m].fast = c->params.boundary == LBM_BC_CAVITY;
        invariant_divisor(c->grid.nx, &t[m].div_nx, &t[m].shift_nx);
        invariant_divisor(c->grid.ny, &t[m].div_ny, &t[m].shift_ny);
    }
}

extern "C" int lbm_batch_create(int count, const lbm_grid* grids, int lattice,
                                const lbm_params* params, const lbm_batch_options* opt,
                                lbm_batch** out) {
    if (!out) return bfail(nullptr, LBM_EINVAL, "out is NULL%s");
    *out = nullptr;
    lbm_batch_options o;
    if (opt) o = *opt; else lbm_batch_default_options(&o);
    if (!params || !valid_batch_args(count, grids, lattice, o.precision))
        return bfail(nullptr, LBM_EINVAL,
                     "invalid batch: count >= 1, grids below 2^31/15 nodes, lattice 15 or 7, FP64 or FP32%s");
    if (o.residual_interval < 2 || (o.residual_interval & 1) || !(o.steady_tol >= 0) ||
        !(o.timeout_s > 0) || o.autotune_steps < 0)
        return bfail(nullptr, LBM_EINVAL, "residual_interval must be even and >= 2; steady_tol >= 0%s");

    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ENOMEM, "host allocation failed%s");
    b->count = count;
    b->Q = lattice;
    b->precision = o.precision;
    b->opt = o;
    b->stream = (cudaStream_t)o.cuda_stream;
    b->state.assign(count, LBM_MEMBER_ACTIVE);
    b->member_bytes = member_table_bytes(o.precision);
    b->sweep = is_sweep(count, params);
    b->unit = true;  // a sweep's higher-order rates are those of member 0
    for (int bb = 9; bb < 15; ++bb) b->unit = b->unit && params[0].omega_f[bb] == 1.0;
    for (int bb = 4; bb < lattice; ++bb) b->unit = b->unit && params[0].omega_g[bb] == 1.0;
    auto bail = [&](int rc) {
        std::string msg = b->err;
        lbm_batch_destroy(b);
        set_last_error(msg.c_str());
        return rc;
    };
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return bfail(nullptr, LBM_ECUDA, "no CUDA device%s");
    }
    if (cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
        return bail(bfail(b, LBM_ECUDA, "cudaDeviceGetAttribute failed%s"));
    const BatchLayout L = batch_layout(count, grids, lattice, o.precision);
    if (o.device_arena) {
        if (o.device_arena_bytes < L.total || ((uintptr_t)o.device_arena & 255))
            return bail(bfail(b, LBM_ENOMEM, "device arena too small or not 256-byte aligned%s"));
        b->arena = o.device_arena;
    } else {
        const cudaError_t e = cudaMalloc(&b->arena, L.total);
        if (e != cudaSuccess) {
            b->arena = nullptr;
            return bail(bfail(b, LBM_ENOMEM, "cudaMalloc of the batch failed: %s", cudaGetErrorString(e)));
        }
        b->own_arena = true;
    }
    char* base = static_cast<char*>(b->arena);
    b->d_members = base + L.members;
    b->d_tiles = reinterpret_cast<BatchTile*>(base + L.tiles);
    b->d_ntiles = reinterpret_cast<int*>(base + L.ntiles);
    b->d_queue = b->d_ntiles + 4;
    b->d_bits = reinterpret_cast<unsigned long long*>(base + L.bits);
    b->d_nonfinite = reinterpret_cast<int*>(base + L.nonfinite);
    b->max_tiles = (int)max_tile_count(count, grids);
    // pinned staging: tiles + tile count in one block, residual bits + flags in another
    if (cudaMallocHost(&b->h_tiles, b->max_tiles * sizeof(BatchTile) + 16) != cudaSuccess ||
        cudaMallocHost(&b->h_bits, count * (sizeof(unsigned long long) + sizeof(int))) != cudaSuccess)
        return bail(bfail(b, LBM_ENOMEM, "cudaMallocHost failed%s"));
    b->h_ntiles = reinterpret_cast<int*>(b->h_tiles + b->max_tiles);
    b->h_nonfinite = reinterpret_cast<int*>(b->h_bits + count);
    if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess)
        return bail(bfail(b, LBM_ECUDA, "cudaStreamCreate failed%s"));
    if (cudaMemsetAsync(b->d_ntiles, 0, 64, b->stream) != cudaSuccess)
        return bail(bfail(b, LBM_ECUDA, "cudaMemsetAsync failed%s"));

    for (int m = 0; m < count; ++m) {
        lbm_options mo;
        lbm_default_options(&mo);
        mo.precision = o.precision;
        mo.seed = o.seed + (uint64_t)m;
        mo.noise_amp = o.noise_amp;
        mo.residual_interval = 0;  // checks are the batch's
        mo.cuda_stream = o.cuda_stream;
        mo.device_arena = base + L.member_off[m];
        mo.device_arena_bytes = context_arena_bytes(&grids[m], lattice, o.precision);
        mo.timeout_s = o.timeout_s;
        lbm_ctx* c = nullptr;
        const int rc = lbm_create_params(&grids[m], lattice, &params[m], &mo, &c);
        if (rc != LBM_OK) {
            b->err = std::string("member ") + std::to_string(m) + ": " + lbm_last_error(nullptr);
            return bail(rc);
        }
        c->owner = b;
        b->members.push_back(c);
        b->params64.push_back(dev_params<double>(c));
        b->params32.push_back(dev_params<float>(c));
    }
    std::vector<unsigned char> table;
    if (o.precision == LBM_FP64) fill_member_table<double>(b, table);
    else fill_member_table<float>(b, table);
    if (cudaMemcpyAsync(b->d_members, table.data(), table.size(), cudaMemcpyHostToDevice, b->stream) !=
        cudaSuccess)
        return bail(bfail(b, LBM_ECUDA, "upload of the member table failed%s"));
    int rc = bwait(b);  // the table is a host vector: finish the copy before it goes
    if (rc != LBM_OK) return bail(rc);

    if (o.tiling.threads != 0) {
        rc = apply_tiling(b, o.tiling);
    } else {
        Variant vs[kMaxVariants];
        batch_variants(b, vs);
        int occ = 0, cache_all = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, vs[0].fn, vs[0].threads,
                                                      smem_for(b, 1, &cache_all));
        rc = apply_tiling(b, lbm_batch_tiling{vs[0].threads, vs[0].min_blocks, LBM_TILE_LINEAR,
                                              std::max(1, occ), 1});
        if (rc == LBM_OK && o.autotune_steps > 0)
            rc = lbm_batch_autotune(b, o.autotune_steps, nullptr, 0, nullptr);
    }
    if (rc != LBM_OK) return bail(rc);
    *out = b;
    return LBM_OK;
}

extern "C" int lbm_batch_step_with(lbm_batch* b, int64_t n, int mode) {
    NvtxRange nvtx("lbm_batch_step");
    if (!b || n < 0 || mode < LBM_BATCH_GRAPH || mode > LBM_BATCH_SEQUENTIAL)
        return bfail(b, LBM_EINVAL, "invalid batch, step count or mode%s");
    DeviceGuard g(b->device);
    const int I = b->opt.residual_interval;
    while (n > 0 && n_active(b) > 0) {
        if (mode == LBM_BATCH_GRAPH && b->steps % I == 0 && n >= I) {
            if (!b->graph) {
                int rc = capture_graph(b);
                if (rc != LBM_OK) return rc;
            }
            BATCH_CUDA(b, cudaGraphLaunch(b->graph, b->stream));
            advance(b, I);
            n -= I;
            int rc = check(b);
            if (rc != LBM_OK) return rc;
            continue;
        }
        const int parity = (int)(b->steps & 1);
        int rc = with_real(b, [&](auto tag) {
            using S = decltype(tag);
            if (mode == LBM_BATCH_SEQUENTIAL) return sequential_step<S>(b, parity);
            BATCH_CUDA(b, launch_batch_step<S>(b, parity, b->stream));
            return LBM_OK;
        });
        if (rc != LBM_OK) return rc;
        advance(b, 1);
        n -= 1;
        if (b->steps % I == 0) {
            rc = with_real(b, [&](auto tag) {
                BATCH_CUDA(b, launch_batch_residual<decltype(tag)>(b, (int)(b->steps & 1), b->stream));
                return LBM_OK;
            });
            if (rc == LBM_OK) rc = check(b);
            if (rc != LBM_OK) return rc;
        }
    }
    return LBM_OK;
}

extern "C" int lbm_batch_step(lbm_batch* b, int64_t n) {
    return lbm_batch_step_with(b, n, LBM_BATCH_GRAPH);
}

extern "C" int lbm_batch_status(const lbm_batch* b, int* state, int64_t* steps, double* residual) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch%s");
    for (int m = 0; m < b->count; ++m) {
        if (state) state[m] = b->state[m];
        if (steps) steps[m] = b->members[m]->steps;
        if (residual) residual[m] = b->members[m]->last_residual;
    }
    return LBM_OK;
}

extern "C" int lbm_batch_member(lbm_batch* b, int index, lbm_ctx** member) {
    if (!b || !member || index < 0 || index >= b->count)
        return bfail(b, LBM_EINVAL, "member index out of range%s");
    *member = b->members[index];
    return LBM_OK;
}

extern "C" int lbm_batch_count(const lbm_batch* b) { return b ? b->count : 0; }

extern "C" int64_t lbm_batch_steps_done(const lbm_batch* b) { return b ? b->steps : -1; }

extern "C" int64_t lbm_batch_active_nodes(const lbm_batch* b) {
    if (!b) return 0;
    int64_t n = 0;
    for (int m = 0; m < b->count; ++m)
        if (b->state[m] == LBM_MEMBER_ACTIVE) n += b->members[m]->ncell;
    return n;
}

extern "C" int lbm_batch_autotune(lbm_batch* b, int trial_steps, lbm_batch_trial* trials,
                                  int max_trials, int* n_trials) {
    if (!b || trial_steps < 1) return bfail(b, LBM_EINVAL, "invalid batch or trial_steps%s");
    DeviceGuard g(b->device);
    if (n_trials) *n_trials = 0;
    if (n_active(b) == 0) return LBM_OK;
    Variant vs[kMaxVariants];
    const int nv = batch_variants(b, vs);
    int cache_all = 0;
    const size_t smem = smem_for(b, 1, &cache_all);
    std::vector<lbm_batch_trial> res;
    for (int v = 0; v < nv; ++v) {
        int occ = 0;
        BATCH_CUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, vs[v].fn, vs[v].threads, smem));
        if (occ < 1) continue;
        for (int mapping : {LBM_TILE_LINEAR, LBM_TILE_ROWS})
            for (int factor : {1, 2, 4})
                for (int bps : {occ, 0})
                    res.push_back(lbm_batch_trial{{vs[v].threads, vs[v].min_blocks, mapping, bps, factor}, 0.0});
    }
    cudaEvent_t e0, e1;
    BATCH_CUDA(b, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return bfail(b, LBM_ECUDA, "cudaEventCreate failed%s");
    }
    const int parity = (int)(b->steps & 1);  // read the current state, write the other buffer
    int rc = LBM_OK;
    for (auto& t : res) {
        rc = apply_tiling(b, t.tiling);
        if (rc != LBM_OK) break;
        // every trial launch has the same parity: its queue counter is zeroed before it
        rc = with_real(b, [&](auto tag) {
            using S = decltype(tag);
            BATCH_CUDA(b, cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(int), b->stream));
            BATCH_CUDA(b, launch_batch_step<S>(b, parity, b->stream));
            BATCH_CUDA(b, cudaEventRecord(e0, b->stream));
            for (int s = 0; s < trial_steps; ++s) {
                BATCH_CUDA(b, cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(int), b->stream));
                BATCH_CUDA(b, launch_batch_step<S>(b, parity, b->stream));
            }
            BATCH_CUDA(b, cudaEventRecord(e1, b->stream));
            BATCH_CUDA(b, cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(int), b->stream));
            return LBM_OK;
        });
        if (rc == LBM_OK) rc = bwait(b);
        if (rc != LBM_OK) break;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = bfail(b, LBM_ECUDA, "cudaEventElapsedTime failed%s");
            break;
        }
        t.ms_per_step = ms / trial_steps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LBM_OK) return rc;
    size_t best = 0;
    for (size_t i = 1; i < res.size(); ++i)
        if (res[i].ms_per_step < res[best].ms_per_step) best = i;
    rc = apply_tiling(b, res[best].tiling);
    if (rc != LBM_OK) return rc;
    if (trials)
        for (int i = 0; i < (int)res.size() && i < max_trials; ++i) trials[i] = res[i];
    if (n_trials) *n_trials = (int)res.size();
    return LBM_OK;
}

extern "C" int lbm_batch_get_tiling(const lbm_batch* b, lbm_batch_tiling* out) {
    if (!b || !out) return bfail(nullptr, LBM_EINVAL, "NULL argument%s");
    *out = b->tiling;
    return LBM_OK;
}

extern "C" int lbm_batch_set_tiling(lbm_batch* b, const lbm_batch_tiling* t) {
    if (!b || !t) return bfail(b, LBM_EINVAL, "NULL argument%s");
    DeviceGuard g(b->device);
    return apply_tiling(b, *t);
}

extern "C" int lbm_batch_synchronize(lbm_batch* b) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "NULL batch%s");
    DeviceGuard g(b->device);
    return bwait(b);
}

extern "C" const char* lbm_batch_last_error(const lbm_batch* b) {
    return b ? b->err.c_str() : lbm_last_error(nullptr);
}
