// slabs.cu -- one cavity split into z-slabs with a halo exchange (include/lbm_slabs.h).
//
// Every slab is an ordinary context on its owned planes plus halo planes, so each slab
// step is the same kernel launch lbm_step makes (the method of arXiv:1710.04751: Eqs. 2b,
// 13b streaming, Appendix A / Sec. 2.2 / Appendix C collisions, Sec. 3 walls).  After the
// steps of all slabs one copy kernel moves every cut plane of the new state into the
// neighbours' halo planes: a table of (source, destination, length) entries built once
// per buffer parity.  The slab kernels of one step run concurrently, each on a stream of
// its own forked from the decomposition's stream and joined before the exchange, so
// together they fill the GPU as one kernel over the whole grid would.
#include <new>
#include <vector>

#include "context.h"
#include "lattice.cuh"
#include "lbm_slabs.h"

using namespace lbm;

namespace lbm {
// one copy of an exchange: `bytes` bytes, a multiple of 2 (stored elements are 2, 4 or 8
// bytes wide)
struct HaloCopy {
    const void* src;
    void* dst;
    int64_t bytes;
};
}  // namespace lbm

namespace {

template <typename W>
__device__ __forceinline__ void copy_words(const void* src, void* dst, int64_t n) {
    const W* s = static_cast<const W*>(src);
    W* d = static_cast<W*>(dst);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) d[i] = s[i];
}

// One block row per table entry; the widest word that source, destination and length
// all allow (16 bytes for whole planes of most grids).
__global__ void halo_copy_kernel(const HaloCopy* __restrict__ table) {
    const HaloCopy h = table[blockIdx.y];
    const uintptr_t a = (uintptr_t)h.src | (uintptr_t)h.dst | (uintptr_t)h.bytes;
    if ((a & 15) == 0) copy_words<uint4>(h.src, h.dst, h.bytes / 16);
    else if ((a & 3) == 0) copy_words<uint32_t>(h.src, h.dst, h.bytes / 4);
    else copy_words<uint16_t>(h.src, h.dst, h.bytes / 2);
}

}  // namespace

struct lbm_slabs {
    lbm_grid grid;
    int Q = 0, precision = 0, nslabs = 0;
    lbm_options opt;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::vector<lbm_ctx*> m;
    std::vector<int> z0, own, hlo, hhi;
    int cur = 0;
    int64_t steps = 0;
    double last_residual = -1.0;
    HaloCopy* table = nullptr;  // device: 2 * entries, one list per new-state buffer
    int entries = 0;
    int64_t max_bytes = 0;
    int64_t halo_bytes = 0;
    std::vector<cudaStream_t> side;  // slabs 1.. run on these, forked from and joined to `stream`
    std::vector<cudaEvent_t> ev;     // ev[0] the fork, ev[k] slab k's join
    cudaStream_t capture = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool graphs_failed = false;
    std::string err;
};

namespace {

int sfail(lbm_slabs* s, int code, const char* fmt, const char* detail = nullptr) {
    return record_error(s ? &s->err : nullptr, code, fmt, detail);
}

#define SLABS_CUDA(s, call)                                                          \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return sfail((s), LBM_ECUDA, "CUDA error in " #call ": %s",              \
                         cudaGetErrorString(e_));                                    \
    } while (0)

void free_slabs(lbm_slabs* s) {
    if (!s) return;
    DeviceGuard g(s->device);
    for (int b = 0; b < 2; ++b)
        if (s->graph[b]) cudaGraphExecDestroy(s->graph[b]);
    if (s->capture) cudaStreamDestroy(s->capture);
    for (cudaStream_t t : s->side) cudaStreamDestroy(t);
    for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
    if (s->table) cudaFree(s->table);
    for (lbm_ctx* c : s->m)
        if (c) destroy_context(c);
    delete s;
}

// The copies of one exchange into the buffers `nb` (the new state): for every slab, its
// first owned plane to the halo above the slab below it, its last owned plane to the
// halo below the slab above it (neighbours wrap around when z is periodic).
std::vector<HaloCopy> exchange_list(const lbm_slabs* s, int nb) {
    std::vector<HaloCopy> out;
    const int S = s->nslabs;
    const int64_t nxy = (int64_t)s->grid.nx * s->grid.ny;
    const bool dev16 = s->precision == LBM_FP16_DEV || s->precision == LBM_BF16_DEV;
    const size_t rs = s->m[0]->rsize;
    auto add_plane = [&](const lbm_ctx* src, int zs, const lbm_ctx* dst, int zd) {
        const int64_t bytes = nxy * (int64_t)rs;
        for (int side = 0; side < 2; ++side) {
            const int q = side == 0 ? 15 : s->Q;
            const char* sb = static_cast<const char*>(side == 0 ? src->dev.F[nb] : src->dev.G[nb]);
            char* db = static_cast<char*>(side == 0 ? dst->dev.F[nb] : dst->dev.G[nb]);
            for (int a = 0; a < q; ++a) {
                const int64_t so = ((int64_t)a * src->plane + zs * nxy) * (int64_t)rs;
                const int64_t dof = ((int64_t)a * dst->plane + zd * nxy) * (int64_t)rs;
                out.push_back({sb + so, db + dof, bytes});
            }
        }
        if (dev16) {  // the FP32 node temperatures the thermal deviations refer to
            const char* sb = static_cast<const char*>(src->dev.T[nb]);
            char* db = static_cast<char*>(dst->dev.T[nb]);
            out.push_back({sb + zs * nxy * 4, db + zd * nxy * 4, nxy * 4});
        }
    };
    for (int k = 0; k < S; ++k) {
        const lbm_ctx* c = s->m[k];
        if (s->hlo[k]) {  // halo below slab k <- last owned plane of the slab below
            const int b = (k + S - 1) % S;
            add_plane(s->m[b], s->hlo[b] + s->own[b] - 1, c, 0);
        }
        if (s->hhi[k]) {  // halo above slab k <- first owned plane of the slab above
            const int a = (k + 1) % S;
            add_plane(s->m[a], s->hlo[a], c, s->hlo[k] + s->own[k]);
        }
    }
    return out;
}

int launch_exchange(lbm_slabs* s, int nb, cudaStream_t st) {
    if (s->entries == 0) return LBM_OK;
    const int threads = 256;
    const int64_t want = (s->max_bytes / 16 + threads - 1) / threads;
    const dim3 grid((unsigned)(want < 1 ? 1 : want < 64 ? want : 64), (unsigned)s->entries);
    halo_copy_kernel<<<grid, threads, 0, st>>>(s->table + (size_t)nb * s->entries);
    SLABS_CUDA(s, cudaGetLastError());
    return LBM_OK;
}

// One step of every slab from buffer `cur`, the exchange into cur ^ 1 and, when the step
// count after it reaches a multiple of the residual interval, each slab's residual check.
template <typename S>
int enqueue_slab_step(lbm_slabs* s, const std::vector<ParamsOf<S>>& p, int cur, int64_t steps_after,
                      cudaStream_t st) {
    const int S_ = s->nslabs;
    if (S_ > 1) {  // fork: slab k >= 1 on side[k - 1]
        SLABS_CUDA(s, cudaEventRecord(s->ev[0], st));
        for (int k = 1; k < S_; ++k) SLABS_CUDA(s, cudaStreamWaitEvent(s->side[k - 1], s->ev[0], 0));
    }
    for (int k = 0; k < S_; ++k)
        SLABS_CUDA(s, launch_step<S>(s->m[k]->dev, cur, p[k], k == 0 ? st : s->side[k - 1]));
    for (int k = 1; k < S_; ++k) {  // join before the exchange reads the new planes
        SLABS_CUDA(s, cudaEventRecord(s->ev[k], s->side[k - 1]));
        SLABS_CUDA(s, cudaStreamWaitEvent(st, s->ev[k], 0));
    }
    int rc = launch_exchange(s, cur ^ 1, st);
    if (rc != LBM_OK) return rc;
    const int R = s->opt.residual_interval;
    if (R > 0 && steps_after % R == 0) {
        for (int k = 0; k < s->nslabs; ++k) {
            SLABS_CUDA(s, cudaMemsetAsync(s->m[k]->dev.resid_bits, 0, sizeof(unsigned long long), st));
            SLABS_CUDA(s, launch_residual<S>(s->m[k]->dev, cur ^ 1, p[k], 1, st));
        }
    }
    return LBM_OK;
}

#ifndef LBM_SLAB_GRAPHS
#define LBM_SLAB_GRAPHS 1
#endif
// residual_interval steps from buffer `cur` as one graph (captured on first use; NULL
// when capture is not possible, and then never tried again)
template <typename S>
cudaGraphExec_t slab_graph(lbm_slabs* s, const std::vector<ParamsOf<S>>& p, int cur) {
    if (!LBM_SLAB_GRAPHS || s->graphs_failed) return nullptr;
    if (s->graph[cur]) return s->graph[cur];
    const int R = s->opt.residual_interval;
    bool ok = s->capture || cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking) == cudaSuccess;
    cudaGraph_t g = nullptr;
    if (ok) ok = cudaStreamBeginCapture(s->capture, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        int b = cur, rc = LBM_OK;
        for (int i = 1; i <= R && rc == LBM_OK; ++i, b ^= 1) rc = enqueue_slab_step<S>(s, p, b, i, s->capture);
        const cudaError_t e2 = cudaStreamEndCapture(s->capture, &g);
        ok = rc == LBM_OK && e2 == cudaSuccess && g;
    }
    if (ok) ok = cudaGraphInstantiate(&s->graph[cur], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        s->graph[cur] = nullptr;
        s->graphs_failed = true;
        cudaGetLastError();
        s->err.clear();
    }
    return s->graph[cur];
}

template <typename S>
int run_slab_steps_(lbm_slabs* s, int64_t n, bool* checked) {
    std::vector<ParamsOf<S>> p;
    for (lbm_ctx* c : s->m) p.push_back(dev_params<typename Storage<S>::real>(c));
    const int R = s->opt.residual_interval;
    for (int64_t done = 0; done < n;) {
        if (R > 0 && s->steps % R == 0 && n - done >= R) {
            if (cudaGraphExec_t g = slab_graph<S>(s, p, s->cur)) {
                SLABS_CUDA(s, cudaGraphLaunch(g, s->stream));
                if (R & 1) s->cur ^= 1;
                s->steps += R;
                done += R;
                *checked = true;
                continue;
            }
        }
        const int rc = enqueue_slab_step<S>(s, p, s->cur, s->steps + 1, s->stream);
        if (rc != LBM_OK) return rc;
        s->cur ^= 1;
        s->steps += 1;
        done += 1;
        if (R > 0 && s->steps % R == 0) *checked = true;
    }
    return LBM_OK;
}

template <typename S>
int run_slab_steps(lbm_slabs* s, int64_t n, bool* checked) {
    const int rc = run_slab_steps_<S>(s, n, checked);
    for (lbm_ctx* c : s->m) {  // the members' own view (their transfers read buffer cur)
        c->cur = s->cur;
        c->steps = s->steps;
    }
    return rc;
}

// global plane of slab k's local plane z (wrapping when z is periodic)
int global_plane(const lbm_slabs* s, int k, int z) {
    const int nz = s->grid.nz;
    return ((s->z0[k] - s->hlo[k] + z) % nz + nz) % nz;
}

}  // namespace

extern "C" int lbm_slabs_plan(int nz, int nslabs, int boundary, const int* owned, int* z0,
                              int* nz_owned, int* halo_lo, int* halo_hi) {
    if (nz < 1 || nslabs < 1 || nslabs > nz)
        return sfail(nullptr, LBM_EINVAL, "need 1 <= nslabs <= nz%s");
    int64_t sum = 0;
    if (owned) {
        for (int k = 0; k < nslabs; ++k) {
            if (owned[k] < 1) return sfail(nullptr, LBM_EINVAL, "every slab needs >= 1 owned plane%s");
            sum += owned[k];
        }
        if (sum != nz) return sfail(nullptr, LBM_EINVAL, "the owned planes must sum to nz%s");
    }
    const bool zper = (boundary & 4) != 0;
    int start = 0;
    for (int k = 0; k < nslabs; ++k) {
        const int o = owned ? owned[k] : nz / nslabs + (k < nz % nslabs ? 1 : 0);
        if (z0) z0[k] = start;
        if (nz_owned) nz_owned[k] = o;
        if (halo_lo) halo_lo[k] = nslabs > 1 && (zper || k > 0) ? 1 : 0;
        if (halo_hi) halo_hi[k] = nslabs > 1 && (zper || k < nslabs - 1) ? 1 : 0;
        start += o;
    }
    return LBM_OK;
}

extern "C" int lbm_slabs_create(const lbm_grid* grid, int lattice, const lbm_params* params,
                                const lbm_options* opt, int nslabs, const int* owned,
                                lbm_slabs** out) {
    NvtxRange nvtx("lbm_slabs_create");
    if (!out) return sfail(nullptr, LBM_EINVAL, "out is NULL%s");
    *out = nullptr;
    if (!grid || grid->nx < 1 || grid->ny < 1 || grid->nz < 1)
        return sfail(nullptr, LBM_EINVAL, "invalid grid%s");
    if (!params) return sfail(nullptr, LBM_EINVAL, "params is NULL%s");
    lbm_options o;
    if (opt) o = *opt; else lbm_default_options(&o);
    if (o.device_arena) return sfail(nullptr, LBM_EINVAL, "slabs allocate their own device memory%s");
    lbm_slabs* s = new (std::nothrow) lbm_slabs();
    if (!s) return sfail(nullptr, LBM_ENOMEM, "host allocation failed%s");
    s->grid = *grid;
    s->Q = lattice;
    s->precision = o.precision;
    s->nslabs = nslabs;
    s->opt = o;
    s->stream = (cudaStream_t)o.cuda_stream;
    if (nslabs >= 1) {
        s->z0.resize(nslabs); s->own.resize(nslabs); s->hlo.resize(nslabs); s->hhi.resize(nslabs);
    }
    int rc = lbm_slabs_plan(grid->nz, nslabs, params->boundary, owned, s->z0.data(), s->own.data(),
                            s->hlo.data(), s->hhi.data());
    if (rc != LBM_OK) {
        delete s;
        return rc;
    }
    cudaGetDevice(&s->device);
    const int64_t nxy = (int64_t)grid->nx * grid->ny;
    for (int k = 0; k < nslabs; ++k) {
        const lbm_grid g = {grid->nx, grid->ny, s->hlo[k] + s->own[k] + s->hhi[k]};
        lbm_ctx* c = nullptr;
        // the slab's local plane 0 is global plane z0 - halo_lo (wrapped): its noise is
        // drawn for the global cell indices, so the halo planes start as their owners do
        const int64_t cell0 = (int64_t)global_plane(s, k, 0) * nxy;
        rc = create_context(&g, lattice, params, &o, cell0, &c);
        if (rc != LBM_OK) {
            free_slabs(s);
            return rc;  // the member's message stays in lbm_slabs_last_error(NULL)
        }
        s->m.push_back(c);
    }
    // the streams and events of the fork / join (none for a single slab)
    for (int k = 0; k < nslabs && nslabs > 1; ++k) {
        cudaEvent_t e = nullptr;
        cudaStream_t t = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess ||
            (k > 0 && cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess)) {
            if (e) cudaEventDestroy(e);
            free_slabs(s);
            return sfail(nullptr, LBM_ECUDA, "stream or event creation failed%s");
        }
        s->ev.push_back(e);
        if (k > 0) s->side.push_back(t);
    }
    // exchange tables for both parities
    std::vector<HaloCopy> lists[2] = {exchange_list(s, 0), exchange_list(s, 1)};
    s->entries = (int)lists[0].size();
    for (const HaloCopy& h : lists[0]) {
        s->max_bytes = h.bytes > s->max_bytes ? h.bytes : s->max_bytes;
        s->halo_bytes += h.bytes;
    }
    if (s->entries > 65535) {
        free_slabs(s);
        return sfail(nullptr, LBM_EINVAL, "too many slabs for one exchange launch%s");
    }
    if (s->entries) {
        const size_t bytes = 2 * (size_t)s->entries * sizeof(HaloCopy);
        if (cudaMalloc(&s->table, bytes) != cudaSuccess) {
            free_slabs(s);
            return sfail(nullptr, LBM_ENOMEM, "cudaMalloc of the exchange table failed%s");
        }
        std::vector<HaloCopy> both(lists[0]);
        both.insert(both.end(), lists[1].begin(), lists[1].end());
        cudaError_t e = cudaMemcpy(s->table, both.data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_slabs(s);
            return sfail(nullptr, LBM_ECUDA, "copy of the exchange table failed: %s", cudaGetErrorString(e));
        }
    }
    *out = s;
    return LBM_OK;
}

extern "C" int lbm_slabs_step(lbm_slabs* s, int64_t n) {
    NvtxRange nvtx("lbm_slabs_step");
    if (!s || n < 0) return sfail(s, LBM_EINVAL, "invalid decomposition or step count%s");
    DeviceGuard g(s->device);
    bool checked = false;
    int rc = with_storage(s->precision, [&](auto tag) { return run_slab_steps<decltype(tag)>(s, n, &checked); });
    if (rc != LBM_OK || !checked) return rc;
    for (lbm_ctx* c : s->m) {
        SLABS_CUDA(s, cudaMemcpyAsync(c->host_bits, c->dev.resid_bits, sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, s->stream));
        SLABS_CUDA(s, cudaMemcpyAsync(c->host_bits + 1, c->dev.nonfinite, sizeof(int),
                                      cudaMemcpyDeviceToHost, s->stream));
    }
    rc = wait_stream_for(s->stream, s->opt.timeout_s, &s->err);
    if (rc != LBM_OK) return rc;
    double worst = 0.0;
    bool bad = false;
    for (lbm_ctx* c : s->m) {
        double r;
        memcpy(&r, &c->host_bits[0], sizeof r);
        c->last_residual = r;
        worst = r > worst ? r : worst;
        bad = bad || *reinterpret_cast<int*>(c->host_bits + 1) != 0;
    }
    s->last_residual = worst;
    if (bad) return sfail(s, LBM_EDIVERGED, "non-finite temperature detected%s");
    return LBM_OK;
}

extern "C" int lbm_slabs_residual(lbm_slabs* s, double* max_dT) {
    if (!s || !max_dT) return sfail(s, LBM_EINVAL, "NULL argument%s");
    *max_dT = s->last_residual;
    return LBM_OK;
}

// Populations: each member's owned planes straight to (or, halo planes included, from)
// the whole-grid arrays through its FP64 transfer of a cell range.  An upload takes the
// slab's planes in runs of consecutive global planes (a halo across a periodic z face
// starts a new run).
static int slab_transfer(lbm_slabs* s, double* f, double* g, const double* fin, const double* gin) {
    const int64_t nxy = (int64_t)s->grid.nx * s->grid.ny;
    const int64_t N = nxy * s->grid.nz;
    for (int k = 0; k < s->nslabs; ++k) {
        lbm_ctx* c = s->m[k];
        int rc = LBM_OK;
        if (fin) {
            const int nzb = c->grid.nz;
            for (int z = 0; z < nzb && rc == LBM_OK;) {
                const int zg = global_plane(s, k, z);
                int len = 1;
                while (z + len < nzb && global_plane(s, k, z + len) == zg + len) ++len;
                rc = transfer_cells(c, nullptr, nullptr, fin + zg * nxy, gin + zg * nxy, z * nxy,
                                    len * nxy, N);
                z += len;
            }
        } else {
            rc = transfer_cells(c, f + (int64_t)s->z0[k] * nxy, g + (int64_t)s->z0[k] * nxy, nullptr,
                                nullptr, (int64_t)s->hlo[k] * nxy, (int64_t)s->own[k] * nxy, N);
        }
        if (rc == LBM_OK) rc = transfer_done(c, fin != nullptr);
        if (rc != LBM_OK) return sfail(s, rc, "slab transfer failed: %s", c->err.c_str());
    }
    if (fin) s->last_residual = -1.0;
    return LBM_OK;
}

extern "C" int lbm_slabs_get_populations(lbm_slabs* s, double* f, double* g) {
    NvtxRange nvtx("lbm_slabs_get_populations");
    if (!s || !f || !g) return sfail(s, LBM_EINVAL, "NULL argument%s");
    DeviceGuard gd(s->device);
    return slab_transfer(s, f, g, nullptr, nullptr);
}

extern "C" int lbm_slabs_set_populations(lbm_slabs* s, const double* f, const double* g) {
    NvtxRange nvtx("lbm_slabs_set_populations");
    if (!s || !f || !g) return sfail(s, LBM_EINVAL, "NULL argument%s");
    DeviceGuard gd(s->device);
    return slab_transfer(s, nullptr, nullptr, f, g);
}

extern "C" int lbm_slabs_fields(lbm_slabs* s, double* rho, double* ux, double* uy, double* uz,
                                double* T) {
    NvtxRange nvtx("lbm_slabs_fields");
    if (!s) return sfail(s, LBM_EINVAL, "NULL decomposition%s");
    DeviceGuard gd(s->device);
    const int64_t nxy = (int64_t)s->grid.nx * s->grid.ny;
    double* outs[5] = {rho, ux, uy, uz, T};
    for (int k = 0; k < s->nslabs; ++k) {
        lbm_ctx* c = s->m[k];
        double* mine[5];
        for (int i = 0; i < 5; ++i) mine[i] = outs[i] ? outs[i] + (int64_t)s->z0[k] * nxy : nullptr;
        const int rc = fields_cells(c, mine, (int64_t)s->hlo[k] * nxy, (int64_t)s->own[k] * nxy);
        if (rc != LBM_OK) return sfail(s, rc, "slab fields failed: %s", c->err.c_str());
    }
    return LBM_OK;
}

extern "C" int lbm_slabs_count(const lbm_slabs* s) { return s ? s->nslabs : -1; }
extern "C" int64_t lbm_slabs_steps_done(const lbm_slabs* s) { return s ? s->steps : -1; }
extern "C" int64_t lbm_slabs_halo_bytes(const lbm_slabs* s) { return s ? s->halo_bytes : -1; }

extern "C" int lbm_slabs_synchronize(lbm_slabs* s) {
    if (!s) return sfail(s, LBM_EINVAL, "NULL decomposition%s");
    DeviceGuard gd(s->device);
    return wait_stream_for(s->stream, s->opt.timeout_s, &s->err);
}

extern "C" const char* lbm_slabs_last_error(const lbm_slabs* s) {
    return s ? s->err.c_str() : lbm_last_error(nullptr);
}

extern "C" void lbm_slabs_destroy(lbm_slabs* s) { free_slabs(s); }

// ---------------------------------------------------------------------------------
// The message of one cut for a decomposition over several processes (host only).
// ---------------------------------------------------------------------------------
namespace {
// Populations whose e_z is `dir` (+1 or -1), in the paper's direction order.
int cut_ids(int lattice, int dir, int* flow, int* scalar, int* nscalar) {
    int nf = 0, ns = 0;
    for (int a = 0; a < 15; ++a) {
        if (ez(a) != dir) continue;
        flow[nf++] = a;
        if (a < lattice) scalar[ns++] = a;
    }
    *nscalar = ns;
    return nf;
}

int check_cut(const lbm_grid* g, int lattice, int plane, int dir) {
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1) return sfail(nullptr, LBM_EINVAL, "invalid slab grid%s");
    if (lattice != LBM_THERMAL_D3Q15 && lattice != LBM_THERMAL_D3Q7)
        return sfail(nullptr, LBM_EINVAL, "lattice must be 15 or 7%s");
    if (dir != 1 && dir != -1) return sfail(nullptr, LBM_EINVAL, "direction must be +1 or -1%s");
    if (plane < 0 || plane >= g->nz) return sfail(nullptr, LBM_EINVAL, "plane outside the slab%s");
    return LBM_OK;
}

template <bool PACK>
int move_cut(const lbm_grid* g, int lattice, int plane, int dir, double* f, double* gp, double* msg) {
    int rc = check_cut(g, lattice, plane, dir);
    if (rc != LBM_OK) return rc;
    if (!f || !gp || !msg) return sfail(nullptr, LBM_EINVAL, "NULL array%s");
    int flow[15], scalar[15], ns = 0;
    const int nf = cut_ids(lattice, dir, flow, scalar, &ns);
    const int64_t nxy = (int64_t)g->nx * g->ny, ncell = nxy * g->nz, off = (int64_t)plane * nxy;
    double* m = msg;
    for (int side = 0; side < 2; ++side) {
        double* p = side == 0 ? f : gp;
        const int* ids = side == 0 ? flow : scalar;
        for (int n = 0, cnt = side == 0 ? nf : ns; n < cnt; ++n, m += nxy) {
            double* row = p + ids[n] * ncell + off;
            for (int64_t c = 0; c < nxy; ++c) {
                if (PACK) m[c] = row[c];
                else row[c] = m[c];
            }
        }
    }
    return LBM_OK;
}
}  // namespace

extern "C" int lbm_slabs_cut_populations(int lattice, int dir, int* flow_ids, int* n_flow,
                                         int* scalar_ids, int* n_scalar) {
    if ((lattice != LBM_THERMAL_D3Q15 && lattice != LBM_THERMAL_D3Q7) || (dir != 1 && dir != -1))
        return sfail(nullptr, LBM_EINVAL, "lattice must be 15 or 7 and direction +1 or -1%s");
    int flow[15], scalar[15], ns = 0;
    const int nf = cut_ids(lattice, dir, flow, scalar, &ns);
    for (int n = 0; n < nf && flow_ids; ++n) flow_ids[n] = flow[n];
    for (int n = 0; n < ns && scalar_ids; ++n) scalar_ids[n] = scalar[n];
    if (n_flow) *n_flow = nf;
    if (n_scalar) *n_scalar = ns;
    return LBM_OK;
}

extern "C" int64_t lbm_slabs_cut_values(int nx, int ny, int lattice) {
    if (nx < 1 || ny < 1 || (lattice != LBM_THERMAL_D3Q15 && lattice != LBM_THERMAL_D3Q7)) return 0;
    return (int64_t)(5 + (lattice == LBM_THERMAL_D3Q15 ? 5 : 1)) * nx * ny;
}

extern "C" int lbm_slabs_pack_cut(const lbm_grid* slab_grid, int lattice, int plane, int dir,
                                  const double* f, const double* g, double* msg) {
    return move_cut<true>(slab_grid, lattice, plane, dir, const_cast<double*>(f),
                          const_cast<double*>(g), msg);
}

extern "C" int lbm_slabs_unpack_cut(const lbm_grid* slab_grid, int lattice, int plane, int dir,
                                    const double* msg, double* f, double* g) {
    return move_cut<false>(slab_grid, lattice, plane, dir, f, g, const_cast<double*>(msg));
}

