// api.cu -- the C ABI declared in include/lbm.h: context life cycle, parameter
// derivation (Sec. 3 of arXiv:1710.04751), the time-step loop and host transfers.
#include <math.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <new>
#include <string>
#include <thread>

#include "context.h"

using namespace lbm;

static thread_local std::string g_err;

void lbm::set_last_error(const char* msg) { g_err = msg; }

int lbm::record_error(std::string* slot, int code, const char* fmt, const char* detail) {
    char buf[512];
    snprintf(buf, sizeof buf, fmt, detail ? detail : "");
    if (slot) *slot = buf;
    g_err = buf;
    return code;
}

extern "C" void lbm_default_options(lbm_options* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = LBM_FP32;
    o->seed = 1;
    o->noise_amp = 1e-6;
    o->cs2_phi = 0.0;  // lattice default: 1/3 (D3Q15), 1/4 (D3Q7)
    o->e4_mode = 0;
    o->adiabatic_mode = LBM_ADIABATIC_SPECULAR;
    o->residual_interval = 100;
    o->cuda_stream = nullptr;
    o->device_arena = nullptr;
    o->device_arena_bytes = 0;
    o->timeout_s = 600.0;
}

static bool valid_grid(const lbm_grid* g) {
    return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 &&
           (double)g->nx * g->ny * g->nz < 4.0e9;
}

static bool valid_lattice(int q) { return q == LBM_THERMAL_D3Q15 || q == LBM_THERMAL_D3Q7; }

extern "C" int lbm_derive_params(const lbm_grid* grid, int lattice, double Ra, double Pr,
                                 double Ma, const lbm_options* opt, lbm_params* out) {
    lbm_options o;
    if (opt) o = *opt; else lbm_default_options(&o);
    if (!out || !valid_grid(grid)) return fail(nullptr, LBM_EINVAL, "invalid grid%s");
    if (!valid_lattice(lattice)) return fail(nullptr, LBM_EINVAL, "lattice must be 15 or 7%s");
    if (!(Ra > 0) || !(Pr > 0) || !(Ma > 0))
        return fail(nullptr, LBM_EINVAL, "Ra, Pr and Ma must be positive%s");
    // Sec. 3: Ra = g beta dT L^3 / (alpha nu), Pr = nu / alpha, U0 = sqrt(g beta dT L)
    const double L = grid->nx, dT = 1.0;
    const double U0 = Ma * sqrt(1.0 / 3.0);
    if (U0 >= 0.3) return fail(nullptr, LBM_EINVAL, "Ma * c_s must stay below 0.3%s");
    const double gbeta = U0 * U0 / (dT * L);
    const double nu = sqrt(Pr / Ra) * U0 * L;
    const double alpha = nu / Pr;
    // c_sphi^2: "typically 1/3" (Sec. 2.2).  On D3Q7 that value gives a negative rest
    // equilibrium phi (1 - 3 c_sphi^2 - u^2) for any u != 0, so D3Q7 defaults to 1/4.
    const double cs2p = o.cs2_phi > 0 ? o.cs2_phi : (lattice == 15 ? 1.0 / 3.0 : 0.25);
    if (!(cs2p > 0 && cs2p <= (lattice == 15 ? 0.5 : 1.0 / 3.0)))
        return fail(nullptr, LBM_EINVAL, "cs2_phi outside the range with non-negative rest weights%s");
    const double om_nu = 1.0 / (3.0 * nu + 0.5);       // nu = c_s^2 (1/omega - 1/2), App. A
    const double om_phi = 1.0 / (alpha / cs2p + 0.5);  // D = c_sphi^2 (1/omega - 1/2), Eq. 23
    if (!(om_nu > 0 && om_nu < 2) || !(om_phi > 0 && om_phi < 2))
        return fail(nullptr, LBM_EINVAL, "relaxation rate outside (0, 2)%s");
    memset(out, 0, sizeof *out);
    // App. A: "nu = c_s^2 (1/omega_j - 1/2), j = 5, ..., 9" counts the moments from 1:
    // the five shear moments g^_4..g^_8.  The bulk moment g^_9 and the rest relax at 1
    // ("set to unity"); relaxing g^_9 at omega_nu as well makes the 91^3, Ra = 1e5
    // cavity of Sec. 3 diverge.
    for (int b = 0; b < 15; ++b) {
        out->omega_f[b] = (b >= 4 && b <= 8) ? om_nu : 1.0;
        out->omega_g[b] = (b >= 1 && b <= 3) ? om_phi : 1.0;
    }
    out->gbeta = gbeta;
    out->T_hot = 0.5 * dT;
    out->T_cold = -0.5 * dT;
    out->cs2_phi = cs2p;
    out->U0 = U0;
    out->e4_mode = o.e4_mode;
    out->adiabatic_mode = o.adiabatic_mode;
    out->boundary = LBM_BC_CAVITY;
    return LBM_OK;
}

static int64_t plane_of(int64_t ncell) { return (ncell + 63) / 64 * 64; }

struct Layout {
    size_t F[2], G[2], T[2], snap, staging, partials, result, bits, total;
};

// bytes of one stored population and of the arithmetic type, by precision
static size_t storage_bytes(int precision) {
    return precision == LBM_FP64 ? 8 : precision == LBM_FP32 ? 4 : 2;
}
static size_t compute_bytes(int precision) { return precision == LBM_FP64 ? 8 : 4; }

static bool valid_precision(int p) {
    return p == LBM_FP64 || p == LBM_FP32 || p == LBM_FP16_DEV || p == LBM_BF16_DEV;
}

static Layout layout_of(const lbm_grid* g, int q, int precision) {
    const int64_t ncell = (int64_t)g->nx * g->ny * g->nz;
    const int64_t plane = plane_of(ncell);
    const size_t rs = storage_bytes(precision);
    Layout L;
    size_t off = 0;
    for (int b = 0; b < 2; ++b) { L.F[b] = off; off = align_up(off + 15 * plane * rs, 256); }
    for (int b = 0; b < 2; ++b) { L.G[b] = off; off = align_up(off + q * plane * rs, 256); }
    // 16-bit forms: FP32 node temperatures the stored thermal deviations refer to
    const bool dev = precision == LBM_FP16_DEV || precision == LBM_BF16_DEV;
    for (int b = 0; b < 2; ++b) { L.T[b] = off; off = align_up(off + (dev ? plane * 4 : 0), 256); }
    L.snap = off; off = align_up(off + plane * compute_bytes(precision), 256);
    L.staging = off; off = align_up(off + plane * 8, 256);
    L.partials = off; off = align_up(off + 2 * kPartialBlocks * 8, 256);
    L.result = off; off = align_up(off + kResultDoubles * 8, 256);
    L.bits = off; off = align_up(off + 256, 256);
    L.total = off;
    return L;
}

extern "C" size_t lbm_arena_bytes(const lbm_grid* grid, int lattice, int precision) {
    if (!valid_grid(grid) || !valid_lattice(lattice) || !valid_precision(precision)) return 0;
    return layout_of(grid, lattice, precision).total;
}

size_t lbm::context_arena_bytes(const lbm_grid* g, int q, int precision) {
    return layout_of(g, q, precision).total;
}

template <typename real>
DevParams<real> lbm::dev_params(const lbm_ctx* c) {
    DevParams<real> p;
    memset(&p, 0, sizeof p);
    const lbm_params& P = c->params;
    for (int b = 0; b < 15; ++b) {
        p.om_f[b] = (real)P.omega_f[b];
        p.om_g[b] = (real)P.omega_g[b];
    }
    const double cs = P.cs2_phi;
    double w0, w1, w7;
    if (c->Q == 15) {
        w7 = cs * cs / 8.0;
        w1 = 0.5 * (cs - cs * cs);
        w0 = 1.0 - 6.0 * w1 - 8.0 * w7;
    } else {
        w7 = 0.0;
        w1 = 0.5 * cs;
        w0 = 1.0 - 6.0 * w1;
    }
    const double cs2 = 1.0 / 3.0;
    const double f7 = cs2 * cs2 / 8.0, f1 = 0.5 * (cs2 - cs2 * cs2), f0 = 1.0 - 6.0 * f1 - 8.0 * f7;
    for (int a = 0; a < 15; ++a) {
        const double wg = a == 0 ? w0 : a < 7 ? w1 : w7;
        p.wg[a] = (real)wg;
        // stored-value offsets of the flow populations (16-bit forms): rest-state values
        p.wf[a] = (real)(a == 0 ? f0 : a < 7 ? f1 : f7);
    }
    p.gbeta = (real)P.gbeta;
    p.T0 = (real)(0.5 * (P.T_hot + P.T_cold));
    p.T_hot = (real)P.T_hot;
    p.T_cold = (real)P.T_cold;
    p.cs2_phi = (real)P.cs2_phi;
    p.heat_source = (real)P.heat_source;
    p.ext_fx = (real)P.ext_force[0];
    p.ext_fy = (real)P.ext_force[1];
    p.ext_fz = (real)P.ext_force[2];
    p.e4_mode = P.e4_mode;
    p.adiabatic_mode = P.adiabatic_mode;
    p.boundary = P.boundary;
    p.nx = c->grid.nx;
    p.ny = c->grid.ny;
    p.nz = c->grid.nz;
    p.ncell = c->ncell;
    p.plane = c->plane;
    p.cell0 = c->cell0;
    return p;
}
template DevParams<double> lbm::dev_params<double>(const lbm_ctx*);
template DevParams<float> lbm::dev_params<float>(const lbm_ctx*);

// Wait for all work on a stream, polling an event with a time bound.
int lbm::wait_stream_for(cudaStream_t stream, double timeout_s, std::string* slot) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess)
        return record_error(slot, LBM_ECUDA, "CUDA error in cudaEventCreate: %s", cudaGetErrorString(e));
    e = cudaEventRecord(ev, stream);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev);
        return record_error(slot, LBM_ECUDA, "CUDA error in cudaEventRecord: %s", cudaGetErrorString(e));
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        e = cudaEventQuery(ev);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) {
            cudaEventDestroy(ev);
            return record_error(slot, LBM_ECUDA, "CUDA error while waiting: %s", cudaGetErrorString(e));
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) {
            cudaEventDestroy(ev);
            return record_error(slot, LBM_ETIMEOUT, "timed out waiting for the GPU%s");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
    }
    cudaEventDestroy(ev);
    return LBM_OK;
}

static int check_params(const lbm_params* p, int q) {
    for (int b = 4; b < 15; ++b)
        if (!(p->omega_f[b] > 0 && p->omega_f[b] < 2)) return 0;
    for (int b = 1; b < q; ++b)
        if (!(p->omega_g[b] > 0 && p->omega_g[b] < 2)) return 0;
    const double cmax = q == 15 ? 0.5 : 1.0 / 3.0;
    if (!(p->cs2_phi > 0 && p->cs2_phi <= cmax)) return 0;
    if (p->e4_mode != 0 && p->e4_mode != 1) return 0;
    if (p->adiabatic_mode != 0 && p->adiabatic_mode != 1) return 0;
    if (p->boundary < 0 || p->boundary > 15) return 0;
    if (!std::isfinite(p->heat_source)) return 0;
    return 1;
}

template <typename S>
static int run_init(lbm_ctx* c) {
    const ParamsOf<S> p = dev_params<typename Storage<S>::real>(c);
    CUDA_OR_FAIL(c, launch_init<S>(c->dev, p, c->opt.seed, c->cell0, c->opt.noise_amp, c->stream));
    CUDA_OR_FAIL(c, launch_residual<S>(c->dev, 0, p, 0, c->stream));
    return LBM_OK;
}

extern "C" int lbm_create_params(const lbm_grid* grid, int lattice, const lbm_params* params,
                                 const lbm_options* opt, lbm_ctx** out) {
    return lbm::create_context(grid, lattice, params, opt, 0, out);
}

int lbm::create_context(const lbm_grid* grid, int lattice, const lbm_params* params,
                        const lbm_options* opt, int64_t cell0, lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL%s");
    *out = nullptr;
    if (!valid_grid(grid)) return fail(nullptr, LBM_EINVAL, "invalid grid%s");
    if (!valid_lattice(lattice)) return fail(nullptr, LBM_EINVAL, "lattice must be 15 or 7%s");
    if (!params || !check_params(params, lattice))
        return fail(nullptr, LBM_EINVAL, "invalid parameters (rates must lie in (0, 2))%s");
    lbm_options o;
    if (opt) o = *opt; else lbm_default_options(&o);
    if (!valid_precision(o.precision))
        return fail(nullptr, LBM_EINVAL, "precision must be one of LBM_FP64, LBM_FP32, LBM_FP16_DEV, LBM_BF16_DEV%s");
    if (o.residual_interval < 0 || !(o.timeout_s > 0))
        return fail(nullptr, LBM_EINVAL, "invalid residual_interval or timeout%s");

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation failed%s");
    c->grid = *grid;
    c->Q = lattice;
    c->precision = o.precision;
    c->params = *params;
    c->opt = o;
    c->ncell = (int64_t)grid->nx * grid->ny * grid->nz;
    c->plane = plane_of(c->ncell);
    c->rsize = storage_bytes(o.precision);
    c->stream = (cudaStream_t)o.cuda_stream;
    c->cur = 0;
    c->steps = 0;
    c->last_residual = -1.0;
    c->cell0 = cell0;
    int rc = LBM_OK;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        rc = fail(nullptr, LBM_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
        delete c;
        return rc;
    }
    const Layout L = layout_of(grid, lattice, o.precision);
    if (o.device_arena) {
        if (o.device_arena_bytes < L.total || ((uintptr_t)o.device_arena & 255)) {
            delete c;
            return fail(nullptr, LBM_ENOMEM, "device arena too small or not 256-byte aligned%s");
        }
        c->arena = o.device_arena;
        c->own_arena = false;
    } else {
        e = cudaMalloc(&c->arena, L.total);
        if (e != cudaSuccess) {
            delete c;
            return fail(nullptr, LBM_ENOMEM, "cudaMalloc of the state failed: %s", cudaGetErrorString(e));
        }
        c->own_arena = true;
    }
    c->arena_bytes = L.total;
    e = cudaMallocHost(&c->host_bits, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        if (c->own_arena) cudaFree(c->arena);
        delete c;
        return fail(nullptr, LBM_ENOMEM, "cudaMallocHost failed: %s", cudaGetErrorString(e));
    }
    char* base = static_cast<char*>(c->arena);
    c->dev.precision = o.precision;
    c->dev.Q = lattice;
    const bool dev16 = o.precision == LBM_FP16_DEV || o.precision == LBM_BF16_DEV;
    for (int b = 0; b < 2; ++b) {
        c->dev.F[b] = base + L.F[b];
        c->dev.G[b] = base + L.G[b];
        c->dev.T[b] = dev16 ? base + L.T[b] : nullptr;
    }
    c->dev.snap = base + L.snap;
    c->dev.staging = reinterpret_cast<double*>(base + L.staging);
    c->dev.partials = reinterpret_cast<double*>(base + L.partials);
    c->dev.result = reinterpret_cast<double*>(base + L.result);
    c->dev.resid_bits = reinterpret_cast<unsigned long long*>(base + L.bits);
    c->dev.nonfinite = reinterpret_cast<int*>(base + L.bits + 64);
    c->dev.step_ctr = reinterpret_cast<unsigned*>(base + L.bits + 128);

    rc = LBM_OK;
    if (cudaMemsetAsync(base + L.bits, 0, 256, c->stream) != cudaSuccess)
        rc = fail(c, LBM_ECUDA, "cudaMemsetAsync failed%s");
    if (rc == LBM_OK)
        rc = with_storage(o.precision, [&](auto tag) { return run_init<decltype(tag)>(c); });
    if (rc == LBM_OK) rc = wait_stream(c);
    if (rc != LBM_OK) {
        g_err = c->err;
        lbm_destroy(c);
        return rc;
    }
    *out = c;
    return LBM_OK;
}

extern "C" int lbm_create(const lbm_grid* grid, int lattice, double Ra, double Pr, double Ma,
                          const lbm_options* opt, lbm_ctx** out) {
    lbm_params p;
    int rc = lbm_derive_params(grid, lattice, Ra, Pr, Ma, opt, &p);
    if (rc != LBM_OK) {
        if (out) *out = nullptr;
        return rc;
    }
    return lbm_create_params(grid, lattice, &p, opt, out);
}

// One step (and, when the step count reaches a multiple of the residual interval, the
// residual check) launched on stream `st` from buffer `cur`.
template <typename S>
static cudaError_t enqueue_step(lbm_ctx* c, const ParamsOf<S>& p, int cur, int64_t steps_after,
                                cudaStream_t st) {
    cudaError_t e = launch_step<S>(c->dev, cur, p, st);
    const int R = c->opt.residual_interval;
    if (e == cudaSuccess && R > 0 && steps_after % R == 0) {
        e = cudaMemsetAsync(c->dev.resid_bits, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = launch_residual<S>(c->dev, cur ^ 1, p, 1, st);
    }
    return e;
}

// The graph of residual_interval steps starting from buffer `cur` (captured on first use;
// NULL when capture is not possible, and then never tried again for this context).
#ifndef LBM_STEP_GRAPHS
#define LBM_STEP_GRAPHS 1
#endif
template <typename S>
static cudaGraphExec_t step_graph(lbm_ctx* c, const ParamsOf<S>& p, int cur) {
    if (!LBM_STEP_GRAPHS || c->graphs_failed) return nullptr;
    if (c->step_graph[cur]) return c->step_graph[cur];
    const int R = c->opt.residual_interval;
    bool ok = c->capture || cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) == cudaSuccess;
    cudaGraph_t g = nullptr;
    if (ok) ok = cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        int b = cur;
        cudaError_t e = cudaSuccess;
        for (int i = 1; i <= R && e == cudaSuccess; ++i, b ^= 1) e = enqueue_step<S>(c, p, b, i, c->capture);
        const cudaError_t e2 = cudaStreamEndCapture(c->capture, &g);
        ok = e == cudaSuccess && e2 == cudaSuccess && g;
    }
    if (ok) ok = cudaGraphInstantiate(&c->step_graph[cur], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        c->step_graph[cur] = nullptr;
        c->graphs_failed = true;
        cudaGetLastError();  // a failed capture leaves no error behind for the next launch
    }
    return c->step_graph[cur];
}

template <typename S>
static int run_steps(lbm_ctx* c, int64_t n, bool* checked) {
    const ParamsOf<S> p = dev_params<typename Storage<S>::real>(c);
    const int R = c->opt.residual_interval;
    for (int64_t s = 0; s < n;) {
        // whole residual intervals, aligned with the step count, go as one graph launch
        if (R > 0 && c->steps % R == 0 && n - s >= R) {
            if (cudaGraphExec_t g = step_graph<S>(c, p, c->cur)) {
                CUDA_OR_FAIL(c, cudaGraphLaunch(g, c->stream));
                if (R & 1) c->cur ^= 1;
                c->steps += R;
                s += R;
                *checked = true;
                continue;
            }
        }
        CUDA_OR_FAIL(c, enqueue_step<S>(c, p, c->cur, c->steps + 1, c->stream));
        c->cur ^= 1;
        c->steps += 1;
        s += 1;
        if (R > 0 && c->steps % R == 0) *checked = true;
    }
    return LBM_OK;
}

extern "C" int lbm_step(lbm_ctx* c, int64_t n) {
    NvtxRange nvtx("lbm_step");
    if (!c || n < 0) return fail(c, LBM_EINVAL, "invalid context or step count%s");
    if (c->owner) return fail(c, LBM_EINVAL, "a batch member is advanced by lbm_batch_step%s");
    DeviceGuard g(c->device);
    bool checked = false;
    int rc = with_storage(c->precision,
                          [&](auto tag) { return run_steps<decltype(tag)>(c, n, &checked); });
    if (rc != LBM_OK || !checked) return rc;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->host_bits, c->dev.resid_bits, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->host_bits + 1, c->dev.nonfinite, sizeof(int),
                                    cudaMemcpyDeviceToHost, c->stream));
    rc = wait_stream(c);
    if (rc != LBM_OK) return rc;
    unsigned long long bits = c->host_bits[0];
    double r;
    memcpy(&r, &bits, sizeof r);
    c->last_residual = r;
    if (*reinterpret_cast<int*>(c->host_bits + 1))
        return fail(c, LBM_EDIVERGED, "non-finite temperature detected%s");
    return LBM_OK;
}

template <typename S>
static int run_fields(lbm_ctx* c, double* const* outs, int64_t first, int64_t count) {
    const ParamsOf<S> p = dev_params<typename Storage<S>::real>(c);
    for (int w = 0; w < 5; ++w) {
        if (!outs[w]) continue;
        CUDA_OR_FAIL(c, launch_field<S>(c->dev, c->cur, p, w, c->stream));
        // the bounded wait comes first: a copy into pageable caller memory would block the
        // host until every earlier kernel on the stream has finished, with no time limit
        int rc = wait_stream(c);
        if (rc != LBM_OK) return rc;
        CUDA_OR_FAIL(c, cudaMemcpyAsync(outs[w], c->dev.staging + first, count * sizeof(double),
                                        cudaMemcpyDeviceToHost, c->stream));
        rc = wait_stream(c);
        if (rc != LBM_OK) return rc;
    }
    return LBM_OK;
}

int lbm::fields_cells(lbm_ctx* c, double* const outs[5], int64_t first, int64_t count) {
    if (!c || first < 0 || count < 0 || first + count > c->ncell)
        return fail(c, LBM_EINVAL, "invalid cell range%s");
    DeviceGuard g(c->device);
    return with_storage(c->precision,
                        [&](auto tag) { return run_fields<decltype(tag)>(c, outs, first, count); });
}

extern "C" int lbm_fields(lbm_ctx* c, double* rho, double* ux, double* uy, double* uz, double* T) {
    NvtxRange nvtx("lbm_fields");
    if (!c) return fail(c, LBM_EINVAL, "NULL context%s");
    double* outs[5] = {rho, ux, uy, uz, T};
    return fields_cells(c, outs, 0, c->ncell);
}

extern "C" int lbm_nusselt(lbm_ctx* c, lbm_nu* out) {
    NvtxRange nvtx("lbm_nusselt");
    if (!c || !out) return fail(c, LBM_EINVAL, "NULL argument%s");
    if (c->grid.nx < 2) return fail(c, LBM_EINVAL, "lbm_nusselt needs nx >= 2%s");
    DeviceGuard g(c->device);
    int lrc = with_storage(c->precision, [&](auto tag) {
        using S = decltype(tag);
        CUDA_OR_FAIL(c, launch_nusselt<S>(c->dev, c->cur, dev_params<typename Storage<S>::real>(c),
                                          c->params.U0, c->stream));
        return LBM_OK;
    });
    if (lrc != LBM_OK) return lrc;
    // bounded wait before the copy into host stack memory (see run_fields)
    int rc = wait_stream(c);
    if (rc != LBM_OK) return rc;
    double r[kResultDoubles];
    CUDA_OR_FAIL(c, cudaMemcpyAsync(r, c->dev.result, 11 * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
    rc = wait_stream(c);
    if (rc != LBM_OK) return rc;
    out->hot_wall_mean = r[0];
    out->cold_wall_mean = r[1];
    out->mid_mean = r[2];
    out->mid_max = r[3];
    out->mid_max_z = r[4];
    out->mid_min = r[5];
    out->mid_min_z = r[6];
    out->umax = r[7];
    out->umax_z = r[8];
    out->wmax = r[9];
    out->wmax_x = r[10];
    return LBM_OK;
}

extern "C" int lbm_residual(lbm_ctx* c, double* max_dT) {
    if (!c || !max_dT) return fail(c, LBM_EINVAL, "NULL argument%s");
    *max_dT = c->last_residual;
    return LBM_OK;
}

// Cells [first, first + n) of every population between the current state and FP64 host
// arrays whose population a starts at a * hs (queued on the context's stream).
template <typename S>
static int transfer_cells_(lbm_ctx* c, double* f, double* g, const double* fin, const double* gin,
                           int64_t first, int64_t n, int64_t hs) {
    using real = typename Storage<S>::real;
    const ParamsOf<S> p = dev_params<real>(c);
    const bool upload = fin || gin;
    // 16-bit forms only, else NULL
    float* Tn = c->dev.T[c->cur] ? static_cast<float*>(c->dev.T[c->cur]) + first : nullptr;
    if (upload && Storage<S>::deviation) {
        // the node temperatures the thermal deviations will refer to: T = sum_a g_a
        for (int a = 0; a < c->Q; ++a) {
            CUDA_OR_FAIL(c, cudaMemcpyAsync(c->dev.staging, gin + (int64_t)a * hs, n * sizeof(double),
                                            cudaMemcpyHostToDevice, c->stream));
            CUDA_OR_FAIL(c, launch_accumulate_T(Tn, c->dev.staging, n, a == 0, c->stream));
        }
    }
    if (!upload) {
        // every earlier kernel (the steps) finishes under the bounded wait before the first
        // copy into caller memory, which would otherwise block the host without a limit;
        // what follows is one short conversion kernel per plane
        const int rc = wait_stream(c);
        if (rc != LBM_OK) return rc;
    }
    for (int side = 0; side < 2; ++side) {
        const int q = side == 0 ? 15 : c->Q;
        S* dev = static_cast<S*>(side == 0 ? c->dev.F[c->cur] : c->dev.G[c->cur]);
        // stored-value offset: flow w_a; thermal w^phi_a times the node temperature
        const float* Tplane = side == 1 ? Tn : nullptr;
        for (int a = 0; a < q; ++a) {
            S* plane = dev + (int64_t)a * c->plane + first;
            const double offset = (double)(side == 0 ? p.wf[a] : p.wg[a]);
            if (upload) {  // host -> device
                const double* src = (side == 0 ? fin : gin) + (int64_t)a * hs;
                CUDA_OR_FAIL(c, cudaMemcpyAsync(c->dev.staging, src, n * sizeof(double),
                                                cudaMemcpyHostToDevice, c->stream));
                CUDA_OR_FAIL(c, launch_to_storage<S>(plane, c->dev.staging, n, offset, Tplane, c->stream));
            } else {  // device -> host
                double* dst = (side == 0 ? f : g) + (int64_t)a * hs;
                CUDA_OR_FAIL(c, launch_to_double<S>(c->dev.staging, plane, n, offset, Tplane, c->stream));
                CUDA_OR_FAIL(c, cudaMemcpyAsync(dst, c->dev.staging, n * sizeof(double),
                                                cudaMemcpyDeviceToHost, c->stream));
            }
            // the staging plane is reused plane after plane: stream order keeps each copy
            // behind the conversion that last used it, so no host wait is needed here
        }
    }
    return LBM_OK;
}

int lbm::transfer_cells(lbm_ctx* c, double* f, double* g, const double* fin, const double* gin,
                        int64_t first, int64_t count, int64_t hstride) {
    if (!c || first < 0 || count < 0 || first + count > c->ncell || hstride < count)
        return fail(c, LBM_EINVAL, "invalid cell range%s");
    DeviceGuard gd(c->device);
    return with_storage(c->precision, [&](auto tag) {
        return transfer_cells_<decltype(tag)>(c, f, g, fin, gin, first, count, hstride);
    });
}

int lbm::transfer_done(lbm_ctx* c, bool uploaded) {
    DeviceGuard gd(c->device);
    if (uploaded) {  // the residual's snapshot of the new state
        const int rc = with_storage(c->precision, [&](auto tag) {
            using S = decltype(tag);
            CUDA_OR_FAIL(c, launch_residual<S>(c->dev, c->cur, dev_params<typename Storage<S>::real>(c), 0,
                                               c->stream));
            return LBM_OK;
        });
        if (rc != LBM_OK) return rc;
        c->last_residual = -1.0;
    }
    return wait_stream(c);  // the host arrays (download) or sources (upload) are done with
}

template <typename S>
static int transfer(lbm_ctx* c, double* f, double* g, const double* fin, const double* gin) {
    const int rc = transfer_cells_<S>(c, f, g, fin, gin, 0, c->ncell, c->ncell);
    return rc != LBM_OK ? rc : transfer_done(c, fin || gin);
}

extern "C" int lbm_get_populations(lbm_ctx* c, double* f, double* g) {
    NvtxRange nvtx("lbm_get_populations");
    if (!c || !f || !g) return fail(c, LBM_EINVAL, "NULL argument%s");
    DeviceGuard gd(c->device);
    return with_storage(c->precision, [&](auto tag) {
        return transfer<decltype(tag)>(c, f, g, nullptr, nullptr);
    });
}

extern "C" int lbm_set_populations(lbm_ctx* c, const double* f, const double* g) {
    NvtxRange nvtx("lbm_set_populations");
    if (!c || !f || !g) return fail(c, LBM_EINVAL, "NULL argument%s");
    DeviceGuard gd(c->device);
    return with_storage(c->precision, [&](auto tag) {
        return transfer<decltype(tag)>(c, nullptr, nullptr, f, g);
    });
}

// Native-precision transfers: one copy per population plane between the host array and
// the state buffer (FP32 and FP64 contexts).
static int transfer_native(lbm_ctx* c, void* f, void* g, const void* fin, const void* gin) {
    if (c->precision != LBM_FP32 && c->precision != LBM_FP64)
        return fail(c, LBM_EINVAL, "native transfers need an FP32 or FP64 context%s");
    const bool upload = fin || gin;
    const size_t es = c->precision == LBM_FP64 ? 8 : 4;
    const size_t bytes = (size_t)c->ncell * es;
    if (!upload) {  // bounded wait before copies into caller memory (see transfer_cells_)
        const int rc = wait_stream(c);
        if (rc != LBM_OK) return rc;
    }
    for (int side = 0; side < 2; ++side) {
        const int q = side == 0 ? 15 : c->Q;
        char* dev = static_cast<char*>(side == 0 ? c->dev.F[c->cur] : c->dev.G[c->cur]);
        for (int a = 0; a < q; ++a) {
            char* plane = dev + (size_t)a * c->plane * es;
            if (upload) {
                const char* src = static_cast<const char*>(side == 0 ? fin : gin) + (size_t)a * bytes;
                CUDA_OR_FAIL(c, cudaMemcpyAsync(plane, src, bytes, cudaMemcpyHostToDevice, c->stream));
            } else {
                char* dst = static_cast<char*>(side == 0 ? f : g) + (size_t)a * bytes;
                CUDA_OR_FAIL(c, cudaMemcpyAsync(dst, plane, bytes, cudaMemcpyDeviceToHost, c->stream));
            }
        }
    }
    if (upload) {
        int rc = with_storage(c->precision, [&](auto tag) {
            using S = decltype(tag);
            CUDA_OR_FAIL(c, launch_residual<S>(c->dev, c->cur, dev_params<typename Storage<S>::real>(c), 0,
                                               c->stream));
            return LBM_OK;
        });
        if (rc != LBM_OK) return rc;
        c->last_residual = -1.0;
    }
    return wait_stream(c);
}

extern "C" int lbm_get_populations_native(lbm_ctx* c, void* f, void* g) {
    NvtxRange nvtx("lbm_get_populations_native");
    if (!c || !f || !g) return fail(c, LBM_EINVAL, "NULL argument%s");
    DeviceGuard gd(c->device);
    return transfer_native(c, f, g, nullptr, nullptr);
}

extern "C" int lbm_set_populations_native(lbm_ctx* c, const void* f, const void* g) {
    NvtxRange nvtx("lbm_set_populations_native");
    if (!c || !f || !g) return fail(c, LBM_EINVAL, "NULL argument%s");
    DeviceGuard gd(c->device);
    return transfer_native(c, nullptr, nullptr, f, g);
}

extern "C" int lbm_set_fields(lbm_ctx* c, const double* rho, const double* ux, const double* uy,
                              const double* uz, const double* T) {
    return lbm_init_fields(c, rho, ux, uy, uz, T, 0);
}

extern "C" int lbm_init_fields(lbm_ctx* c, const double* rho, const double* ux, const double* uy,
                               const double* uz, const double* T, int iterations) {
    if (!c || !ux || !uy || !uz || !T || iterations < 0)
        return fail(c, LBM_EINVAL, "NULL argument or negative iterations%s");
    DeviceGuard gd(c->device);
    int rc = with_storage(c->precision, [&](auto tag) {
        using S = decltype(tag);
        const ParamsOf<S> p = dev_params<typename Storage<S>::real>(c);
        CUDA_OR_FAIL(c, launch_set_fields<S>(c->dev, c->cur, p, rho, ux, uy, uz, T, c->stream));
        const int rounds = iterations + (iterations & 1);  // even: the state stays in its buffer
        for (int it = 0; it < rounds; ++it) {
            CUDA_OR_FAIL(c, launch_step<S>(c->dev, c->cur, p, c->stream));
            c->cur ^= 1;
            CUDA_OR_FAIL(c, launch_reimpose<S>(c->dev, c->cur, p, ux, uy, uz, T, c->stream));
        }
        CUDA_OR_FAIL(c, launch_residual<S>(c->dev, c->cur, p, 0, c->stream));
        return LBM_OK;
    });
    if (rc != LBM_OK) return rc;
    c->last_residual = -1.0;
    return wait_stream(c);
}

// ---------------------------------------------------------------------------------
// Checkpoint files: header, then FP64 populations (flow planes, then scalar planes).
// ---------------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];       // "LBMCKPT1"
    uint32_t version;    // 1
    int32_t lattice;     // Q of the scalar populations
    int32_t precision;   // LBM_FP64 ... LBM_BF16_DEV
    int32_t grid[3];
    int64_t steps;
    lbm_params params;
};
const char kCkptMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '1'};

bool read_header(FILE* fp, CkptHeader* h) {
    return fread(h, sizeof *h, 1, fp) == 1 && memcmp(h->magic, kCkptMagic, 8) == 0 && h->version == 1 &&
           (h->lattice == 15 || h->lattice == 7) && h->grid[0] > 0 && h->grid[1] > 0 && h->grid[2] > 0;
}
}  // namespace

extern "C" int lbm_save(lbm_ctx* c, const char* path) {
    NvtxRange nvtx("lbm_save");
    if (!c || !path) return fail(c, LBM_EINVAL, "NULL argument%s");
    const int64_t nf = 15 * c->ncell, ng = (int64_t)c->Q * c->ncell;
    double* f = static_cast<double*>(malloc((size_t)(nf + ng) * sizeof(double)));
    if (!f) return fail(c, LBM_ENOMEM, "no host memory for the checkpoint%s");
    double* g = f + nf;
    int rc = lbm_get_populations(c, f, g);
    if (rc != LBM_OK) {
        free(f);
        return rc;
    }
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.lattice = c->Q;
    h.precision = c->precision;
    h.grid[0] = c->grid.nx;
    h.grid[1] = c->grid.ny;
    h.grid[2] = c->grid.nz;
    h.steps = c->steps;
    h.params = c->params;
    FILE* fp = fopen(path, "wb");
    bool ok = fp && fwrite(&h, sizeof h, 1, fp) == 1 &&
              fwrite(f, sizeof(double), (size_t)(nf + ng), fp) == (size_t)(nf + ng);
    if (fp && fclose(fp) != 0) ok = false;
    free(f);
    if (!ok) {
        remove(path);
        return fail(c, LBM_EINVAL, "cannot write the checkpoint file%s");
    }
    return LBM_OK;
}

extern "C" int lbm_checkpoint_info(const char* path, lbm_grid* grid, int* lattice, int* precision,
                                   lbm_params* params, int64_t* steps) {
    if (!path) return fail(nullptr, LBM_EINVAL, "NULL path%s");
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(nullptr, LBM_EINVAL, "cannot open the checkpoint file%s");
    CkptHeader h;
    const bool ok = read_header(fp, &h);
    fclose(fp);
    if (!ok) return fail(nullptr, LBM_EINVAL, "not a checkpoint file%s");
    if (grid) *grid = lbm_grid{h.grid[0], h.grid[1], h.grid[2]};
    if (lattice) *lattice = h.lattice;
    if (precision) *precision = h.precision;
    if (params) *params = h.params;
    if (steps) *steps = h.steps;
    return LBM_OK;
}

extern "C" int lbm_restore(lbm_ctx* c, const char* path) {
    NvtxRange nvtx("lbm_restore");
    if (!c || !path) return fail(c, LBM_EINVAL, "NULL argument%s");
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(c, LBM_EINVAL, "cannot open the checkpoint file%s");
    CkptHeader h;
    if (!read_header(fp, &h)) {
        fclose(fp);
        return fail(c, LBM_EINVAL, "not a checkpoint file%s");
    }
    if (h.grid[0] != c->grid.nx || h.grid[1] != c->grid.ny || h.grid[2] != c->grid.nz ||
        h.lattice != c->Q || h.precision != c->precision) {
        fclose(fp);
        return fail(c, LBM_EINVAL, "the checkpoint's grid, lattice or precision differ from the context's%s");
    }
    const int64_t nf = 15 * c->ncell, ng = (int64_t)c->Q * c->ncell;
    double* f = static_cast<double*>(malloc((size_t)(nf + ng) * sizeof(double)));
    if (!f) {
        fclose(fp);
        return fail(c, LBM_ENOMEM, "no host memory for the checkpoint%s");
    }
    const bool ok = fread(f, sizeof(double), (size_t)(nf + ng), fp) == (size_t)(nf + ng);
    fclose(fp);
    if (!ok) {
        free(f);
        return fail(c, LBM_EINVAL, "the checkpoint file is short%s");
    }
    const int rc = lbm_set_populations(c, f, f + nf);
    free(f);
    if (rc == LBM_OK) c->steps = h.steps;
    return rc;
}

extern "C" int lbm_get_params(const lbm_ctx* c, lbm_params* out) {
    if (!c || !out) return LBM_EINVAL;
    *out = c->params;
    return LBM_OK;
}

extern "C" int64_t lbm_steps_done(const lbm_ctx* c) { return c ? c->steps : -1; }

extern "C" const char* lbm_last_error(const lbm_ctx* c) {
    return c ? c->err.c_str() : g_err.c_str();
}

extern "C" int lbm_set_timeout(lbm_ctx* c, double timeout_s) {
    if (!c || !(timeout_s > 0)) return fail(c, LBM_EINVAL, "NULL context or timeout <= 0%s");
    c->opt.timeout_s = timeout_s;
    return LBM_OK;
}

extern "C" int lbm_synchronize(lbm_ctx* c) {
    if (!c) return fail(c, LBM_EINVAL, "NULL context%s");
    DeviceGuard g(c->device);
    return wait_stream(c);
}

extern "C" void lbm_destroy(lbm_ctx* c) {
    if (!c || c->owner) return;  // batch members go with their batch
    lbm::destroy_context(c);
}

void lbm::destroy_context(lbm_ctx* c) {
    {
        DeviceGuard g(c->device);
        wait_stream(c);
        for (cudaGraphExec_t& g : c->step_graph)
            if (g) cudaGraphExecDestroy(g);
        if (c->capture) cudaStreamDestroy(c->capture);
        if (c->own_arena && c->arena) cudaFree(c->arena);
        if (c->host_bits) cudaFreeHost(c->host_bits);
    }
    delete c;
}
