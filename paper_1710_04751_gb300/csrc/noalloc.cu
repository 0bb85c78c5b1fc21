// noalloc.cu -- lbm_nusselt_noalloc: the Nusselt / peak-velocity reduction of
// lbm_nusselt for populations the caller already holds in device memory, without any
// device allocation by the library.
//
// Who needs it: a caller whose device memory is owned by something else -- an
// application or framework that reserves all of it up front and hands out slices, a
// real-time loop that must not pay for (or risk the failure of) cudaMalloc/cudaFree in
// steady state, a plug-in that is not allowed to allocate after start-up.  Such callers
// keep their populations in their own buffers and still want the library's reduction.
//
// The reduction needs a little global scratch (one partial pair per face block and the
// eleven results).  Here it lives in a file-scope static __device__ array, so every GPU
// that loads this library holds it until the process exits.  Host code must not pass
// the array's name to a kernel (in host code that name is only a host-side stand-in):
// its device address is looked up once per device with cudaGetSymbolAddress, on the
// first call made with that device current, and that pointer is what the kernels get.
// The cached address belongs to the device's primary context: a caller that resets the
// device (cudaDeviceReset) must not use this entry point in the same process afterwards,
// since the module, and with it the array, is loaded again at another address.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <mutex>
#include <thread>

#include "lbm.h"
#include "internal.h"

using namespace lbm;

namespace {

constexpr int kNoAllocBlocks = 1024;                   // face blocks of 256 face cells
constexpr int kNoAllocFaceCells = kNoAllocBlocks * 256;  // max ny * nz: 262144 (e.g. 512 x 512)
constexpr int kScratchDoubles = 2 * kNoAllocBlocks + 16;  // partial pairs + results: 16.5 KB

static __device__ __align__(256) double lbm_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};  // device address of the array, per device

// One-time set-up for the current device: the array's device address.
cudaError_t scratch_for_current_device(double** out, int* device) {
    cudaError_t e = cudaGetDevice(device);
    if (e != cudaSuccess) return e;
    if (*device < 0 || *device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[*device]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, lbm_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[*device] = static_cast<double*>(ptr);
    }
    *out = g_scratch_ptr[*device];
    return cudaSuccess;
}

int fail(int code, const char* msg) {
    char buf[320];
    snprintf(buf, sizeof buf, "lbm_nusselt_noalloc: %s", msg);
    set_last_error(buf);  // read back with lbm_last_error(NULL)
    return code;
}

template <typename real>
DevParams<real> params_for(const lbm_grid& g, int Q, const lbm_params& P, int64_t plane) {
    DevParams<real> p;
    memset(&p, 0, sizeof p);
    for (int b = 0; b < 15; ++b) {
        p.om_f[b] = (real)P.omega_f[b];
        p.om_g[b] = (real)P.omega_g[b];
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
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.ncell = (int64_t)g.nx * g.ny * g.nz;
    p.plane = plane;
    (void)Q;
    return p;
}

// Bounded wait on the stream by polling (no event object is created).
cudaError_t wait_polling(cudaStream_t st, double timeout_s, bool* timed_out) {
    const auto t0 = std::chrono::steady_clock::now();
    *timed_out = false;
    for (;;) {
        const cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) return e;
        if (e != cudaErrorNotReady) return e;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) {
            *timed_out = true;
            return cudaSuccess;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
    }
}

}  // namespace

extern "C" int lbm_nusselt_noalloc(const void* f_dev, const void* g_dev, int64_t plane,
                                   int precision, const lbm_grid* grid, int lattice,
                                   const lbm_params* params, void* cuda_stream, lbm_nu* out) {
    if (!f_dev || !g_dev || !grid || !params || !out) return fail(LBM_EINVAL, "NULL argument");
    if (grid->nx < 2 || grid->ny < 1 || grid->nz < 1) return fail(LBM_EINVAL, "needs nx >= 2, ny, nz >= 1");
    if (lattice != LBM_THERMAL_D3Q15 && lattice != LBM_THERMAL_D3Q7)
        return fail(LBM_EINVAL, "lattice must be 15 or 7");
    if (precision != LBM_FP32 && precision != LBM_FP64)
        return fail(LBM_EINVAL, "precision must be LBM_FP32 or LBM_FP64");
    const int64_t ncell = (int64_t)grid->nx * grid->ny * grid->nz;
    if (plane < ncell) return fail(LBM_EINVAL, "plane stride smaller than nx*ny*nz");
    const int64_t nface = (int64_t)grid->ny * grid->nz;
    if (nface > kNoAllocFaceCells) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "ny*nz = %lld exceeds the static scratch limit of %d face cells (1024 blocks "
                 "of 256)", (long long)nface, kNoAllocFaceCells);
        return fail(LBM_EINVAL, buf);
    }
    double* scratch = nullptr;
    int device = -1;
    cudaError_t e = scratch_for_current_device(&scratch, &device);
    if (e != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
    double* partials = scratch;
    double* result = scratch + 2 * kNoAllocBlocks;
    const int blocks = (int)((nface + 255) / 256);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == LBM_FP64) {
        const DevParams<double> p = params_for<double>(*grid, lattice, *params, plane);
        e = launch_nusselt_into<double>(static_cast<const double*>(f_dev),
                                        static_cast<const double*>(g_dev), p, params->U0, lattice,
                                        blocks, partials, result, st);
    } else {
        const DevParams<float> p = params_for<float>(*grid, lattice, *params, plane);
        e = launch_nusselt_into<float>(static_cast<const float*>(f_dev),
                                       static_cast<const float*>(g_dev), p, params->U0, lattice,
                                       blocks, partials, result, st);
    }
    if (e != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
    // The bounded wait comes before the copy: a device-to-host copy into pageable memory
    // (the stack array below) returns only once every earlier kernel on the stream has
    // finished, so issued first it would wait without any time limit.
    bool timed_out = false;
    e = wait_polling(st, 600.0, &timed_out);
    if (e != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
    if (timed_out) return fail(LBM_ETIMEOUT, "timed out waiting for the GPU");
    double r[11];  // the stream is idle now: this copy is all that is left to wait for
    e = cudaMemcpyAsync(r, result, sizeof r, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
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
