// internal.h -- declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Kernel parameters, passed by value (they land in the constant bank).
template <typename real>
struct DevParams {
    real om_f[15];      // flow relaxation rates (App. A)
    real om_g[15];      // thermal relaxation rates (Sec. 2.2 / App. C)
    real wg[15];        // thermal rest weights w^phi_a (anti-bounce-back)
    real gbeta, T0, T_hot, T_cold, cs2_phi;
    real ext_fx, ext_fy, ext_fz;
    int e4_mode, adiabatic_mode, boundary;
    int nx, ny, nz;
    int64_t ncell;      // nx * ny * nz
    int64_t plane;      // elements between population planes (ncell rounded up to 64)
};

// Host-side view of one context's device buffers for the launchers.
struct DevState {
    int precision;      // 0 fp64, 1 fp32
    int Q;              // 15 or 7
    void* F[2];
    void* G[2];
    void* snap;         // temperature snapshot for the residual
    double* staging;    // one plane of doubles
    double* partials;   // per-block reduction partials
    double* result;     // reduction results
    unsigned long long* resid_bits;
    int* nonfinite;
};

constexpr int kPartialBlocks = 1024;   // max blocks of the face reduction
constexpr int kResultDoubles = 16;

// Launchers (return cudaGetLastError()).  `cur` selects the source buffer of a step.
template <typename real>
cudaError_t launch_step(const DevState& s, int cur, const DevParams<real>& p, cudaStream_t st);
template <typename real>
cudaError_t launch_init(const DevState& s, const DevParams<real>& p, uint64_t seed, double amp,
                        cudaStream_t st);
template <typename real>
cudaError_t launch_to_real(real* dst, const double* src, int64_t n, cudaStream_t st);
template <typename real>
cudaError_t launch_to_double(double* dst, const real* src, int64_t n, cudaStream_t st);
template <typename real>
cudaError_t launch_field(const DevState& s, int cur, const DevParams<real>& p, int which,
                         cudaStream_t st);
template <typename real>
cudaError_t launch_residual(const DevState& s, int cur, const DevParams<real>& p, int record,
                            cudaStream_t st);
template <typename real>
cudaError_t launch_nusselt(const DevState& s, int cur, const DevParams<real>& p, double U0,
                           cudaStream_t st);

// Nusselt reduction into caller-provided device scratch: one face block per 256 face
// cells (`blocks` of them, partial pairs at partials[0 .. 2*blocks)), result[0..11).
template <typename real>
cudaError_t launch_nusselt_into(const real* F, const real* G, const DevParams<real>& p, double U0,
                                int Q, int blocks, double* partials, double* result,
                                cudaStream_t st);

// Message returned by lbm_last_error(NULL) on this thread.
void set_last_error(const char* msg);

}  // namespace lbm
