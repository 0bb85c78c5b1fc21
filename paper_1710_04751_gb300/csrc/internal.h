// internal.h -- declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "storage.cuh"

namespace lbm {

// Kernel parameters, passed by value (they land in the constant bank).
template <typename real>
struct DevParams {
    real om_f[15];      // flow relaxation rates (App. A)
    real om_g[15];      // thermal relaxation rates (Sec. 2.2 / App. C)
    real wg[15];        // thermal rest weights w^phi_a (anti-bounce-back)
    real wf[15];        // stored-value offsets of the flow populations (16-bit forms: w_a)
    real gbeta, T0, T_hot, T_cold, cs2_phi;
    real heat_source;   // uniform scalar source R (Eq. 4)
    real ext_fx, ext_fy, ext_fz;
    int e4_mode, adiabatic_mode, boundary;
    int nx, ny, nz;
    int64_t ncell;      // nx * ny * nz
    int64_t plane;      // elements between population planes (ncell rounded up to 64)
    int64_t cell0;      // global index of cell 0 (slabs of a larger grid; 0 otherwise)
};

// Host-side view of one context's device buffers for the launchers.
struct DevState {
    int precision;      // 0 fp64, 1 fp32, 2 fp16 deviations, 3 bf16 deviations
    int Q;              // 15 or 7
    void* F[2];
    void* G[2];
    void* T[2];         // 16-bit forms: FP32 node temperature the thermal deviations refer to
    void* snap;         // temperature snapshot for the residual
    double* staging;    // one plane of doubles
    double* partials;   // per-block reduction partials
    double* result;     // reduction results
    unsigned long long* resid_bits;
    int* nonfinite;
    unsigned* step_ctr; // 16-bit forms: steps taken, per buffer parity (the rounding dither)
};

constexpr int kPartialBlocks = 1024;   // max blocks of the face reduction
constexpr int kResultDoubles = 16;

// Launchers (return cudaGetLastError()), templated on the storage type S (double,
// float, __half, __nv_bfloat16); arithmetic is Storage<S>::real.  `cur` selects the
// source buffer of a step.
template <typename S>
using ParamsOf = DevParams<typename Storage<S>::real>;

template <typename S>
cudaError_t launch_step(const DevState& s, int cur, const ParamsOf<S>& p, cudaStream_t st);
// (cell0: global index of the context's cell 0, for the seeded initial noise)
template <typename S>
cudaError_t launch_init(const DevState& s, const ParamsOf<S>& p, uint64_t seed, int64_t cell0,
                        double amp, cudaStream_t st);
// one population plane between FP64 host values and storage (offset: that plane's
// stored-value offset, used by the 16-bit forms)
// (thermal planes of the 16-bit forms: offset = w^phi_a and Tn the node temperatures)
template <typename S>
cudaError_t launch_to_storage(S* dst, const double* src, int64_t n, double offset, const float* Tn,
                              cudaStream_t st);
template <typename S>
cudaError_t launch_to_double(double* dst, const S* src, int64_t n, double offset, const float* Tn,
                             cudaStream_t st);
// Tn = src (first) or Tn += src, in FP32: node temperatures of an uploaded state
cudaError_t launch_accumulate_T(float* Tn, const double* src, int64_t n, int first, cudaStream_t st);
template <typename S>
cudaError_t launch_field(const DevState& s, int cur, const ParamsOf<S>& p, int which,
                         cudaStream_t st);
template <typename S>
cudaError_t launch_residual(const DevState& s, int cur, const ParamsOf<S>& p, int record,
                            cudaStream_t st);
template <typename S>
cudaError_t launch_nusselt(const DevState& s, int cur, const ParamsOf<S>& p, double U0,
                           cudaStream_t st);

// Nusselt reduction into caller-provided device scratch: one face block per 256 face
// cells (`blocks` of them, partial pairs at partials[0 .. 2*blocks)), result[0..11).
template <typename S>
cudaError_t launch_nusselt_into(const S* F, const S* G, const ParamsOf<S>& p, double U0,
                                int Q, int blocks, double* partials, double* result,
                                cudaStream_t st);

// Populations of buffer `cur` set to the equilibria of the given device fields (rho NULL:
// 1), in every storage form.
template <typename S>
cudaError_t launch_set_fields(const DevState& s, int cur, const ParamsOf<S>& p, const double* rho,
                              const double* ux, const double* uy, const double* uz,
                              const double* T, cudaStream_t st);

// p <- p - p_eq(current u, T) + p_eq(target u, T) on buffer `cur` (rho kept).
template <typename S>
cudaError_t launch_reimpose(const DevState& s, int cur, const ParamsOf<S>& p, const double* ux,
                            const double* uy, const double* uz, const double* T, cudaStream_t st);

// Message returned by lbm_last_error(NULL) on this thread.
void set_last_error(const char* msg);

}  // namespace lbm
