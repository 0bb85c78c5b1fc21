// context.h -- the library's private view of a context (include/lbm.h declares it opaque)
// and the helpers the C ABI translation units share (not installed).
#pragma once

#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>

#include "internal.h"
#include "lbm.h"

// NVTX ranges around the C ABI's calls (header-only NVTX 3: no cost without a tool attached;
// build with -DLBM_NO_NVTX to leave them out).
#ifndef LBM_NO_NVTX
#include <nvtx3/nvToolsExt.h>
#endif
namespace lbm {
struct NvtxRange {
#ifndef LBM_NO_NVTX
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
#else
    explicit NvtxRange(const char*) {}
#endif
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace lbm

struct lbm_batch;

struct lbm_ctx {
    lbm_grid grid;
    int Q;
    int precision;
    lbm_params params;
    lbm_options opt;
    int64_t ncell, plane;
    size_t rsize;
    int device;
    cudaStream_t stream;
    void* arena;
    bool own_arena;
    size_t arena_bytes;
    lbm::DevState dev;
    int cur;              // buffer holding the current state
    int64_t steps;
    double last_residual; // < 0: none recorded yet
    unsigned long long* host_bits;  // pinned: residual bits + flag
    lbm_batch* owner;     // non-NULL: a member of a batch, stepped by the batch only
    std::string err;
    // lbm_step's graphs: residual_interval steps and the residual check that ends them,
    // one per starting buffer, captured on a private stream when first needed
    cudaStream_t capture = nullptr;
    cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
    bool graphs_failed = false;  // capture not possible here: launch the steps one by one
    int64_t cell0 = 0;  // global index of cell 0 (slabs of a larger grid), for the initial noise
};

namespace lbm {

// Formats the message (fmt holds one %s for detail), stores it in *slot (if any) and as
// the thread's last error, and returns code.
int record_error(std::string* slot, int code, const char* fmt, const char* detail = nullptr);

inline int fail(lbm_ctx* ctx, int code, const char* fmt, const char* detail = nullptr) {
    return record_error(ctx ? &ctx->err : nullptr, code, fmt, detail);
}

// Waits for all work queued on `stream`, polling an event, for at most timeout_s seconds.
int wait_stream_for(cudaStream_t stream, double timeout_s, std::string* err_slot);

inline int wait_stream(lbm_ctx* c) { return wait_stream_for(c->stream, c->opt.timeout_s, &c->err); }

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Kernel parameters of a context in the arithmetic type `real`.
template <typename real>
DevParams<real> dev_params(const lbm_ctx* c);

// Frees a context (lbm_destroy without the batch-member check).
void destroy_context(lbm_ctx* c);

// lbm_create_params with the initial noise drawn for global cell indices cell0 + c (a slab
// of a larger grid starts from that grid's state); cell0 = 0 is lbm_create_params.
int create_context(const lbm_grid* grid, int lattice, const lbm_params* params,
                   const lbm_options* opt, int64_t cell0, lbm_ctx** out);

// FP64 host populations <-> cells [first, first + count) of the current state, population
// a of the host side starting at a * hstride (download: f, g; upload: fin, gin).  Queued
// on the context's stream; transfer_done ends a series of them (an upload with the
// residual's snapshot) with a bounded wait.  lbm_get/set_populations are the whole range.
int transfer_cells(lbm_ctx* c, double* f, double* g, const double* fin, const double* gin,
                   int64_t first, int64_t count, int64_t hstride);
int transfer_done(lbm_ctx* c, bool uploaded);

// lbm_fields for cells [first, first + count): outs[w] (rho, ux, uy, uz, T; NULL = skip)
// receive count values each.
int fields_cells(lbm_ctx* c, double* const outs[5], int64_t first, int64_t count);

// Bytes of the device arena of one context.
size_t context_arena_bytes(const lbm_grid* g, int q, int precision);

// Run fn(S{}) with S the storage type of the precision.
template <typename Fn>
int with_storage(int precision, Fn&& fn) {
    switch (precision) {
    case LBM_FP64: return fn(double{});
    case LBM_FP32: return fn(float{});
    case LBM_FP16_DEV: return fn(__half{});
    default: return fn(__nv_bfloat16{});
    }
}

}  // namespace lbm

#define CUDA_OR_FAIL(ctx, call)                                                     \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return ::lbm::fail((ctx), LBM_ECUDA, "CUDA error in " #call ": %s",     \
                               cudaGetErrorString(e_));                             \
    } while (0)

// Keeps the caller's current device and restores it on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
