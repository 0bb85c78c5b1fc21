// bridge.cu -- between the solver and the warm-start network: the training targets of a
// solved cavity, and a cavity started from the network's prediction (the equilibria of
// the predicted fields, lbm_set_fields), resampled trilinearly when the grids differ.
#include "../context.h"
#include "lbm_net.h"
#include "nn.h"

using namespace lbm;

namespace {

// out[c * 4 + j] = scale * field[c]
__global__ void put_channel_kernel(const double* __restrict__ field, int64_t n, int j, double scale,
                                   float* __restrict__ out) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x)
        out[c * 4 + j] = (float)(scale * field[c]);
}

// Trilinear resampling of a cell-centred m^3 prediction [voxel][4] onto the nx x ny x nz
// nodes of a context (node i at (i + 1/2) / nx of the box, clamped at the walls), scaled
// back to lattice units: u = p * U0, T = p / 2.
__global__ void resample_kernel(const float* __restrict__ pred, int m, int nx, int ny, int nz,
                                double U0, double* __restrict__ ux, double* __restrict__ uy,
                                double* __restrict__ uz, double* __restrict__ T) {
    const int64_t total = (int64_t)nx * ny * nz;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((int64_t)nx * ny));
        const double s[3] = {(i + 0.5) * m / nx - 0.5, (j + 0.5) * m / ny - 0.5, (k + 0.5) * m / nz - 0.5};
        int lo[3];
        double w[3];
        for (int d = 0; d < 3; ++d) {
            const double v = fmin(fmax(s[d], 0.0), (double)(m - 1));
            lo[d] = min((int)floor(v), m - 2 < 0 ? 0 : m - 2);
            w[d] = m == 1 ? 0.0 : v - lo[d];
        }
        double acc[4] = {0, 0, 0, 0};
        for (int corner = 0; corner < 8; ++corner) {
            const int dx = corner & 1, dy = (corner >> 1) & 1, dz = corner >> 2;
            const double wt = (dx ? w[0] : 1 - w[0]) * (dy ? w[1] : 1 - w[1]) * (dz ? w[2] : 1 - w[2]);
            if (wt == 0.0) continue;
            const int64_t v = ((int64_t)(lo[2] + dz) * m + (lo[1] + dy)) * m + (lo[0] + dx);
            for (int q = 0; q < 4; ++q) acc[q] += wt * pred[v * 4 + q];
        }
        ux[c] = acc[0] * U0;
        uy[c] = acc[1] * U0;
        uz[c] = acc[2] * U0;
        T[c] = 0.5 * acc[3];
    }
}

}  // namespace

extern "C" int lbm_net_targets(lbm_ctx* c, float* out) {
    if (!c || !out) return fail(c, LBM_EINVAL, "NULL argument%s");
    if (!(c->params.U0 > 0)) return fail(c, LBM_EINVAL, "the context has no velocity scale U0%s");
    DeviceGuard g(c->device);
    const int64_t n = c->ncell;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 65535);
    int rc = with_storage(c->precision, [&](auto tag) {
        using S = decltype(tag);
        const ParamsOf<S> p = dev_params<typename Storage<S>::real>(c);
        for (int j = 0; j < 4; ++j) {
            CUDA_OR_FAIL(c, launch_field<S>(c->dev, c->cur, p, j + 1, c->stream));
            const double scale = j < 3 ? 1.0 / c->params.U0 : 2.0;
            put_channel_kernel<<<blocks, 256, 0, c->stream>>>(c->dev.staging, n, j, scale, out);
            CUDA_OR_FAIL(c, cudaGetLastError());
        }
        return LBM_OK;
    });
    if (rc != LBM_OK) return rc;
    return wait_stream(c);
}

extern "C" int lbm_net_warm_start(lbm_ctx* c, const float* pred, int m, int iterations) {
    if (!c || !pred || m < 1 || iterations < 0)
        return fail(c, LBM_EINVAL, "NULL prediction, grid size < 1 or negative iterations%s");
    if (!(c->params.U0 > 0)) return fail(c, LBM_EINVAL, "the context has no velocity scale U0%s");
    DeviceGuard g(c->device);
    const int64_t n = c->ncell;
    double* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, (size_t)4 * n * sizeof(double));
    if (e != cudaSuccess) return fail(c, LBM_ENOMEM, "cudaMalloc failed: %s", cudaGetErrorString(e));
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 65535);
    resample_kernel<<<blocks, 256, 0, c->stream>>>(pred, m, c->grid.nx, c->grid.ny, c->grid.nz,
                                                   c->params.U0, buf, buf + n, buf + 2 * n, buf + 3 * n);
    e = cudaGetLastError();
    int rc = e == cudaSuccess
                 ? lbm_init_fields(c, nullptr, buf, buf + n, buf + 2 * n, buf + 3 * n, iterations)
                 : fail(c, LBM_ECUDA, "resampling failed: %s", cudaGetErrorString(e));
    cudaFree(buf);  // lbm_init_fields waited for the stream
    return rc;
}
