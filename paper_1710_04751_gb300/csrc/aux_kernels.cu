// aux_kernels.cu -- initial state, precision conversion, macroscopic fields and the
// FP64 reductions (Nusselt numbers, peak velocities, convergence residual) of the
// cavity problem of arXiv:1710.04751, Sec. 3.
#include <math.h>

#include "internal.h"
#include "lattice.cuh"

namespace lbm {

// ---------------------------------------------------------------------------------
// Initial state: fluid at rest (f = rest weights) and T = seeded uniform noise in
// [-amp, amp], g = w^phi T.  The noise is splitmix64 (Steele, Lea & Flood 2014, with
// S. Vigna's published constants) of (seed xor cell index), top 53 bits.  The cell index
// is global: a context holding planes of a larger grid (one slab of a decomposition)
// passes the global index of its cell 0 as cell0 and so starts from the same state.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

template <typename S, int Q>
__global__ void init_kernel(S* __restrict__ F, S* __restrict__ G, float* __restrict__ Tn,
                            ParamsOf<S> p, uint64_t seed, int64_t cell0, double amp, double w0, double w1,
                            double w7, double v0, double v1, double v7) {
    using real = typename Storage<S>::real;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.ncell) return;
    const uint64_t r = splitmix64(seed ^ (uint64_t)(c + cell0));
    const double u01 = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    const double T = amp * (2.0 * u01 - 1.0);
#pragma unroll
    for (int a = 0; a < 15; ++a)
        F[a * p.plane + c] = Storage<S>::store_f((real)(a == 0 ? w0 : a < 7 ? w1 : w7), p.wf[a]);
    // 16-bit forms: g is stored as its deviation from w^phi_a T of this node (zero here)
    real Tref = real(0);
    if constexpr (Storage<S>::deviation) {
        Tref = (real)T;
        Tn[c] = (float)T;
    }
#pragma unroll
    for (int a = 0; a < Q; ++a)
        G[a * p.plane + c] = Storage<S>::store((real)((a == 0 ? v0 : a < 7 ? v1 : v7) * T), p.wg[a] * Tref);
}

template <typename S>
cudaError_t launch_init(const DevState& s, const ParamsOf<S>& p, uint64_t seed, int64_t cell0,
                        double amp, cudaStream_t st) {
    // rest weights: flow (c_s^2 = 1/3) and thermal (c_sphi^2), from the equilibria
    const double cs2 = 1.0 / 3.0, ct = (double)p.cs2_phi;
    const double w7 = cs2 * cs2 / 8.0, w1 = 0.5 * (cs2 - cs2 * cs2), w0 = 1.0 - 6.0 * w1 - 8.0 * w7;
    double v7, v1, v0;
    if (s.Q == 15) {
        v7 = ct * ct / 8.0;
        v1 = 0.5 * (ct - ct * ct);
        v0 = 1.0 - 6.0 * v1 - 8.0 * v7;
    } else {
        v7 = 0.0;
        v1 = 0.5 * ct;
        v0 = 1.0 - 6.0 * v1;
    }
    const int threads = 256;
    const unsigned blocks = (unsigned)((p.ncell + threads - 1) / threads);
    S* F = static_cast<S*>(s.F[0]);
    S* G = static_cast<S*>(s.G[0]);
    float* Tn = static_cast<float*>(s.T[0]);
    if (s.Q == 15)
        init_kernel<S, 15><<<blocks, threads, 0, st>>>(F, G, Tn, p, seed, cell0, amp, w0, w1, w7, v0, v1, v7);
    else
        init_kernel<S, 7><<<blocks, threads, 0, st>>>(F, G, Tn, p, seed, cell0, amp, w0, w1, w7, v0, v1, v7);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Conversion of one population plane between FP64 host values and storage (host
// transfers stage FP64 planes).  The 16-bit forms encode and decode exactly as the step
// kernel does (FP32 offset arithmetic), so set(get(state)) restores the FP16 state.
// ---------------------------------------------------------------------------------
// offset of node c: `offset` (flow planes), or `offset` * Tn[c] (thermal planes of the
// 16-bit forms, offset = w^phi_a)
template <typename S>
__device__ __forceinline__ typename Storage<S>::real conv_offset(double offset,
                                                                 const float* __restrict__ Tn,
                                                                 int64_t c) {
    using real = typename Storage<S>::real;
    return Tn ? (real)offset * Tn[c] : (real)offset;
}
template <typename S>
__global__ void to_storage_kernel(S* __restrict__ dst, const double* __restrict__ src, int64_t n,
                                  double offset, const float* __restrict__ Tn) {
    using real = typename Storage<S>::real;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x)
        dst[c] = Tn ? Storage<S>::store((real)src[c], conv_offset<S>(offset, Tn, c))
                    : Storage<S>::store_f((real)src[c], (real)offset);
}
template <typename S>
__global__ void to_double_kernel(double* __restrict__ dst, const S* __restrict__ src, int64_t n,
                                 double offset, const float* __restrict__ Tn) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x)
        dst[c] = (double)(Tn ? Storage<S>::load(src[c], conv_offset<S>(offset, Tn, c))
                             : Storage<S>::load_f(src[c], (typename Storage<S>::real)offset));
}
// Tn[c] (+)= (float) src[c]: the node temperature of a state being uploaded (16-bit forms)
__global__ void accumulate_T_kernel(float* __restrict__ Tn, const double* __restrict__ src,
                                    int64_t n, int first) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x)
        Tn[c] = first ? (float)src[c] : Tn[c] + (float)src[c];
}

static unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <typename S>
cudaError_t launch_to_storage(S* dst, const double* src, int64_t n, double offset, const float* Tn,
                              cudaStream_t st) {
    to_storage_kernel<S><<<grid_for(n, 256), 256, 0, st>>>(dst, src, n, offset, Tn);
    return cudaGetLastError();
}
template <typename S>
cudaError_t launch_to_double(double* dst, const S* src, int64_t n, double offset, const float* Tn,
                             cudaStream_t st) {
    to_double_kernel<S><<<grid_for(n, 256), 256, 0, st>>>(dst, src, n, offset, Tn);
    return cudaGetLastError();
}
cudaError_t launch_accumulate_T(float* Tn, const double* src, int64_t n, int first, cudaStream_t st) {
    accumulate_T_kernel<<<grid_for(n, 256), 256, 0, st>>>(Tn, src, n, first);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Macroscopic fields of the stored (post-collision) state: rho = sum f, T = sum g,
// rho u = sum f e - F/2 (collision added F to the momentum, Eq. 2a), in FP64.
// ---------------------------------------------------------------------------------
// stored thermal population a of node c, decoded
template <typename S>
__device__ __forceinline__ double thermal_value(const S* __restrict__ G, const float* __restrict__ Tn,
                                                const ParamsOf<S>& p, int a, int64_t c) {
    typename Storage<S>::real off = 0;
    if constexpr (Storage<S>::deviation) off = p.wg[a] * Tn[c];
    return (double)Storage<S>::load(G[a * p.plane + c], off);
}

template <typename S, int Q>
__device__ __forceinline__ void node_macro(const S* __restrict__ F, const S* __restrict__ G,
                                           const float* __restrict__ Tn,
                                           const ParamsOf<S>& p, int64_t c, double& rho,
                                           double& ux, double& uy, double& uz, double& T) {
    double r = 0, jx = 0, jy = 0, jz = 0, t = 0;
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        const double v = (double)Storage<S>::load_f(F[a * p.plane + c], p.wf[a]);
        r += v;
        jx += ex(a) * v;
        jy += ey(a) * v;
        jz += ez(a) * v;
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) t += thermal_value<S>(G, Tn, p, a, c);
    t -= 0.5 * (double)p.heat_source;  // collision added R: phi = sum g~ - R/2 (Eq. 25)
    const double Fz = (double)p.ext_fz + (double)p.gbeta * (t - (double)p.T0);
    rho = r;
    ux = (jx - 0.5 * (double)p.ext_fx) / r;
    uy = (jy - 0.5 * (double)p.ext_fy) / r;
    uz = (jz - 0.5 * Fz) / r;
    T = t;
}

template <typename S, int Q>
__global__ void field_kernel(const S* __restrict__ F, const S* __restrict__ G,
                             const float* __restrict__ Tn, ParamsOf<S> p, int which,
                             double* __restrict__ out) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < p.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        double rho, ux, uy, uz, T;
        node_macro<S, Q>(F, G, Tn, p, c, rho, ux, uy, uz, T);
        out[c] = which == 0 ? rho : which == 1 ? ux : which == 2 ? uy : which == 3 ? uz : T;
    }
}

template <typename S>
cudaError_t launch_field(const DevState& s, int cur, const ParamsOf<S>& p, int which,
                         cudaStream_t st) {
    const S* F = static_cast<const S*>(s.F[cur]);
    const S* G = static_cast<const S*>(s.G[cur]);
    const float* Tn = static_cast<const float*>(s.T[cur]);
    if (s.Q == 15)
        field_kernel<S, 15><<<grid_for(p.ncell, 256), 256, 0, st>>>(F, G, Tn, p, which, s.staging);
    else
        field_kernel<S, 7><<<grid_for(p.ncell, 256), 256, 0, st>>>(F, G, Tn, p, which, s.staging);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Warp / block reductions in FP64.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
// (value, index) arg-max with ties broken toward the smaller index
__device__ __forceinline__ void argmax_combine(double& v, int& idx, double v2, int i2) {
    if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
}
__device__ __forceinline__ void warp_argmax(double& v, int& idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_down_sync(0xffffffffu, v, o);
        const int i2 = __shfl_down_sync(0xffffffffu, idx, o);
        argmax_combine(v, idx, v2, i2);
    }
}

// ---------------------------------------------------------------------------------
// Residual: max over the grid of |T - T_snapshot|, snapshot <- T, and a flag for any
// non-finite T.  With record == 0 the kernel only refreshes the snapshot.
// ---------------------------------------------------------------------------------
template <typename S, int Q>
__global__ void __launch_bounds__(256) residual_kernel(const S* __restrict__ G,
                                                       const float* __restrict__ Tn,
                                                       typename Storage<S>::real* __restrict__ snap,
                                                       ParamsOf<S> p, int record,
                                                       unsigned long long* __restrict__ max_bits,
                                                       int* __restrict__ nonfinite) {
    using real = typename Storage<S>::real;
    double local = 0.0;
    int bad = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < p.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        real T = real(0);
#pragma unroll
        for (int a = 0; a < Q; ++a) T += (real)thermal_value<S>(G, Tn, p, a, c);
        T -= real(0.5) * p.heat_source;
        if (!isfinite(T)) bad = 1;
        const double d = fabs((double)T - (double)snap[c]);
        if (d > local) local = d;
        snap[c] = T;
    }
    if (!record) return;
    __shared__ double red[8];
    local = warp_max(local);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = local;
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(nonfinite, 1);
    __syncthreads();
    if (warp == 0) {
        double v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        v = warp_max(v);
        // non-negative doubles order like their bit patterns
        if (lane == 0) atomicMax(max_bits, (unsigned long long)__double_as_longlong(v));
    }
}

template <typename S>
cudaError_t launch_residual(const DevState& s, int cur, const ParamsOf<S>& p, int record,
                            cudaStream_t st) {
    using real = typename Storage<S>::real;
    const S* G = static_cast<const S*>(s.G[cur]);
    const float* Tn = static_cast<const float*>(s.T[cur]);
    real* snap = static_cast<real*>(s.snap);
    const unsigned blocks = grid_for(p.ncell, 256) > 152 * 8 ? 152 * 8 : grid_for(p.ncell, 256);
    if (s.Q == 15)
        residual_kernel<S, 15><<<blocks, 256, 0, st>>>(G, Tn, snap, p, record, s.resid_bits, s.nonfinite);
    else
        residual_kernel<S, 7><<<blocks, 256, 0, st>>>(G, Tn, snap, p, record, s.resid_bits, s.nonfinite);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Nusselt numbers (Sec. 3): local Nu = L |dT/dn| / dT with the second-order one-sided
// derivative (9 T_1 - T_2 - 8 T_w)/3 at the half-way wall.  Kernel 1 sums the local Nu
// of both x faces per block; kernel 2 (one block) adds the partials in a fixed order
// and evaluates the symmetry-plane lines: Nu(z) on the hot wall, |u_x|(z) on the
// vertical centreline and |u_z|(x) on the horizontal centreline.
// ---------------------------------------------------------------------------------
template <typename S, int Q>
__device__ __forceinline__ double node_T(const S* __restrict__ G, const float* __restrict__ Tn,
                                         const ParamsOf<S>& p, int i, int j, int k) {
    const int64_t c = ((int64_t)k * p.ny + j) * p.nx + i;
    double t = 0.0;
#pragma unroll
    for (int a = 0; a < Q; ++a) t += thermal_value<S>(G, Tn, p, a, c);
    return t - 0.5 * (double)p.heat_source;
}

template <typename S, int Q>
__global__ void __launch_bounds__(256) nusselt_faces_kernel(const S* __restrict__ G,
                                                            const float* __restrict__ Tn,
                                                            ParamsOf<S> p,
                                                            double* __restrict__ partials) {
    const double L = p.nx, dT = (double)p.T_hot - (double)p.T_cold;
    double hot = 0.0, cold = 0.0;
    const int64_t nface = (int64_t)p.ny * p.nz;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nface;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(f % p.ny), k = (int)(f / p.ny);
        const double th1 = node_T<S, Q>(G, Tn, p, p.nx - 1, j, k);
        const double th2 = node_T<S, Q>(G, Tn, p, p.nx - 2, j, k);
        const double tc1 = node_T<S, Q>(G, Tn, p, 0, j, k);
        const double tc2 = node_T<S, Q>(G, Tn, p, 1, j, k);
        hot += -L * (9.0 * th1 - th2 - 8.0 * (double)p.T_hot) / (3.0 * dT);
        cold += L * (9.0 * tc1 - tc2 - 8.0 * (double)p.T_cold) / (3.0 * dT);
    }
    __shared__ double red[2][8];
    hot = warp_sum(hot);
    cold = warp_sum(cold);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = hot; red[1][warp] = cold; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double h = 0.0, c = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { h += red[0][w]; c += red[1][w]; }
        partials[2 * blockIdx.x] = h;
        partials[2 * blockIdx.x + 1] = c;
    }
}

template <typename S, int Q>
__global__ void __launch_bounds__(256) nusselt_lines_kernel(const S* __restrict__ F,
                                                            const S* __restrict__ G,
                                                            const float* __restrict__ Tn,
                                                            ParamsOf<S> p, int nblocks,
                                                            double U0,
                                                            const double* __restrict__ partials,
                                                            double* __restrict__ result) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const double L = nx, dT = (double)p.T_hot - (double)p.T_cold;
    const int j0 = (ny - 1) / 2, j1 = ny / 2, i0 = (nx - 1) / 2, i1 = nx / 2;
    const int k0 = (nz - 1) / 2, k1 = nz / 2;
    // mid-plane Nu(z) on the hot wall: sum, max, min
    double nsum = 0.0, nmax = -INFINITY, nmin = -INFINITY;  // nmin kept as max of -Nu
    int kmax = 0x7fffffff, kmin = 0x7fffffff;
    double umax = -1.0, wmax = -1.0;
    int kum = 0x7fffffff, iwm = 0x7fffffff;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        const double t1 = 0.5 * (node_T<S, Q>(G, Tn, p, nx - 1, j0, k) + node_T<S, Q>(G, Tn, p, nx - 1, j1, k));
        const double t2 = 0.5 * (node_T<S, Q>(G, Tn, p, nx - 2, j0, k) + node_T<S, Q>(G, Tn, p, nx - 2, j1, k));
        const double nu = -L * (9.0 * t1 - t2 - 8.0 * (double)p.T_hot) / (3.0 * dT);
        nsum += nu;
        argmax_combine(nmax, kmax, nu, k);
        argmax_combine(nmin, kmin, -nu, k);
        double r, ux, uy, uz, T, acc = 0.0;
        const int is[2] = {i0, i1}, js[2] = {j0, j1};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                node_macro<S, Q>(F, G, Tn, p, ((int64_t)k * ny + js[b]) * nx + is[a], r, ux, uy, uz, T);
                acc += ux;
            }
        argmax_combine(umax, kum, fabs(0.25 * acc), k);
    }
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        double r, ux, uy, uz, T, acc = 0.0;
        const int js[2] = {j0, j1}, ks[2] = {k0, k1};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                node_macro<S, Q>(F, G, Tn, p, ((int64_t)ks[b] * ny + js[a]) * nx + i, r, ux, uy, uz, T);
                acc += uz;
            }
        argmax_combine(wmax, iwm, fabs(0.25 * acc), i);
    }
    // face sums: every thread adds a fixed slice of the partials, then a fixed tree
    double hot = 0.0, cold = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        hot += partials[2 * b];
        cold += partials[2 * b + 1];
    }
    nsum = warp_sum(nsum);
    hot = warp_sum(hot);
    cold = warp_sum(cold);
    warp_argmax(nmax, kmax);
    warp_argmax(nmin, kmin);
    warp_argmax(umax, kum);
    warp_argmax(wmax, iwm);
    __shared__ double sv[7][8];
    __shared__ int si[4][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        sv[0][warp] = nsum; sv[1][warp] = hot; sv[2][warp] = cold;
        sv[3][warp] = nmax; sv[4][warp] = nmin; sv[5][warp] = umax; sv[6][warp] = wmax;
        si[0][warp] = kmax; si[1][warp] = kmin; si[2][warp] = kum; si[3][warp] = iwm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0, s2 = 0;
        double vmax = sv[3][0], vmin = sv[4][0], vu = sv[5][0], vw = sv[6][0];
        int amax = si[0][0], amin = si[1][0], au = si[2][0], aw = si[3][0];
        for (int w = 0; w < nw; ++w) {
            s0 += sv[0][w]; s1 += sv[1][w]; s2 += sv[2][w];
            if (w) {
                argmax_combine(vmax, amax, sv[3][w], si[0][w]);
                argmax_combine(vmin, amin, sv[4][w], si[1][w]);
                argmax_combine(vu, au, sv[5][w], si[2][w]);
                argmax_combine(vw, aw, sv[6][w], si[3][w]);
            }
        }
        const double u0 = U0 > 0.0 ? U0 : 1.0;
        result[0] = s1 / ((double)ny * nz);
        result[1] = s2 / ((double)ny * nz);
        result[2] = s0 / nz;
        result[3] = vmax;
        result[4] = (amax + 0.5) / nz;
        result[5] = -vmin;
        result[6] = (amin + 0.5) / nz;
        result[7] = vu / u0;
        result[8] = (au + 0.5) / nz;
        result[9] = vw / u0;
        result[10] = (aw + 0.5) / nx;
    }
}

template <typename S>
cudaError_t launch_nusselt(const DevState& s, int cur, const ParamsOf<S>& p, double U0,
                           cudaStream_t st) {
    const S* F = static_cast<const S*>(s.F[cur]);
    const S* G = static_cast<const S*>(s.G[cur]);
    const float* Tn = static_cast<const float*>(s.T[cur]);
    int64_t nface = (int64_t)p.ny * p.nz;
    int blocks = (int)((nface + 255) / 256);
    if (blocks > kPartialBlocks) blocks = kPartialBlocks;
    if (s.Q == 15) {
        nusselt_faces_kernel<S, 15><<<blocks, 256, 0, st>>>(G, Tn, p, s.partials);
        nusselt_lines_kernel<S, 15><<<1, 256, 0, st>>>(F, G, Tn, p, blocks, U0, s.partials, s.result);
    } else {
        nusselt_faces_kernel<S, 7><<<blocks, 256, 0, st>>>(G, Tn, p, s.partials);
        nusselt_lines_kernel<S, 7><<<1, 256, 0, st>>>(F, G, Tn, p, blocks, U0, s.partials, s.result);
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_nusselt_into(const S* F, const S* G, const ParamsOf<S>& p, double U0,
                                int Q, int blocks, double* partials, double* result,
                                cudaStream_t st) {
    // FP32 / FP64 only: no node-temperature plane
    if (Q == 15) {
        nusselt_faces_kernel<S, 15><<<blocks, 256, 0, st>>>(G, nullptr, p, partials);
        nusselt_lines_kernel<S, 15><<<1, 256, 0, st>>>(F, G, nullptr, p, blocks, U0, partials, result);
    } else {
        nusselt_faces_kernel<S, 7><<<blocks, 256, 0, st>>>(G, nullptr, p, partials);
        nusselt_lines_kernel<S, 7><<<1, 256, 0, st>>>(F, G, nullptr, p, blocks, U0, partials, result);
    }
    return cudaGetLastError();
}

#define LBM_INSTANTIATE(S)                                                                         \
    template cudaError_t launch_init<S>(const DevState&, const ParamsOf<S>&, uint64_t, int64_t,     \
                                        double, cudaStream_t);                                     \
    template cudaError_t launch_to_storage<S>(S*, const double*, int64_t, double, const float*,     \
                                              cudaStream_t);                                       \
    template cudaError_t launch_to_double<S>(double*, const S*, int64_t, double, const float*,      \
                                             cudaStream_t);                                        \
    template cudaError_t launch_field<S>(const DevState&, int, const ParamsOf<S>&, int,             \
                                         cudaStream_t);                                            \
    template cudaError_t launch_residual<S>(const DevState&, int, const ParamsOf<S>&, int,          \
                                            cudaStream_t);                                         \
    template cudaError_t launch_nusselt<S>(const DevState&, int, const ParamsOf<S>&, double,        \
                                           cudaStream_t);                                          \
    template cudaError_t launch_nusselt_into<S>(const S*, const S*, const ParamsOf<S>&, double, int, \
                                                int, double*, double*, cudaStream_t);
LBM_INSTANTIATE(double)
LBM_INSTANTIATE(float)
LBM_INSTANTIATE(__half)
LBM_INSTANTIATE(__nv_bfloat16)

}  // namespace lbm
