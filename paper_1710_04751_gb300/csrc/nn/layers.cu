// layers.cu -- the non-GEMM kernels of the warm-start network.  Activations are
// channels-last, [voxel][channel] with voxel = ((b * n + z) * n + y) * n + x, BF16 where a
// GEMM reads them and FP32 for gradients.  A 3x3x3 convolution with zero padding is the
// GEMM of its im2col matrix: row = output voxel, column k = tap * cin + ci with
// tap = (kz * 3 + ky) * 3 + kx reading the input at (z + kz - 1, y + ky - 1, x + kx - 1),
// columns padded with zeros to a multiple of 64.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "nn.h"

namespace lbm {
namespace nn {

__device__ __forceinline__ int64_t vox(int b, int z, int y, int x, int n) {
    return (((int64_t)b * n + z) * n + y) * n + x;
}

static unsigned blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b > 1048576 ? 1048576 : b);
}

// ---- im2col --------------------------------------------------------------------------
// 8 channels (16 bytes) per thread when cin % 8 == 0, else one element per thread.
__global__ void im2col8_kernel(const __nv_bfloat16* __restrict__ X, int B, int n, int cin, int Kp,
                               __nv_bfloat16* __restrict__ Xcol) {
    const int kq = Kp / 8;
    const int64_t total = (int64_t)B * n * n * n * kq;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = q / kq;
        const int k = (int)(q - m * kq) * 8;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (k < 27 * cin) {
            const int tap = k / cin, ci = k - tap * cin;
            const int kz = tap / 9, ky = (tap / 3) % 3, kx = tap % 3;
            const int x = (int)(m % n), y = (int)((m / n) % n), z = (int)((m / ((int64_t)n * n)) % n);
            const int b = (int)(m / ((int64_t)n * n * n));
            const int sz = z + kz - 1, sy = y + ky - 1, sx = x + kx - 1;
            if ((unsigned)sz < (unsigned)n && (unsigned)sy < (unsigned)n && (unsigned)sx < (unsigned)n)
                v = *reinterpret_cast<const uint4*>(X + vox(b, sz, sy, sx, n) * cin + ci);
        }
        *reinterpret_cast<uint4*>(Xcol + m * Kp + k) = v;
    }
}

__global__ void im2col1_kernel(const __nv_bfloat16* __restrict__ X, int B, int n, int cin, int Kp,
                               __nv_bfloat16* __restrict__ Xcol) {
    const int64_t total = (int64_t)B * n * n * n * Kp;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = q / Kp;
        const int k = (int)(q - m * Kp);
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (k < 27 * cin) {
            const int tap = k / cin, ci = k - tap * cin;
            const int kz = tap / 9, ky = (tap / 3) % 3, kx = tap % 3;
            const int x = (int)(m % n), y = (int)((m / n) % n), z = (int)((m / ((int64_t)n * n)) % n);
            const int b = (int)(m / ((int64_t)n * n * n));
            const int sz = z + kz - 1, sy = y + ky - 1, sx = x + kx - 1;
            if ((unsigned)sz < (unsigned)n && (unsigned)sy < (unsigned)n && (unsigned)sx < (unsigned)n)
                v = X[vox(b, sz, sy, sx, n) * cin + ci];
        }
        Xcol[m * Kp + k] = v;
    }
}

cudaError_t im2col(const __nv_bfloat16* X, int B, int n, int cin, int Kp, __nv_bfloat16* Xcol,
                   cudaStream_t st) {
    const int64_t M = (int64_t)B * n * n * n;
    if (cin % 8 == 0)
        im2col8_kernel<<<blocks_for(M * (Kp / 8), 256), 256, 0, st>>>(X, B, n, cin, Kp, Xcol);
    else
        im2col1_kernel<<<blocks_for(M * Kp, 256), 256, 0, st>>>(X, B, n, cin, Kp, Xcol);
    return cudaGetLastError();
}

// ---- im2col, transposed: XcolT[k][m] = Xcol[m][k], written directly ---------------------
// A tile is (tap, 32-channel chunk, 64 consecutive voxels); blocks take tiles by grid
// stride, the 27 cin / 32 tiles of a voxel block one after the other (their sources stay
// in cache while the XcolT rows stream out).  Each thread reads 8 channels (16 B) of one shifted source voxel and scatters them
// into a shared [32 channels][66] BF16 tile (rows of 33 words: the 8 channel rows a warp
// writes, and the 32 row segments it reads back, fall in distinct banks); each thread then
// writes 8 voxels of one channel row (16 B) of XcolT.  Rows k >= 27 cin are not touched.
#ifndef LBM_IM2COLT_VOXELS_FASTEST
#define LBM_IM2COLT_VOXELS_FASTEST 0
#endif
__global__ void __launch_bounds__(256) im2colT_kernel(const __nv_bfloat16* __restrict__ X, int ln, int cin,
                                                      int M, int tiles, __nv_bfloat16* __restrict__ XcolT) {
    __shared__ uint32_t tileW[32 * 33];
    unsigned short* tileH = reinterpret_cast<unsigned short*>(tileW);
    const int n = 1 << ln, mask = n - 1;
    const int chunks = cin >> 5, tcs = 27 * chunks;
    const int t = threadIdx.x;
    const int v = t >> 2, g = t & 3;   // load phase: voxel of the tile, 8-channel group
    const int c = t >> 3, sg = t & 7;  // store phase: channel row, 8-voxel segment
    const int vblocks = (M + 63) >> 6;
    for (int it = blockIdx.x; it < tiles; it += gridDim.x) {
#if LBM_IM2COLT_VOXELS_FASTEST
        // the voxel block runs fastest: long runs of each XcolT row are written together
        const int tc = it / vblocks, vb = it - tc * vblocks;
#else
        // the (tap, chunk) index runs fastest: the tiles in flight share their source voxels
        const int vb = it / tcs, tc = it - vb * tcs;
#endif
        const int tap = tc / chunks, c0 = (tc - tap * chunks) << 5;
        const int kz = tap / 9, ky = (tap / 3) % 3, kx = tap % 3;
        const int m0 = vb << 6;
        {
            const int m = m0 + v;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (m < M) {
                const int sx = (m & mask) + kx - 1, sy = ((m >> ln) & mask) + ky - 1;
                const int sz = ((m >> (2 * ln)) & mask) + kz - 1, b = m >> (3 * ln);
                if ((unsigned)sz < (unsigned)n && (unsigned)sy < (unsigned)n && (unsigned)sx < (unsigned)n) {
                    const int src = (((b << ln) + sz) << ln | sy) << ln | sx;
                    val = *reinterpret_cast<const uint4*>(X + (int64_t)src * cin + c0 + g * 8);
                }
            }
            const uint32_t w[4] = {val.x, val.y, val.z, val.w};
#pragma unroll
            for (int e = 0; e < 8; ++e)
                tileH[(g * 8 + e) * 66 + v] = (unsigned short)(w[e >> 1] >> ((e & 1) * 16));
        }
        __syncthreads();
        {
            const int m = m0 + sg * 8;
            if (m < M) {  // M is a multiple of 8: the segment is whole
                const uint32_t* row = tileW + c * 33 + sg * 4;
                *reinterpret_cast<uint4*>(XcolT + (int64_t)(tap * cin + c0 + c) * M + m) =
                    make_uint4(row[0], row[1], row[2], row[3]);
            }
        }
        __syncthreads();
    }
}

bool im2colT_supported(int n, int cin, int64_t M) {
    return cin % 32 == 0 && M % 8 == 0 && n >= 1 && (n & (n - 1)) == 0 && M < (int64_t(1) << 31) &&
           (M + 63) / 64 * 27 * (cin / 32) < (int64_t(1) << 31);
}

cudaError_t im2colT(const __nv_bfloat16* X, int B, int n, int cin, int Kp, __nv_bfloat16* XcolT,
                    cudaStream_t st) {
    const int64_t M = (int64_t)B * n * n * n;
    if (!im2colT_supported(n, cin, M) || Kp < 27 * cin || ((uintptr_t)X & 15) || ((uintptr_t)XcolT & 15))
        return cudaErrorInvalidValue;
    int ln = 0;
    while ((1 << ln) < n) ++ln;
    const int tiles = (int)((M + 63) / 64 * 27 * (cin / 32));
    const unsigned grid = (unsigned)std::min(tiles, 152 * 8 * 4);
    im2colT_kernel<<<grid, 256, 0, st>>>(X, ln, cin, (int)M, tiles, XcolT);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || Kp == 27 * cin) return e;
    // the padding rows 27 cin .. Kp - 1 read as zeros
    return cudaMemsetAsync(XcolT + (int64_t)27 * cin * M, 0, (size_t)(Kp - 27 * cin) * M * 2, st);
}

// ---- transpose of a BF16 matrix (32 x 32 tiles through shared memory) -----------------
__global__ void transpose_kernel(const __nv_bfloat16* __restrict__ in, int64_t R, int64_t C,
                                 int64_t ld_in, __nv_bfloat16* __restrict__ out, int64_t ld_out) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[i][threadIdx.x] = in[r * ld_in + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) out[c * ld_out + r] = tile[threadIdx.x][i];
    }
}

cudaError_t transpose(const __nv_bfloat16* in, int64_t R, int64_t C, int64_t ld_in,
                      __nv_bfloat16* out, int64_t ld_out, cudaStream_t st) {
    const int64_t gy = (R + 31) / 32, gx = (C + 31) / 32;
    if (gy > 65535) {  // long matrices: in slabs of 65535 tile rows
        for (int64_t r = 0; r < R; r += 65535 * 32) {
            const int64_t rr = R - r < 65535 * 32 ? R - r : 65535 * 32;
            cudaError_t e = transpose(in + r * ld_in, rr, C, ld_in, out + r, ld_out, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    transpose_kernel<<<dim3((unsigned)gx, (unsigned)gy), dim3(32, 8), 0, st>>>(in, R, C, ld_in, out,
                                                                            ld_out);
    return cudaGetLastError();
}

// ---- bias + ReLU -------------------------------------------------------------------------
__global__ void bias_relu_kernel(const float* __restrict__ Y, const float* __restrict__ bias,
                                 int64_t M, int C, __nv_bfloat16* __restrict__ A, int64_t ldA,
                                 int c_off) {
    const int64_t total = M * C;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = q / C;
        const int c = (int)(q - m * C);
        A[m * ldA + c_off + c] = __float2bfloat16_rn(fmaxf(Y[q] + bias[c], 0.f));
    }
}

cudaError_t bias_relu(const float* Y, const float* bias, int64_t M, int C, __nv_bfloat16* A,
                      int64_t ldA, int c_off, cudaStream_t st) {
    bias_relu_kernel<<<blocks_for(M * C, 256), 256, 0, st>>>(Y, bias, M, C, A, ldA, c_off);
    return cudaGetLastError();
}

// Gradient sums over rows are taken in a fixed order -- rows ascending within a thread,
// then the threads of a block, then the blocks in a fixed tree (sum_partials_kernel) -- so
// that training gives the same result on every run.

// out[i] = sum over b of part[b ld + first + i], one block of 256 threads per i: thread t
// adds the partials t, t + 256, ... in order, then the 256 sums are added pairwise in a
// fixed tree (the same order on every run, independent of timing).
__global__ void __launch_bounds__(256) sum_partials_kernel(const float* __restrict__ part, int nblocks, int ld,
                                                           int first, float* __restrict__ out) {
    __shared__ float red[256];
    const int i = blockIdx.x, t = threadIdx.x;
    float s = 0.f;
    for (int b = t; b < nblocks; b += 256) s += part[(int64_t)b * ld + first + i];
    red[t] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) out[i] = red[0];
}

static void sum_partials(const float* part, int nblocks, int ld, int first, int count, float* out,
                         cudaStream_t st) {
    sum_partials_kernel<<<count, 256, 0, st>>>(part, nblocks, ld, first, out);
}

static int64_t rows_per_block(int64_t M, int64_t at_least, int max_blocks) {
    return std::max<int64_t>(at_least, (M + max_blocks - 1) / max_blocks);
}

// dZ = dA where A > 0 (BF16, the GEMM operand) and the per-block sums of dZ over channels:
// thread t takes channel c = t % C and every R-th row (R = 256 / C lanes, lane t / C) of
// the block's rows; the lanes are then added in order.  C <= 256, blockDim = 256.
__global__ void relu_bwd_kernel(const float* __restrict__ dA, const __nv_bfloat16* __restrict__ A,
                                int64_t ldA, int a_off, int64_t M, int C, int64_t rows,
                                __nv_bfloat16* __restrict__ dZ, float* __restrict__ part) {
    __shared__ float acc[256];
    const int R = 256 / C;
    const int c = threadIdx.x % C, r = threadIdx.x / C;
    const int64_t m0 = (int64_t)blockIdx.x * rows, m1 = m0 + rows < M ? m0 + rows : M;
    float s = 0.f;
    if (r < R) {
        for (int64_t m = m0 + r; m < m1; m += R) {
            const float g = __bfloat162float(A[m * ldA + a_off + c]) > 0.f ? dA[m * C + c] : 0.f;
            dZ[m * C + c] = __float2bfloat16_rn(g);
            s += g;
        }
    }
    acc[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.f;
        for (int l = 0; l < R; ++l) t += acc[l * C + threadIdx.x];
        part[(int64_t)blockIdx.x * C + threadIdx.x] = t;
    }
}

// The same with 8 channels per thread (16-byte loads of A and dZ, two 16-byte loads of dA):
// thread t takes the channel group g = t % G (G = C / 8) and every R-th row (R = 256 / G
// lanes); the per-channel sums of the lanes are then added in lane order.
__global__ void relu_bwd8_kernel(const float* __restrict__ dA, const __nv_bfloat16* __restrict__ A,
                                 int64_t ldA, int a_off, int M, int C, int rows,
                                 __nv_bfloat16* __restrict__ dZ, float* __restrict__ part) {
    __shared__ float acc[256][9];
    const int G = C >> 3, R = 256 / G;
    const int g = threadIdx.x % G, r = threadIdx.x / G;
    const int m0 = blockIdx.x * rows, m1 = min(m0 + rows, M);
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r < R) {
#pragma unroll 2
        for (int m = m0 + r; m < m1; m += R) {
            const uint4 a = *reinterpret_cast<const uint4*>(A + (int64_t)m * ldA + a_off + 8 * g);
            const float4 d0 = *reinterpret_cast<const float4*>(dA + (int64_t)m * C + 8 * g);
            const float4 d1 = *reinterpret_cast<const float4*>(dA + (int64_t)m * C + 8 * g + 4);
            const __nv_bfloat162* ah = reinterpret_cast<const __nv_bfloat162*>(&a);
            const float d[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
            uint4 o;
            uint32_t* ow = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 af = __bfloat1622float2(ah[j]);
                const float g0 = af.x > 0.f ? d[2 * j] : 0.f, g1 = af.y > 0.f ? d[2 * j + 1] : 0.f;
                const __nv_bfloat162 q = __floats2bfloat162_rn(g0, g1);
                ow[j] = *reinterpret_cast<const uint32_t*>(&q);
                s[2 * j] += g0;
                s[2 * j + 1] += g1;
            }
            *reinterpret_cast<uint4*>(dZ + (int64_t)m * C + 8 * g) = o;
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[threadIdx.x][j] = s[j];
    __syncthreads();
    if (threadIdx.x < C) {
        const int gc = threadIdx.x >> 3, j = threadIdx.x & 7;
        float t = 0.f;
        for (int l = 0; l < R; ++l) t += acc[l * G + gc][j];
        part[(int64_t)blockIdx.x * C + threadIdx.x] = t;
    }
}

cudaError_t relu_bwd(const float* dA, const __nv_bfloat16* A, int64_t ldA, int a_off, int64_t M,
                     int C, __nv_bfloat16* dZ, float* db, float* part, cudaStream_t st) {
    if (C < 1 || C > 256 || M < 1) return cudaErrorInvalidValue;
    const bool vec = C % 8 == 0 && ldA % 8 == 0 && a_off % 8 == 0 && ((uintptr_t)A & 15) == 0 &&
                     ((uintptr_t)dA & 15) == 0 && ((uintptr_t)dZ & 15) == 0 && M < (int64_t(1) << 31) - 65536;
    if (vec) {
        const int64_t rows = rows_per_block(M, 256 / (C / 8), kMaxPartialBlocks);
        const int nblocks = (int)((M + rows - 1) / rows);
        relu_bwd8_kernel<<<nblocks, 256, 0, st>>>(dA, A, ldA, a_off, (int)M, C, (int)rows, dZ, part);
        sum_partials(part, nblocks, C, 0, C, db, st);
        return cudaGetLastError();
    }
    const int64_t rows = rows_per_block(M, 256 / C, kMaxPartialBlocks);
    const int nblocks = (int)((M + rows - 1) / rows);
    relu_bwd_kernel<<<nblocks, 256, 0, st>>>(dA, A, ldA, a_off, M, C, rows, dZ, part);
    sum_partials(part, nblocks, C, 0, C, db, st);
    return cudaGetLastError();
}

// ---- 2x average pooling and nearest upsampling (n = the fine grid) ---------------------
__global__ void avgpool_kernel(const __nv_bfloat16* __restrict__ X, int B, int n, int C,
                               __nv_bfloat16* __restrict__ P) {
    const int h = n / 2;
    const int64_t total = (int64_t)B * h * h * h * C;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = q / C;
        const int c = (int)(q - v * C);
        const int x = (int)(v % h), y = (int)((v / h) % h), z = (int)((v / ((int64_t)h * h)) % h);
        const int b = (int)(v / ((int64_t)h * h * h));
        float s = 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d)
            s += __bfloat162float(X[vox(b, 2 * z + (d >> 2), 2 * y + ((d >> 1) & 1), 2 * x + (d & 1), n) * C + c]);
        P[q] = __float2bfloat16_rn(0.125f * s);
    }
}

__global__ void avgpool_bwd_kernel(const float* __restrict__ dP, int B, int n, int C,
                                   float* __restrict__ dX, int accumulate) {
    const int h = n / 2;
    const int64_t total = (int64_t)B * n * n * n * C;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = q / C;
        const int c = (int)(q - v * C);
        const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)((v / ((int64_t)n * n)) % n);
        const int b = (int)(v / ((int64_t)n * n * n));
        const float g = 0.125f * dP[vox(b, z / 2, y / 2, x / 2, h) * C + c];
        dX[q] = accumulate ? dX[q] + g : g;
    }
}

// U[fine voxel][c_off + c] = X[coarse voxel][c] (U has row stride ldU)
__global__ void upsample_kernel(const __nv_bfloat16* __restrict__ X, int B, int n, int C,
                                __nv_bfloat16* __restrict__ U, int64_t ldU, int c_off) {
    const int h = n / 2;
    const int64_t total = (int64_t)B * n * n * n * C;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = q / C;
        const int c = (int)(q - v * C);
        const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)((v / ((int64_t)n * n)) % n);
        const int b = (int)(v / ((int64_t)n * n * n));
        U[v * ldU + c_off + c] = X[vox(b, z / 2, y / 2, x / 2, h) * C + c];
    }
}

// dX[coarse][c] = sum of the 8 fine children dU[child][c_off + c]
__global__ void upsample_bwd_kernel(const float* __restrict__ dU, int64_t ldU, int c_off, int B,
                                    int n, int C, float* __restrict__ dX) {
    const int h = n / 2;
    const int64_t total = (int64_t)B * h * h * h * C;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = q / C;
        const int c = (int)(q - v * C);
        const int x = (int)(v % h), y = (int)((v / h) % h), z = (int)((v / ((int64_t)h * h)) % h);
        const int b = (int)(v / ((int64_t)h * h * h));
        float s = 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d)
            s += dU[vox(b, 2 * z + (d >> 2), 2 * y + ((d >> 1) & 1), 2 * x + (d & 1), n) * ldU + c_off + c];
        dX[q] = s;
    }
}

// The same four operations, 8 channels per thread (16-byte accesses) and 32-bit indices,
// when C and the row strides are multiples of 8 and the totals fit in 31 bits.
__device__ __forceinline__ void voxel_of(int v, int n, int& b, int& z, int& y, int& x) {
    x = v % n;
    int r = v / n;
    y = r % n;
    r /= n;
    z = r % n;
    b = r / n;
}

__global__ void avgpool8_kernel(const __nv_bfloat16* __restrict__ X, int n, int C8, int total,
                                __nv_bfloat16* __restrict__ P) {
    const int h = n / 2;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int v = q / C8, cg = q - v * C8;
        int b, z, y, x;
        voxel_of(v, h, b, z, y, x);
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int src = ((b * n + 2 * z + (d >> 2)) * n + 2 * y + ((d >> 1) & 1)) * n + 2 * x + (d & 1);
            const uint4 w = *reinterpret_cast<const uint4*>(X + ((int64_t)src * C8 + cg) * 8);
            const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&w);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(h2[e]);
                s[2 * e] += f.x;
                s[2 * e + 1] += f.y;
            }
        }
        uint4 o;
        __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
        for (int e = 0; e < 4; ++e) o2[e] = __floats2bfloat162_rn(0.125f * s[2 * e], 0.125f * s[2 * e + 1]);
        *reinterpret_cast<uint4*>(P + (int64_t)q * 8) = o;
    }
}

__global__ void avgpool_bwd8_kernel(const float* __restrict__ dP, int n, int C8, int total,
                                    float* __restrict__ dX, int accumulate) {
    const int h = n / 2;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int v = q / C8, cg = q - v * C8;
        int b, z, y, x;
        voxel_of(v, n, b, z, y, x);
        const int src = ((b * h + z / 2) * h + y / 2) * h + x / 2;
        const float4* g = reinterpret_cast<const float4*>(dP + ((int64_t)src * C8 + cg) * 8);
        float4* d = reinterpret_cast<float4*>(dX + (int64_t)q * 8);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float4 a = g[e];
            a.x *= 0.125f, a.y *= 0.125f, a.z *= 0.125f, a.w *= 0.125f;
            if (accumulate) {
                const float4 o = d[e];
                a.x += o.x, a.y += o.y, a.z += o.z, a.w += o.w;
            }
            d[e] = a;
        }
    }
}

__global__ void upsample8_kernel(const __nv_bfloat16* __restrict__ X, int n, int C8, int total,
                                 __nv_bfloat16* __restrict__ U, int ldU, int c_off) {
    const int h = n / 2;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int v = q / C8, cg = q - v * C8;
        int b, z, y, x;
        voxel_of(v, n, b, z, y, x);
        const int src = ((b * h + z / 2) * h + y / 2) * h + x / 2;
        *reinterpret_cast<uint4*>(U + (int64_t)v * ldU + c_off + cg * 8) =
            *reinterpret_cast<const uint4*>(X + ((int64_t)src * C8 + cg) * 8);
    }
}

__global__ void upsample_bwd8_kernel(const float* __restrict__ dU, int ldU, int c_off, int n, int C8,
                                     int total, float* __restrict__ dX) {
    const int h = n / 2;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int v = q / C8, cg = q - v * C8;
        int b, z, y, x;
        voxel_of(v, h, b, z, y, x);
        float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int src = ((b * n + 2 * z + (d >> 2)) * n + 2 * y + ((d >> 1) & 1)) * n + 2 * x + (d & 1);
            const float4* g = reinterpret_cast<const float4*>(dU + (int64_t)src * ldU + c_off + cg * 8);
            const float4 a = g[0], c = g[1];
            s0.x += a.x, s0.y += a.y, s0.z += a.z, s0.w += a.w;
            s1.x += c.x, s1.y += c.y, s1.z += c.z, s1.w += c.w;
        }
        float4* d = reinterpret_cast<float4*>(dX + (int64_t)q * 8);
        d[0] = s0;
        d[1] = s1;
    }
}

static bool vec8_ok(int64_t total, int C, int64_t ld, int c_off, const void* a, const void* b) {
    return C % 8 == 0 && ld % 8 == 0 && c_off % 8 == 0 && total / 8 < (int64_t(1) << 31) &&
           ((uintptr_t)a & 15) == 0 && ((uintptr_t)b & 15) == 0;
}

cudaError_t avgpool(const __nv_bfloat16* X, int B, int n, int C, __nv_bfloat16* P, cudaStream_t st) {
    const int64_t total = (int64_t)B * (n / 2) * (n / 2) * (n / 2) * C;
    if (vec8_ok((int64_t)B * n * n * n * C, C, C, 0, X, P)) {
        avgpool8_kernel<<<blocks_for(total / 8, 256), 256, 0, st>>>(X, n, C / 8, (int)(total / 8), P);
        return cudaGetLastError();
    }
    avgpool_kernel<<<blocks_for(total, 256), 256, 0, st>>>(X, B, n, C, P);
    return cudaGetLastError();
}
cudaError_t avgpool_bwd(const float* dP, int B, int n, int C, float* dX, int accumulate, cudaStream_t st) {
    const int64_t total = (int64_t)B * n * n * n * C;
    if (vec8_ok(total, C, C, 0, dP, dX)) {
        avgpool_bwd8_kernel<<<blocks_for(total / 8, 256), 256, 0, st>>>(dP, n, C / 8, (int)(total / 8), dX,
                                                                         accumulate);
        return cudaGetLastError();
    }
    avgpool_bwd_kernel<<<blocks_for(total, 256), 256, 0, st>>>(dP, B, n, C, dX, accumulate);
    return cudaGetLastError();
}
cudaError_t upsample(const __nv_bfloat16* X, int B, int n, int C, __nv_bfloat16* U, int64_t ldU,
                     int c_off, cudaStream_t st) {
    const int64_t total = (int64_t)B * n * n * n * C;
    if (vec8_ok(total, C, ldU, c_off, X, U) && (int64_t)B * n * n * n * ldU < (int64_t(1) << 31)) {
        upsample8_kernel<<<blocks_for(total / 8, 256), 256, 0, st>>>(X, n, C / 8, (int)(total / 8), U, (int)ldU,
                                                                      c_off);
        return cudaGetLastError();
    }
    upsample_kernel<<<blocks_for(total, 256), 256, 0, st>>>(X, B, n, C, U, ldU, c_off);
    return cudaGetLastError();
}
cudaError_t upsample_bwd(const float* dU, int64_t ldU, int c_off, int B, int n, int C, float* dX,
                         cudaStream_t st) {
    const int64_t total = (int64_t)B * (n / 2) * (n / 2) * (n / 2) * C;
    if (vec8_ok((int64_t)B * n * n * n * C, C, ldU, c_off, dU, dX) && (int64_t)B * n * n * n * ldU < (int64_t(1) << 31)) {
        upsample_bwd8_kernel<<<blocks_for(total / 8, 256), 256, 0, st>>>(dU, (int)ldU, c_off, n, C / 8,
                                                                          (int)(total / 8), dX);
        return cudaGetLastError();
    }
    upsample_bwd_kernel<<<blocks_for(total, 256), 256, 0, st>>>(dU, ldU, c_off, B, n, C, dX);
    return cudaGetLastError();
}

// ---- channel slices (concatenation) -------------------------------------------------------
__global__ void copy_channels_kernel(const __nv_bfloat16* __restrict__ S, int64_t M, int C,
                                     __nv_bfloat16* __restrict__ D, int64_t ldD, int c_off) {
    const int64_t total = M * C;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = q / C;
        D[m * ldD + c_off + (q - m * C)] = S[q];
    }
}
// dS[m][c] (+)= dD[m][c_off + c]
__global__ void slice_grad_kernel(const float* __restrict__ dD, int64_t ldD, int c_off, int64_t M,
                                  int C, float* __restrict__ dS, int accumulate) {
    const int64_t total = M * C;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = q / C;
        const float g = dD[m * ldD + c_off + (q - m * C)];
        dS[q] = accumulate ? dS[q] + g : g;
    }
}
// 16-byte forms: 8 BF16 channels, 4 FP32 channels per thread (G groups per row, 32-bit indices).
__global__ void copy_channels8_kernel(const __nv_bfloat16* __restrict__ S, int total, int G,
                                      __nv_bfloat16* __restrict__ D, int ldD, int c_off) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int m = q / G, g = q - m * G;
        *reinterpret_cast<uint4*>(D + (int64_t)m * ldD + c_off + 8 * g) = reinterpret_cast<const uint4*>(S)[q];
    }
}
__global__ void slice_grad4_kernel(const float* __restrict__ dD, int ldD, int c_off, int total, int G,
                                   float* __restrict__ dS, int accumulate) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int m = q / G, g = q - m * G;
        float4 v = *reinterpret_cast<const float4*>(dD + (int64_t)m * ldD + c_off + 4 * g);
        if (accumulate) {
            const float4 o = reinterpret_cast<const float4*>(dS)[q];
            v = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
        }
        reinterpret_cast<float4*>(dS)[q] = v;
    }
}
cudaError_t copy_channels(const __nv_bfloat16* S, int64_t M, int C, __nv_bfloat16* D, int64_t ldD,
                          int c_off, cudaStream_t st) {
    if (C % 8 == 0 && ldD % 8 == 0 && c_off % 8 == 0 && ((uintptr_t)S & 15) == 0 && ((uintptr_t)D & 15) == 0 &&
        M * (C / 8) < (int64_t(1) << 30) && ldD < (int64_t(1) << 31)) {
        const int total = (int)(M * (C / 8));
        copy_channels8_kernel<<<blocks_for(total, 256), 256, 0, st>>>(S, total, C / 8, D, (int)ldD, c_off);
        return cudaGetLastError();
    }
    copy_channels_kernel<<<blocks_for(M * C, 256), 256, 0, st>>>(S, M, C, D, ldD, c_off);
    return cudaGetLastError();
}
cudaError_t slice_grad(const float* dD, int64_t ldD, int c_off, int64_t M, int C, float* dS,
                       int accumulate, cudaStream_t st) {
    if (C % 4 == 0 && ldD % 4 == 0 && c_off % 4 == 0 && ((uintptr_t)dD & 15) == 0 && ((uintptr_t)dS & 15) == 0 &&
        M * (C / 4) < (int64_t(1) << 30) && ldD < (int64_t(1) << 31)) {
        const int total = (int)(M * (C / 4));
        slice_grad4_kernel<<<blocks_for(total, 256), 256, 0, st>>>(dD, (int)ldD, c_off, total, C / 4, dS,
                                                                   accumulate);
        return cudaGetLastError();
    }
    slice_grad_kernel<<<blocks_for(M * C, 256), 256, 0, st>>>(dD, ldD, c_off, M, C, dS, accumulate);
    return cudaGetLastError();
}

// ---- the 1x1 output head (C -> 4, linear) ---------------------------------------------------
__global__ void head_kernel(const __nv_bfloat16* __restrict__ A, int64_t M, int C,
                            const float* __restrict__ W, const float* __restrict__ b,
                            float* __restrict__ out) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        float o[4] = {b[0], b[1], b[2], b[3]};
        for (int c = 0; c < C; ++c) {
            const float a = __bfloat162float(A[m * C + c]);
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j] += W[j * C + c] * a;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) out[m * 4 + j] = o[j];
    }
}

// The same with the row read in 16-byte chunks of 8 channels and W, b from shared memory
// (C a multiple of 8, at most 64); the channels are added in the same order.
__global__ void head8_kernel(const __nv_bfloat16* __restrict__ A, int M, int C,
                             const float* __restrict__ W, const float* __restrict__ b,
                             float* __restrict__ out) {
    __shared__ float w[4 * 64 + 4];
    for (int i = threadIdx.x; i < 4 * C; i += blockDim.x) w[i] = W[i];
    if (threadIdx.x < 4) w[4 * C + threadIdx.x] = b[threadIdx.x];
    __syncthreads();
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        float o[4] = {w[4 * C], w[4 * C + 1], w[4 * C + 2], w[4 * C + 3]};
        const uint4* row = reinterpret_cast<const uint4*>(A + (int64_t)m * C);
        for (int g = 0; g < C / 8; ++g) {
            const uint4 v = row[g];
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 a = __bfloat1622float2(h[k]);
                const int c = 8 * g + 2 * k;
#pragma unroll
                for (int j = 0; j < 4; ++j) o[j] += w[j * C + c] * a.x;
#pragma unroll
                for (int j = 0; j < 4; ++j) o[j] += w[j * C + c + 1] * a.y;
            }
        }
        reinterpret_cast<float4*>(out)[m] = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// dA[m][c] = sum_j dOut[m][j] W[j][c] (one thread per row).
__global__ void head_dA_kernel(const float* __restrict__ dOut, int64_t M, int C,
                               const float* __restrict__ W, float* __restrict__ dA) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        const float g[4] = {dOut[m * 4], dOut[m * 4 + 1], dOut[m * 4 + 2], dOut[m * 4 + 3]};
        for (int c = 0; c < C; ++c) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) s += g[j] * W[j * C + c];
            dA[m * C + c] = s;
        }
    }
}

// Per-block sums over the block's rows, in row order: entry i < 4C is dW[j][c] (i = j C + c)
// += dOut[m][j] A[m][c], entries 4C .. 4C+3 are db[j] += dOut[m][j].  C <= 64.
__global__ void head_dW_kernel(const float* __restrict__ dOut, const __nv_bfloat16* __restrict__ A,
                               int64_t M, int C, int64_t rows, float* __restrict__ part) {
    const int E = 4 * C + 4;
    const int64_t m0 = (int64_t)blockIdx.x * rows, m1 = m0 + rows < M ? m0 + rows : M;
    for (int i = threadIdx.x; i < E; i += blockDim.x) {
        const int j = i < 4 * C ? i / C : i - 4 * C;
        const int c = i < 4 * C ? i % C : -1;
        float s = 0.f;
        for (int64_t m = m0; m < m1; ++m)
            s += c >= 0 ? dOut[m * 4 + j] * __bfloat162float(A[m * C + c]) : dOut[m * 4 + j];
        part[(int64_t)blockIdx.x * E + i] = s;
    }
}

cudaError_t head_fwd(const __nv_bfloat16* A, int64_t M, int C, const float* W, const float* b,
                     float* out, cudaStream_t st) {
    if (C % 8 == 0 && C <= 64 && M < (int64_t(1) << 30) && ((uintptr_t)A & 15) == 0 && ((uintptr_t)out & 15) == 0) {
        head8_kernel<<<blocks_for(M, 256), 256, 0, st>>>(A, (int)M, C, W, b, out);
        return cudaGetLastError();
    }
    head_kernel<<<blocks_for(M, 256), 256, 0, st>>>(A, M, C, W, b, out);
    return cudaGetLastError();
}
// The same 4 channels per thread: G = C / 4 threads per row, one 16-byte store each.
__global__ void head_dA4_kernel(const float* __restrict__ dOut, int total, int G,
                                const float* __restrict__ W, float* __restrict__ dA) {
    __shared__ float w[4 * 64];
    const int C = 4 * G;
    for (int i = threadIdx.x; i < 4 * C; i += blockDim.x) w[i] = W[i];
    __syncthreads();
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int m = q / G, c = 4 * (q - m * G);
        const float4 g = reinterpret_cast<const float4*>(dOut)[m];
        float4 o;
        o.x = g.x * w[c] + g.y * w[C + c] + g.z * w[2 * C + c] + g.w * w[3 * C + c];
        o.y = g.x * w[c + 1] + g.y * w[C + c + 1] + g.z * w[2 * C + c + 1] + g.w * w[3 * C + c + 1];
        o.z = g.x * w[c + 2] + g.y * w[C + c + 2] + g.z * w[2 * C + c + 2] + g.w * w[3 * C + c + 2];
        o.w = g.x * w[c + 3] + g.y * w[C + c + 3] + g.z * w[2 * C + c + 3] + g.w * w[3 * C + c + 3];
        reinterpret_cast<float4*>(dA)[q] = o;
    }
}

// The head's weight and bias gradients with 8 channels per thread: thread t takes the
// channel group g = t % G (G = C / 8) and every R-th row of the block (R = 256 / G lanes),
// keeping 32 sums dOut[m][j] A[m][8 g + i] (and, in group 0, the 4 sums of dOut[m][j]);
// the lanes are then added in lane order into the same per-block entries as head_dW_kernel.
__global__ void head_dW8_kernel(const float* __restrict__ dOut, const __nv_bfloat16* __restrict__ A,
                                int M, int C, int rows, float* __restrict__ part) {
    __shared__ float acc[256][37];
    const int G = C >> 3, R = 256 / G;
    const int g = threadIdx.x % G, r = threadIdx.x / G;
    const int m0 = blockIdx.x * rows, m1 = min(m0 + rows, M);
    float s[36];
#pragma unroll
    for (int i = 0; i < 36; ++i) s[i] = 0.f;
    if (r < R) {
        for (int m = m0 + r; m < m1; m += R) {
            const float4 d = reinterpret_cast<const float4*>(dOut)[m];
            const uint4 a = *reinterpret_cast<const uint4*>(A + (int64_t)m * C + 8 * g);
            const __nv_bfloat162* ah = reinterpret_cast<const __nv_bfloat162*>(&a);
            const float dj[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 af = __bfloat1622float2(ah[k]);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    s[j * 8 + 2 * k] += dj[j] * af.x;
                    s[j * 8 + 2 * k + 1] += dj[j] * af.y;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) s[32 + j] += dj[j];
        }
    }
#pragma unroll
    for (int i = 0; i < 36; ++i) acc[threadIdx.x][i] = s[i];
    __syncthreads();
    const int E = 4 * C + 4;
    for (int i = threadIdx.x; i < E; i += blockDim.x) {
        int gi, slot;
        if (i < 4 * C) {
            const int j = i / C, c = i - j * C;
            gi = c >> 3;
            slot = j * 8 + (c & 7);
        } else {
            gi = 0;
            slot = 32 + (i - 4 * C);
        }
        float t = 0.f;
        for (int l = 0; l < R; ++l) t += acc[l * G + gi][slot];
        part[(int64_t)blockIdx.x * E + i] = t;
    }
}

cudaError_t head_bwd(const float* dOut, const __nv_bfloat16* A, int64_t M, int C, const float* W,
                     float* dA, float* dW, float* db, float* part, cudaStream_t st) {
    if (C < 1 || C > 64 || M < 1) return cudaErrorInvalidValue;
    if (C % 8 == 0 && M * (C / 4) < (int64_t(1) << 30) && ((uintptr_t)dOut & 15) == 0 && ((uintptr_t)A & 15) == 0 &&
        ((uintptr_t)dA & 15) == 0) {
        const int total = (int)(M * (C / 4));
        head_dA4_kernel<<<blocks_for(total, 256), 256, 0, st>>>(dOut, total, C / 4, W, dA);
        const int64_t rows = rows_per_block(M, 256 / (C / 8), kMaxPartialBlocks);
        const int nblocks = (int)((M + rows - 1) / rows);
        const int E = 4 * C + 4;
        head_dW8_kernel<<<nblocks, 256, 0, st>>>(dOut, A, (int)M, C, (int)rows, part);
        sum_partials(part, nblocks, E, 0, 4 * C, dW, st);
        sum_partials(part, nblocks, E, 4 * C, 4, db, st);
        return cudaGetLastError();
    }
    unsigned blocks = blocks_for(M, 256);
    if (blocks > 2048) blocks = 2048;
    head_dA_kernel<<<blocks, 256, 0, st>>>(dOut, M, C, W, dA);
    const int64_t rows = rows_per_block(M, 64, kMaxPartialBlocks);
    const int nblocks = (int)((M + rows - 1) / rows);
    const int E = 4 * C + 4;
    head_dW_kernel<<<nblocks, 256, 0, st>>>(dOut, A, M, C, rows, part);
    sum_partials(part, nblocks, E, 0, 4 * C, dW, st);
    sum_partials(part, nblocks, E, 4 * C, 4, db, st);
    return cudaGetLastError();
}

// ---- loss: mean squared error over all outputs ------------------------------------------------
// dOut = 2 (out - target) / count; the per-block sums of (out - target)^2 / count go to
// part[block] and are added to *loss in block order.
__global__ void mse_kernel(const float* __restrict__ out, const float* __restrict__ target,
                           int64_t count, float* __restrict__ dOut, double* __restrict__ part) {
    __shared__ double red[8];
    double s = 0.0;
    const double inv = 1.0 / (double)count;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x) {
        const float d = out[q] - target[q];
        dOut[q] = (float)(2.0 * inv) * d;
        s += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) part[blockIdx.x] = v * inv;
    }
}

// *loss = the sum of the block partials, in the fixed order of sum_partials_kernel (FP64).
__global__ void __launch_bounds__(256) sum_loss_kernel(const double* __restrict__ part, int nblocks,
                                                       double* __restrict__ loss) {
    __shared__ double red[256];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int b = t; b < nblocks; b += 256) s += part[b];
    red[t] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) *loss = red[0];
}

cudaError_t mse(const float* out, const float* target, int64_t count, float* dOut, double* loss,
                double* part, cudaStream_t st) {
    unsigned blocks = blocks_for(count, 256);
    if (blocks > (unsigned)kMaxPartialBlocks) blocks = kMaxPartialBlocks;
    mse_kernel<<<blocks, 256, 0, st>>>(out, target, count, dOut, part);
    sum_loss_kernel<<<1, 256, 0, st>>>(part, (int)blocks, loss);
    return cudaGetLastError();
}

// ---- Adam (Kingma & Ba 2015) on FP32 master values ------------------------------------------
// One launch for every parameter tensor: blockIdx.y selects the tensor.
__global__ void adam_kernel(const __grid_constant__ AdamTable t, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    const AdamSeg& sg = t.seg[blockIdx.y];
    float* __restrict__ p = sg.p;
    const float* __restrict__ g = sg.g;
    float* __restrict__ m = sg.m;
    float* __restrict__ v = sg.v;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sg.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Blocks per tensor: every tensor's elements in at most 4 grid-stride passes.
static unsigned blocks_per_seg(int64_t max_n) {
    const int64_t b = (max_n + 4 * 256 - 1) / (4 * 256);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 4096));
}

cudaError_t adam(const AdamTable& t, float lr, float b1, float b2, float eps, int step, cudaStream_t st) {
    if (t.count < 1 || t.count > kMaxSegs) return cudaErrorInvalidValue;
    int64_t max_n = 0;
    for (int i = 0; i < t.count; ++i) max_n = std::max(max_n, t.seg[i].n);
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<dim3(blocks_per_seg(max_n), t.count), 256, 0, st>>>(t, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

// ---- weights -----------------------------------------------------------------------------------
// W [cout][27 cin] FP32 -> Wb [cout][Kp] BF16 with K index tap * cs + ci for an input stored
// with cs >= cin channels (zero for ci >= cin and in the K padding), the forward operand, and
// Wf [cin][Kpf] BF16 with Wf[ci][t * cout + co] = W[co][(26 - t) * cin + ci]: the weights of
// the convolution that maps the output gradient to the input gradient (every tap
// mirrored, input and output channels exchanged; zero padding to Kpf).  One launch for
// every layer: blockIdx.y selects the layer.
__global__ void pack_weights_kernel(const __grid_constant__ PackTable t) {
    const PackSeg& sg = t.seg[blockIdx.y];
    const float* __restrict__ W = sg.W;
    const int cin = sg.cin, cs = sg.cs, cout = sg.cout, Kp = sg.Kp, Kpf = sg.Kpf;
    const int K27 = 27 * cin;
    const int64_t n1 = (int64_t)cout * Kp, n2 = sg.Wf ? (int64_t)cin * Kpf : 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n1 + n2;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (q < n1) {
            const int co = (int)(q / Kp), k = (int)(q % Kp);
            const int tap = k / cs, ci = k - tap * cs;
            sg.Wb[q] = __float2bfloat16_rn(tap < 27 && ci < cin ? W[(int64_t)co * K27 + tap * cin + ci] : 0.f);
        } else {
            const int64_t r = q - n1;
            const int ci = (int)(r / Kpf), k = (int)(r % Kpf);
            float w = 0.f;
            if (k < 27 * cout) {
                const int tt = k / cout, co = k % cout;
                w = W[(int64_t)co * K27 + (26 - tt) * cin + ci];
            }
            sg.Wf[r] = __float2bfloat16_rn(w);
        }
    }
}
cudaError_t pack_weights(const PackTable& t, cudaStream_t st) {
    if (t.count < 1 || t.count > kMaxSegs) return cudaErrorInvalidValue;
    int64_t max_n = 0;
    for (int i = 0; i < t.count; ++i) {
        const PackSeg& sg = t.seg[i];
        if (sg.cs < sg.cin || sg.Kp < 27 * sg.cs || (sg.Wf && sg.Kpf < 27 * sg.cout)) return cudaErrorInvalidValue;
        max_n = std::max(max_n, (int64_t)sg.cout * sg.Kp + (sg.Wf ? (int64_t)sg.cin * sg.Kpf : 0));
    }
    pack_weights_kernel<<<dim3(blocks_per_seg(max_n), t.count), 256, 0, st>>>(t);
    return cudaGetLastError();
}

// dWT [Kp][cout] (K index tap * cs + ci) -> gW [cout][27 cin], every layer in one launch.
__global__ void unpack_grad_kernel(const __grid_constant__ UnpackTable t) {
    const UnpackSeg& sg = t.seg[blockIdx.y];
    const int cout = sg.cout, cin = sg.cin, cs = sg.cs;
    const int K27 = 27 * cin;
    const int64_t total = (int64_t)cout * K27;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int co = (int)(q / K27), k = (int)(q % K27);
        const int tap = k / cin, ci = k - tap * cin;
        sg.gW[q] = sg.dWT[(int64_t)(tap * cs + ci) * cout + co];
    }
}
cudaError_t unpack_grad(const UnpackTable& t, cudaStream_t st) {
    if (t.count < 1 || t.count > kMaxSegs) return cudaErrorInvalidValue;
    int64_t max_n = 0;
    for (int i = 0; i < t.count; ++i) max_n = std::max(max_n, (int64_t)t.seg[i].cout * 27 * t.seg[i].cin);
    unpack_grad_kernel<<<dim3(blocks_per_seg(max_n), t.count), 256, 0, st>>>(t);
    return cudaGetLastError();
}

// ---- input features ----------------------------------------------------------------------------
// channel 0: distance to the nearest wall / n (half-way walls: node i is i + 1/2 from the
// low wall); 1: heated-face mask (+1 on the hot layer x = n-1, -1 on the cold layer x = 0);
// 2, 3: the sample's normalised log10 Ra and log10 Pr; channels 4 .. ldx - 1 zero (the
// stored row is padded so that the first convolution reads it like any other layer's input).
__global__ void features_kernel(int B, int n, const float* __restrict__ scalars, int ldx,
                                __nv_bfloat16* __restrict__ X) {
    const int64_t total = (int64_t)B * n * n * n;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < total;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)((v / ((int64_t)n * n)) % n);
        const int b = (int)(v / ((int64_t)n * n * n));
        float d = fminf(x + 0.5f, n - 0.5f - x);
        d = fminf(d, fminf(y + 0.5f, n - 0.5f - y));
        d = fminf(d, fminf(z + 0.5f, n - 0.5f - z));
        const float mask = x == n - 1 ? 1.f : (x == 0 ? -1.f : 0.f);
        const __nv_bfloat162 f01 = __floats2bfloat162_rn(d / n, n == 1 ? 0.f : mask);
        const __nv_bfloat162 f23 = __floats2bfloat162_rn(scalars[2 * b], scalars[2 * b + 1]);
        uint4* row = reinterpret_cast<uint4*>(X + v * ldx);
        row[0] = make_uint4(*reinterpret_cast<const uint32_t*>(&f01), *reinterpret_cast<const uint32_t*>(&f23), 0u, 0u);
        for (int j = 1; j < ldx / 8; ++j) row[j] = make_uint4(0u, 0u, 0u, 0u);
    }
}
cudaError_t features(int B, int n, const float* scalars, __nv_bfloat16* X, int ldx, cudaStream_t st) {
    if (ldx < 8 || ldx % 8 || ((uintptr_t)X & 15)) return cudaErrorInvalidValue;
    features_kernel<<<blocks_for((int64_t)B * n * n * n, 256), 256, 0, st>>>(B, n, scalars, ldx, X);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace lbm
