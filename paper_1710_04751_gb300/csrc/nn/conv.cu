// conv.cu -- 3x3x3 convolutions with zero padding as implicit GEMMs on the tcgen05 tensor
// cores:
//   Y[m][co] = sum_{tap, ci} X[m shifted by tap][ci] * W[co][tap * cin + ci]
// for activations X [B][n][n][n][cin] (BF16, channels last, voxel m = ((b n + z) n + y) n + x)
// and W [cout][Kp] (K index tap * cin + ci, tap = (kz 3 + ky) 3 + kx reading the input at
// (z + kz - 1, y + ky - 1, x + kx - 1)).  No im2col matrix goes through HBM: the A operand of
// the K block (tap, channel chunk) is loaded straight from X by one 5D TMA box
//   {BKC channels, bx, by, bz, bb} at (c0, x0 + kx - 1, y0 + ky - 1, z0 + kz - 1, b0),
// the 128 voxels of the M tile (bx by bz bb = 128, whole x-rows) seen through the tap's
// shift; the box's out-of-range part -- the zero padding -- arrives as zeros (TMA fill).
// The box lands in shared memory exactly as the 2D box of an im2col matrix would (rows of
// BKC channels, 128-byte swizzle for 64 channels, 64-byte swizzle for 32), so the MMA side
// is the GEMM's: one CTA of 128 threads per 128 x BN tile, warp 0 lane 0 producing into a
// 4-stage mbarrier ring, warp 1 lane 0 issuing tcgen05.mma into TMEM, all four warps
// draining the accumulator.  Epilogues: bias + ReLU + BF16 (the forward pass) or FP32 (the
// input gradient, the convolution of the output gradient with the mirrored weights).
// Every wait is bounded as in gemm.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "nn.h"
#include "tc.cuh"

namespace lbm {
namespace nn {

namespace {

constexpr int CBM = 128, CSTAGES = 4;

template <int BN, int BKC>
struct ConvSmem {
    static constexpr int A_BYTES = CBM * BKC * 2;
    static constexpr int B_BYTES = BN * BKC * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int BYTES = 1024 + CSTAGES * STAGE + 256;
    static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
};

struct ConvArgs {
    int M, N;               // output rows (B n^3) and columns (cout)
    int n;                  // grid edge
    int chunks;             // channel chunks of BKC per tap (cin / BKC)
    int bx, by, bz;         // the M tile as a box of the grid (with bb = 128 / (bx by bz))
    int mode;               // CONV_BIAS_RELU_BF16 or CONV_F32
    void* C;                // output [M][N]
    const float* bias;      // bias[N] (CONV_BIAS_RELU_BF16)
    int* err;
};

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, int bkc) {
    return bkc == 64 ? sdesc_k_sw128(saddr) : sdesc_k_sw64(saddr);
}

template <int BN, int BKC>
__global__ void __launch_bounds__(128, 1)
    conv_bf16_kernel(const __grid_constant__ CUtensorMap tmX,
                     const __grid_constant__ CUtensorMap tmW, ConvArgs args) {
    using L = ConvSmem<BN, BKC>;
    extern __shared__ uint8_t conv_smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(conv_smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + CSTAGES * L::STAGE);
    uint64_t* empty = full + CSTAGES;
    uint64_t* done = empty + CSTAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ volatile int failed;

    if (*static_cast<volatile int*>(args.err) != 0) return;  // another CTA timed out
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * CBM, n0 = blockIdx.y * BN;
    const int nkb = 27 * args.chunks;

    if (threadIdx.x == 0) {
        failed = 0;
        for (int s = 0; s < CSTAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, L::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    int issued = 0;
    if (warp == 0 && lane == 0) {
        // the tile's first voxel (its x0 is 0 unless a row holds several tiles)
        const int n = args.n;
        const int x0 = m0 % n, y0 = (m0 / n) % n, z0 = (m0 / (n * n)) % n, b0 = m0 / (n * n * n);
        int tap = 0, chunk = 0;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % CSTAGES;
            const uint32_t ph = (uint32_t)(i / CSTAGES) & 1u;
            if (i >= CSTAGES && !mbar_wait(empty + s, ph ^ 1u, args.err, 1, &failed)) {
                failed = 1;
                break;
            }
            if (failed) break;
            uint8_t* a = smem + s * L::STAGE;
            const int kz = tap / 9, ky = (tap / 3) % 3, kx = tap % 3;
            mbar_expect_tx(full + s, L::STAGE);
            tma_load_5d(a, &tmX, full + s, chunk * BKC, x0 + kx - 1, y0 + ky - 1, z0 + kz - 1, b0);
            tma_load_2d(a + L::A_BYTES, &tmW, full + s, i * BKC, n0);
            ++issued;
            if (++chunk == args.chunks) {
                chunk = 0;
                ++tap;
            }
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16_f32(CBM, BN);
        for (int i = 0; i < nkb; ++i) {
            const int s = i % CSTAGES;
            const uint32_t ph = (uint32_t)(i / CSTAGES) & 1u;
            if (failed || !mbar_wait(full + s, ph, args.err, 2, &failed)) {
                failed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a = smem_u32(smem + s * L::STAGE), b = a + L::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BKC / 16; ++kk)
                mma_bf16(tmem, sdesc(a + kk * 32, BKC), sdesc(b + kk * 32, BKC), idesc,
                         (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(empty + s);
        }
        mma_commit(done);  // also when stopped early: every issued MMA drains before dealloc
    }
    __syncwarp();
    if (!mbar_wait(done, 0, args.err, 3)) failed = 1;
    __syncthreads();
    const bool ok = !failed;
    if (warp == 0 && lane == 0 && failed) {  // let every started copy land
        for (int i = max(0, issued - CSTAGES); i < issued; ++i)
            mbar_wait(full + (i % CSTAGES), (uint32_t)(i / CSTAGES) & 1u, args.err, 4);
    }
    tc_fence_after();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            const int col0 = n0 + c;
            if (row >= args.M || col0 >= args.N) continue;
            const bool whole = col0 + 16 <= args.N && (args.N % 8) == 0;  // 16-byte stores
            if (args.mode == CONV_BIAS_RELU_BF16) {
                __nv_bfloat16* C = static_cast<__nv_bfloat16*>(args.C) + (int64_t)row * args.N;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    v[j] = fmaxf(v[j] + (col0 + j < args.N ? args.bias[col0 + j] : 0.f), 0.f);
                if (whole) {
                    uint4 pk[2];
                    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(pk);
#pragma unroll
                    for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                    reinterpret_cast<uint4*>(C + col0)[0] = pk[0];
                    reinterpret_cast<uint4*>(C + col0)[1] = pk[1];
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (col0 + j < args.N) C[col0 + j] = __float2bfloat16_rn(v[j]);
                }
            } else {
                float* C = static_cast<float*>(args.C) + (int64_t)row * args.N;
                if (whole && (args.N % 4) == 0) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        reinterpret_cast<float4*>(C + col0)[j] =
                            make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (col0 + j < args.N) C[col0 + j] = v[j];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, L::TMEM_COLS);
}

// ---------------------------------------------------------------------------------
// The same convolution with the input tile reused across the three ky taps (n >= 16).
// A CTA computes MT consecutive M tiles (MT * 128 voxels: bx = n columns by MT * by rows of
// one plane).  For each (kz, kx, channel chunk) one 5D box brings the MT * by + 2 rows
// around them, shifted by kx - 1 in x and kz - 1 in z; the tile of output tile t and tap
// ky is the 128-row window starting at row (t * by + ky) * bx of that box (whole x-rows,
// so every window starts on a swizzle atom), multiplied into accumulator t with the
// weights of tap (kz, ky, kx).  Each loaded byte serves up to 3 * MT * by / (MT * by + 2)
// windows instead of one (2.4 at n = 64, MT = 4), cutting the operand traffic from L2 that
// bounds the one-tile kernel.  Stage geometry is a runtime property of n and MT.
// ---------------------------------------------------------------------------------
struct RowsArgs {
    int M, N, n, chunks, cin;
    int bx, by, mt;      // tile columns, rows per tile, tiles per CTA
    int a_bytes;         // one stage's input box: (mt by + 2) bx BKC 2 bytes
    int stage_bytes;     // a_bytes + 3 BN BKC 2, rounded up to 1024
    int stages;
    uint32_t tmem_cols;  // mt BN, a power of two >= 32
    int mode;
    void* C;
    const float* bias;
    int* err;
};

template <int BN, int BKC>
__global__ void __launch_bounds__(128, 1)
    conv_rows_kernel(const __grid_constant__ CUtensorMap tmX,
                     const __grid_constant__ CUtensorMap tmW, RowsArgs args) {
    extern __shared__ uint8_t rows_smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(rows_smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = args.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * args.stage_bytes);
    uint64_t* empty = full + S;
    uint64_t* done = empty + S;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ volatile int failed;
    constexpr int B_TILE = BN * BKC * 2;

    if (*static_cast<volatile int*>(args.err) != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int MT = args.mt;
    const int m0 = blockIdx.x * MT * CBM, n0 = blockIdx.y * BN;
    const int nkb = 9 * args.chunks;  // stages: (kz, kx, chunk)

    if (threadIdx.x == 0) {
        failed = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, args.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    int issued = 0;
    if (warp == 0 && lane == 0) {
        const int n = args.n;
        const int y0 = (m0 / n) % n, z0 = (m0 / (n * n)) % n, b0 = m0 / (n * n * n);
        int kz = 0, kx = 0, chunk = 0;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % S;
            const uint32_t ph = (uint32_t)(i / S) & 1u;
            if (i >= S && !mbar_wait(empty + s, ph ^ 1u, args.err, 1, &failed)) {
                failed = 1;
                break;
            }
            if (failed) break;
            uint8_t* a = smem + s * args.stage_bytes;
            mbar_expect_tx(full + s, (uint32_t)(args.a_bytes + 3 * B_TILE));
            tma_load_5d(a, &tmX, full + s, chunk * BKC, kx - 1, y0 - 1, z0 + kz - 1, b0);
            for (int ky = 0; ky < 3; ++ky) {
                const int tap = (kz * 3 + ky) * 3 + kx;
                tma_load_2d(a + args.a_bytes + ky * B_TILE, &tmW, full + s,
                            (tap * args.chunks + chunk) * BKC, n0);
            }
            ++issued;
            if (++chunk == args.chunks) {
                chunk = 0;
                if (++kx == 3) {
                    kx = 0;
                    ++kz;
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16_f32(CBM, BN);
        const int row_bytes = BKC * 2;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % S;
            const uint32_t ph = (uint32_t)(i / S) & 1u;
            if (failed || !mbar_wait(full + s, ph, args.err, 2, &failed)) {
                failed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a = smem_u32(smem + s * args.stage_bytes), b = a + args.a_bytes;
            for (int t = 0; t < MT; ++t) {
                for (int ky = 0; ky < 3; ++ky) {
                    const uint32_t at = a + (uint32_t)((t * args.by + ky) * args.bx * row_bytes);
                    const uint32_t bt = b + (uint32_t)(ky * B_TILE);
#pragma unroll
                    for (int kk = 0; kk < BKC / 16; ++kk)
                        mma_bf16(tmem + (uint32_t)(t * BN), sdesc(at + kk * 32, BKC),
                                 sdesc(bt + kk * 32, BKC), idesc, (i > 0 || ky > 0 || kk > 0) ? 1u : 0u);
                }
            }
            mma_commit(empty + s);
        }
        mma_commit(done);
    }
    __syncwarp();
    if (!mbar_wait(done, 0, args.err, 3)) failed = 1;
    __syncthreads();
    const bool ok = !failed;
    if (warp == 0 && lane == 0 && failed) {
        for (int i = max(0, issued - S); i < issued; ++i)
            mbar_wait(full + (i % S), (uint32_t)(i / S) & 1u, args.err, 4);
    }
    tc_fence_after();
    if (ok) {
        for (int t = 0; t < MT; ++t) {
            const int row = m0 + t * CBM + warp * 32 + lane;
#pragma unroll 1
            for (int c = 0; c < BN; c += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * BN + c), v);
                const int col0 = n0 + c;
                if (row >= args.M || col0 >= args.N) continue;
                const bool whole = col0 + 16 <= args.N && (args.N % 8) == 0;
                if (args.mode == CONV_BIAS_RELU_BF16) {
                    __nv_bfloat16* C = static_cast<__nv_bfloat16*>(args.C) + (int64_t)row * args.N;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        v[j] = fmaxf(v[j] + (col0 + j < args.N ? args.bias[col0 + j] : 0.f), 0.f);
                    if (whole) {
                        uint4 pk[2];
                        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(pk);
#pragma unroll
                        for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        reinterpret_cast<uint4*>(C + col0)[0] = pk[0];
                        reinterpret_cast<uint4*>(C + col0)[1] = pk[1];
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (col0 + j < args.N) C[col0 + j] = __float2bfloat16_rn(v[j]);
                    }
                } else {
                    float* C = static_cast<float*>(args.C) + (int64_t)row * args.N;
                    if (whole && (args.N % 4) == 0) {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            reinterpret_cast<float4*>(C + col0)[j] =
                                make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (col0 + j < args.N) C[col0 + j] = v[j];
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, args.tmem_cols);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// X [B][n][n][n][cin] as a 5D tensor (innermost first) read in boxes of
// {bkc, bx, by, bz, bb}; out-of-range elements read as zeros.
bool make_x_map(CUtensorMap* map, const void* X, int B, int n, int cin, int bkc, int bx, int by,
                int bz, int bb) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[5] = {(cuuint64_t)cin, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n,
                                (cuuint64_t)B};
    const cuuint64_t row = (cuuint64_t)cin * 2;
    const cuuint64_t strides[4] = {row, row * n, row * n * n, row * n * n * n};
    const cuuint32_t box[5] = {(cuuint32_t)bkc, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz,
                               (cuuint32_t)bb};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(X), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              bkc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// W [N][Kp] (row stride ld) read in boxes of bkc x box_rows.
bool make_w_map(CUtensorMap* map, const void* W, int N, int K, long long ld, int bkc, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)bkc, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(W), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              bkc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------------
// Weight gradient as an implicit GEMM on both operands in their natural layouts:
//   dW^T[r][co] = sum over voxels v of X[v + shift(tap)][ci] dZ[v][co],  r = tap cin + ci,
// a contraction over the voxels, so both operands are MN-major for the tensor core (the
// row index r of A and the column index co of B are the contiguous ones in memory) and
// neither X nor dZ is transposed or expanded.  K block = 64 consecutive voxels, the box
// {bx, by, bz, bb} of the grid with bx by bz bb = 64 (x-row segments for n >= 64, whole
// rows, planes or samples below).  A operand of the M tile (128 rows = four (tap,
// 32-channel) groups): four 5D TMA boxes {32 channels, bx, by, bz, bb} of X at
// (ci0, x0 + kx - 1, y0 + ky - 1, z0 + kz - 1, b0) with the 64-byte swizzle, each landing
// as 64 K rows of 32 channels (64 bytes): the canonical MN-major tile, swizzle atoms of 8
// K rows 512 bytes apart, the four channel groups 4 KB apart.  The tap's shift and the
// zero padding come from the box coordinates and TMA's zero fill; the innermost
// coordinate stays a multiple of 32 channels.  B operand: dZ [voxels][cout] in boxes
// {BB channels, 64 voxels} (BB = 64 with the 128-byte swizzle, 32 with the 64-byte one
// when BN = 32), BN / BB of them B_GROUP bytes apart.  Split K over the voxels: split z
// stores its partial tile in slice z of the workspace; the slices are added in order
// afterwards.
// ---------------------------------------------------------------------------------
constexpr int WG_STAGES = 4;

template <int BN>
struct WgradSmem {
    static constexpr int A_BYTES = CBM * 64 * 2, B_BYTES = BN * 64 * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    // 2 KB past the ring: the operand reads of the last stage stay inside the allocation
    // under either assignment of the two descriptor strides
    static constexpr int BYTES = 1024 + WG_STAGES * STAGE + 2048 + 256;
    static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
    static constexpr int BB = BN < 64 ? BN : 64;         // output channels per B box
    static constexpr uint32_t B_GROUP = BB * 2 * 64;     // bytes of one B box (64 K rows)
    static constexpr uint32_t B_ATOM = BB * 2 * 8;       // bytes of 8 K rows of it
    static constexpr uint32_t B_LAYOUT = BB == 64 ? 2u : 4u;
};

struct WgradArgs {
    int rows;            // 27 cin (rows beyond it, up to the padded count, read as zeros)
    int N;               // cout
    int cin, ln;         // input channels, log2 of the grid edge
    int kblocks;         // 64-voxel blocks in all (ceil(B n^3 / 64))
    int kb_per_split;
    int Mrows;           // rows of a workspace slice (the padded 27 cin)
    float* ws;           // [splits][Mrows][N]
    int* err;
};

template <int BN>
__global__ void __launch_bounds__(128, 1)
    conv_wgrad_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB,
                      WgradArgs args) {
    using L = WgradSmem<BN>;
    extern __shared__ uint8_t wg_smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(wg_smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + WG_STAGES * L::STAGE + 2048);
    uint64_t* empty = full + WG_STAGES;
    uint64_t* done = empty + WG_STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ volatile int failed;

    if (*static_cast<volatile int*>(args.err) != 0) return;  // another CTA timed out
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * CBM, n0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * args.kb_per_split;
    const int nkb = min(args.kb_per_split, args.kblocks - kb0);

    if (threadIdx.x == 0) {
        failed = 0;
        for (int s = 0; s < WG_STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, L::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    int issued = 0;
    if (nkb > 0 && warp == 0 && lane == 0) {
        const int ln = args.ln, mask = (1 << ln) - 1;
        // the (tap, channel) groups of the M tile do not change along K
        int gx[4], gy[4], gz[4], gc[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int r = m0 + 32 * g;
            gx[g] = 0, gy[g] = 0, gz[g] = 0, gc[g] = args.cin;  // padding rows: past the channels
            if (r < args.rows) {
                const int tap = r / args.cin;
                gc[g] = r - tap * args.cin;
                gx[g] = tap % 3 - 1;
                gy[g] = (tap / 3) % 3 - 1;
                gz[g] = tap / 9 - 1;
            }
        }
        for (int i = 0; i < nkb; ++i) {
            const int s = i % WG_STAGES;
            const uint32_t ph = (uint32_t)(i / WG_STAGES) & 1u;
            if (i >= WG_STAGES && !mbar_wait(empty + s, ph ^ 1u, args.err, 1, &failed)) {
                failed = 1;
                break;
            }
            if (failed) break;
            uint8_t* a = smem + s * L::STAGE;
            mbar_expect_tx(full + s, L::STAGE);
            const int v0 = (kb0 + i) << 6;
            const int x0 = v0 & mask, y0 = (v0 >> ln) & mask, z0 = (v0 >> (2 * ln)) & mask, b0 = v0 >> (3 * ln);
#pragma unroll
            for (int g = 0; g < 4; ++g)
                tma_load_5d(a + g * 4096, &tmX, full + s, gc[g], x0 + gx[g], y0 + gy[g], z0 + gz[g], b0);
#pragma unroll
            for (int j = 0; j < BN / L::BB; ++j)
                tma_load_2d(a + L::A_BYTES + j * L::B_GROUP, &tmB, full + s, n0 + j * L::BB, v0);
            ++issued;
        }
    } else if (nkb > 0 && warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16_f32_mn(CBM, BN);
        // with one B box the leading offset is never used: give it the K stride too
        constexpr uint32_t b_lbo = BN / L::BB > 1 ? L::B_GROUP : L::B_ATOM;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % WG_STAGES;
            const uint32_t ph = (uint32_t)(i / WG_STAGES) & 1u;
            if (failed || !mbar_wait(full + s, ph, args.err, 2, &failed)) {
                failed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a = smem_u32(smem + s * L::STAGE), b = a + L::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)  // K = 16 per MMA: two atoms of 8 K rows
                mma_bf16(tmem, sdesc_mn(a + kk * 1024, 4096, 512, 4),
                         sdesc_mn(b + kk * 2 * L::B_ATOM, b_lbo, L::B_ATOM, L::B_LAYOUT), idesc,
                         (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(empty + s);
        }
        mma_commit(done);  // also when stopped early: every issued MMA drains before dealloc
    }
    __syncwarp();
    if (nkb > 0 && !mbar_wait(done, 0, args.err, 3)) failed = 1;
    __syncthreads();
    const bool ok = nkb > 0 && !failed;
    if (warp == 0 && lane == 0 && failed) {  // let every started copy land
        for (int i = max(0, issued - WG_STAGES); i < issued; ++i)
            mbar_wait(full + (i % WG_STAGES), (uint32_t)(i / WG_STAGES) & 1u, args.err, 4);
    }
    tc_fence_after();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        float* C = args.ws + ((int64_t)blockIdx.z * args.Mrows + row) * args.N;
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            const int col0 = n0 + c;
            if (row >= args.Mrows || col0 >= args.N) continue;
            if (col0 + 16 <= args.N && (args.N % 4) == 0) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    reinterpret_cast<float4*>(C + col0)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (col0 + j < args.N) C[col0 + j] = v[j];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, L::TMEM_COLS);
}

template <int BN, int BKC>
cudaError_t launch_conv(const CUtensorMap& tx, const CUtensorMap& tw, const ConvArgs& a,
                        cudaStream_t st) {
    using L = ConvSmem<BN, BKC>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(conv_bf16_kernel<BN, BKC>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES);
    });
    if (attr != cudaSuccess) return attr;
    const dim3 grid((a.M + CBM - 1) / CBM, (a.N + BN - 1) / BN, 1);
    conv_bf16_kernel<BN, BKC><<<grid, 128, L::BYTES, st>>>(tx, tw, a);
    return cudaGetLastError();
}

constexpr int kRowsSmemBudget = 200 * 1024;

template <int BN, int BKC>
cudaError_t launch_rows(const CUtensorMap& tx, const CUtensorMap& tw, const RowsArgs& a,
                        cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(conv_rows_kernel<BN, BKC>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    1024 + kRowsSmemBudget + 256);
    });
    if (attr != cudaSuccess) return attr;
    const size_t smem = 1024 + (size_t)a.stages * a.stage_bytes + 256;
    const dim3 grid((a.M + a.mt * CBM - 1) / (a.mt * CBM), (a.N + BN - 1) / BN, 1);
    conv_rows_kernel<BN, BKC><<<grid, 128, smem, st>>>(tx, tw, a);
    return cudaGetLastError();
}

template <int BKC>
cudaError_t launch_rows_bkc(const CUtensorMap& tx, const CUtensorMap& tw, const RowsArgs& a,
                            int BN, cudaStream_t st) {
    switch (BN) {
    case 32: return launch_rows<32, BKC>(tx, tw, a, st);
    case 64: return launch_rows<64, BKC>(tx, tw, a, st);
    case 128: return launch_rows<128, BKC>(tx, tw, a, st);
    default: return launch_rows<256, BKC>(tx, tw, a, st);
    }
}

template <int BKC>
cudaError_t launch_conv_bkc(const CUtensorMap& tx, const CUtensorMap& tw, const ConvArgs& a,
                            int BN, cudaStream_t st) {
    switch (BN) {
    case 32: return launch_conv<32, BKC>(tx, tw, a, st);
    case 64: return launch_conv<64, BKC>(tx, tw, a, st);
    case 128: return launch_conv<128, BKC>(tx, tw, a, st);
    default: return launch_conv<256, BKC>(tx, tw, a, st);
    }
}

template <int BN>
cudaError_t launch_wgrad(const CUtensorMap& tx, const CUtensorMap& tb, const WgradArgs& a, int mtiles, int splits,
                         cudaStream_t st) {
    using L = WgradSmem<BN>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(conv_wgrad_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES);
    });
    if (attr != cudaSuccess) return attr;
    const dim3 grid(mtiles, (a.N + BN - 1) / BN, splits);
    conv_wgrad_kernel<BN><<<grid, 128, L::BYTES, st>>>(tx, tb, a);
    return cudaGetLastError();
}

}  // namespace

// Tiles of >= 128 output channels at n >= 16 take the row-reuse kernel (conv_rows_kernel);
// the rest the one-tile kernel.
#ifndef LBM_CONV_ROWS
#define LBM_CONV_ROWS 1
#endif
constexpr bool kConvRows = LBM_CONV_ROWS != 0;

bool conv_implicit_supported(int n, int cin, int cout) {
    return cin % 32 == 0 && n >= 2 && n <= 256 && (n & (n - 1)) == 0 && cout >= 1 && cout <= 256;
}

cudaError_t conv_implicit(const __nv_bfloat16* X, int B, int n, int cin, const __nv_bfloat16* W,
                          long long ldw, int cout, const float* bias, void* out, int mode, int* err,
                          cudaStream_t st) {
    if (!conv_implicit_supported(n, cin, cout) || B < 1 || ((uintptr_t)X & 15) || ((uintptr_t)W & 15) ||
        (ldw % 8) || ldw < 27LL * cin || (mode == CONV_BIAS_RELU_BF16 && !bias) ||
        (mode != CONV_BIAS_RELU_BF16 && mode != CONV_F32))
        return cudaErrorInvalidValue;
    const int bkc = cin % 64 == 0 ? 64 : 32;
    // the 128-voxel M tile as a box: whole x-rows, then y, z and samples
    const int bx = n < 128 ? n : 128;
    const int by = 128 / bx < n ? 128 / bx : n;
    const int bz = 128 / (bx * by) < n ? 128 / (bx * by) : n;
    const int bb = 128 / (bx * by * bz);
    if (bx * by * bz * bb != 128) return cudaErrorInvalidValue;
    const int BN = cout <= 32 ? 32 : cout <= 64 ? 64 : cout <= 128 ? 128 : 256;
    // the row-reuse kernel where it measured faster: tiles of 128 or more output channels
    // (at 64 and fewer the tensor pipe's reads of the A operand from shared memory bound both
    // kernels, and the one-tile kernel keeps more CTAs per SM)
    if (kConvRows && BN >= 128 && n >= 16 && n <= 128) {
        // tiles of whole x-rows of one plane, MT of them per CTA: as many as the tensor
        // memory (MT BN columns) and two pipeline stages of shared memory allow
        const int by1 = 128 / n;
        const int b_bytes = 3 * BN * bkc * 2;
        int mt = 4;
        while (mt > 1 && (mt * BN > 512 || mt * by1 > n ||
                          2 * (((mt * by1 + 2) * n * bkc * 2 + b_bytes + 1023) / 1024 * 1024) > kRowsSmemBudget))
            mt >>= 1;
        const int a_bytes = (mt * by1 + 2) * n * bkc * 2;
        const int stage = (a_bytes + b_bytes + 1023) / 1024 * 1024;
        if (2 * stage <= kRowsSmemBudget) {
            const int stages = std::min(4, kRowsSmemBudget / stage);
            CUtensorMap tx, tw;
            if (!make_x_map(&tx, X, B, n, cin, bkc, n, mt * by1 + 2, 1, 1) ||
                !make_w_map(&tw, W, cout, 27 * cin, ldw, bkc, BN))
                return cudaErrorInvalidValue;
            RowsArgs a{B * n * n * n, cout, n, cin / bkc, cin, n, by1, mt, a_bytes, stage, stages,
                       (uint32_t)std::max(32, mt * BN), mode, out, bias, err};
            return bkc == 64 ? launch_rows_bkc<64>(tx, tw, a, BN, st) : launch_rows_bkc<32>(tx, tw, a, BN, st);
        }
    }
    CUtensorMap tx, tw;
    if (!make_x_map(&tx, X, B, n, cin, bkc, bx, by, bz, bb) ||
        !make_w_map(&tw, W, cout, 27 * cin, ldw, bkc, BN))
        return cudaErrorInvalidValue;
    ConvArgs a{B * n * n * n, cout, n, cin / bkc, bx, by, bz, mode, out, bias, err};
    return bkc == 64 ? launch_conv_bkc<64>(tx, tw, a, BN, st) : launch_conv_bkc<32>(tx, tw, a, BN, st);
}

bool conv_wgrad_implicit_supported(int B, int n, int cin, int cout) {
    const int64_t M = (int64_t)B * n * n * n;
    return n >= 2 && n <= 256 && (n & (n - 1)) == 0 && cin % 32 == 0 && cout >= 8 && cout <= 256 &&
           cout % 8 == 0 && B >= 1 && M < (int64_t(1) << 31) - 64;
}

cudaError_t conv_wgrad_implicit(const __nv_bfloat16* X, int B, int n, int cin, const __nv_bfloat16* dZ, int cout,
                                int Kp, float* ws, size_t ws_floats, int splits, float* dWT, int accumulate,
                                int* err, cudaStream_t st) {
    if (!conv_wgrad_implicit_supported(B, n, cin, cout) || Kp < 27 * cin || splits < 1 || ((uintptr_t)X & 15) ||
        ((uintptr_t)dZ & 15))
        return cudaErrorInvalidValue;
    const int64_t M = (int64_t)B * n * n * n;
    const int kblocks = (int)((M + 63) / 64);
    const int per = (kblocks + splits - 1) / splits;
    const int used = (kblocks + per - 1) / per;
    const int mtiles = (Kp + CBM - 1) / CBM;
    if ((size_t)used * Kp * cout > ws_floats) return cudaErrorInvalidValue;
    // the 64-voxel K block as a box of the grid: x-row segments, whole rows, planes, samples
    const int bx = n < 64 ? n : 64;
    const int by = 64 / bx < n ? 64 / bx : n;
    const int bz = 64 / (bx * by) < n ? 64 / (bx * by) : n;
    const int bb = 64 / (bx * by * bz);
    if (bx * by * bz * bb != 64) return cudaErrorInvalidValue;
    const int BN = cout <= 32 ? 32 : cout <= 64 ? 64 : cout <= 128 ? 128 : 256;
    CUtensorMap tx, tb;
    if (!make_x_map(&tx, X, B, n, cin, 32, bx, by, bz, bb) ||
        !make_w_map(&tb, dZ, (int)M, cout, cout, BN < 64 ? BN : 64, 64))
        return cudaErrorInvalidValue;
    int ln = 0;
    while ((1 << ln) < n) ++ln;
    WgradArgs a{27 * cin, cout, cin, ln, kblocks, per, Kp, ws, err};
    cudaError_t e;
    switch (BN) {
    case 32: e = launch_wgrad<32>(tx, tb, a, mtiles, used, st); break;
    case 64: e = launch_wgrad<64>(tx, tb, a, mtiles, used, st); break;
    case 128: e = launch_wgrad<128>(tx, tb, a, mtiles, used, st); break;
    default: e = launch_wgrad<256>(tx, tb, a, mtiles, used, st); break;
    }
    if (e != cudaSuccess) return e;
    return add_splits(ws, used, Kp, cout, cout, dWT, accumulate, st);
}

}  // namespace nn
}  // namespace lbm
