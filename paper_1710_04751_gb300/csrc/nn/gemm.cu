// gemm.cu -- BF16 GEMM with FP32 accumulation on the tcgen05 tensor cores:
//   C[M][N] (+)= sum_k A[m][k] * B[n][k]      (both operands K-major, row-major storage)
// One CTA of 128 threads computes a 128 x BN tile (two of them, sharing each B tile, for a
// tall GEMM of 256 columns): warp 0 lane 0 streams 128 x 64 and BN x 64 operand tiles into
// a shared-memory ring of up to 4 stages with TMA (128-byte swizzle);
// warp 1 lane 0 issues tcgen05.mma (M = 128, N = BN, K = 16 per instruction) into a TMEM
// accumulator and frees each stage with tcgen05.commit; then all four warps read the
// accumulator back (warp w owns TMEM lanes 32w..32w+31 = rows 32w..32w+31) and store it.
// grid.z splits K; the split results are added with FP32 atomics, or (GEMM_F32_SPLITS)
// stored in slices of a workspace and added to C in split order by a second kernel, so
// that the sum is the same on every run.  Rows, columns and K
// beyond the operands' extents read as zeros (TMA out-of-bounds fill) and are not stored.
// Every wait is bounded (2 s): on a timeout the kernel records an error code, lets its
// copies and MMAs drain, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "nn.h"
#include "tc.cuh"

namespace lbm {
namespace nn {

constexpr int BM = 128, BK = 64;

// MT 128-row tiles per CTA share each staged B tile (MT = 2 halves the B traffic from L2
// of a tall GEMM); the ring takes what shared memory allows, at most 4 stages.
template <int BN, int MT = 1>
struct GemmSmem {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = MT * A_BYTES + B_BYTES;
    static constexpr int STAGES = (200 * 1024) / STAGE < 4 ? (200 * 1024) / STAGE : 4;
    static constexpr int BYTES = 1024 + STAGES * STAGE + 256;  // + alignment + barriers
    static constexpr uint32_t TMEM_COLS = MT * BN < 32 ? 32 : MT * BN;
};

struct GemmArgs {
    int M, N, K;
    int kblocks_per_split;
    int out_mode;  // GEMM_F32, GEMM_BF16, GEMM_F32_ATOMIC, GEMM_F32_SPLITS
    void* C;
    long long ldc;
    int* err;
    int vec;       // C and its rows are 16-byte aligned: whole 16-column chunks use vector stores
    unsigned long long wait_ns;  // bound of the operand-ring waits (2 s)
    int withhold_loads;  // diagnostic only: issue no operand loads, so the ring wait runs out
};

template <int BN, int MT>
__global__ void __launch_bounds__(128, 1)
    gemm_bf16_tn_kernel(const __grid_constant__ CUtensorMap tmA,
                        const __grid_constant__ CUtensorMap tmB, GemmArgs args) {
    using L = GemmSmem<BN, MT>;
    constexpr int STAGES = L::STAGES;
    extern __shared__ uint8_t gemm_smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(gemm_smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * L::STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ volatile int failed;

    // a CTA that starts after another one timed out does nothing
    if (*static_cast<volatile int*>(args.err) != 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM * MT, n0 = blockIdx.y * BN;
    const int kb_total = (args.K + BK - 1) / BK;
    const int kb0 = blockIdx.z * args.kblocks_per_split;
    const int nkb = min(args.kblocks_per_split, kb_total - kb0);

    if (threadIdx.x == 0) {
        failed = 0;
        for (int s = 0; s < STAGES; ++s) {
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

    int issued = 0;  // producer: stages loaded
    if (nkb > 0 && warp == 0 && lane == 0 && !args.withhold_loads) {
        for (int i = 0; i < nkb; ++i) {
            const int s = i % STAGES;
            const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
            if (i >= STAGES && !mbar_wait(empty + s, ph ^ 1u, args.err, 1, &failed, args.wait_ns)) {
                failed = 1;
                break;
            }
            if (failed) break;
            uint8_t* a = smem + s * L::STAGE;
            mbar_expect_tx(full + s, L::STAGE);
#pragma unroll
            for (int t = 0; t < MT; ++t)
                tma_load_2d(a + t * L::A_BYTES, &tmA, full + s, (kb0 + i) * BK, m0 + t * BM);
            tma_load_2d(a + MT * L::A_BYTES, &tmB, full + s, (kb0 + i) * BK, n0);
            ++issued;
        }
    } else if (nkb > 0 && warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16_f32(BM, BN);
        for (int i = 0; i < nkb; ++i) {
            const int s = i % STAGES;
            const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
            if (failed || !mbar_wait(full + s, ph, args.err, 2, &failed, args.wait_ns)) {
                failed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a = smem_u32(smem + s * L::STAGE), b = a + MT * L::A_BYTES;
#pragma unroll
            for (int t = 0; t < MT; ++t)
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    mma_bf16(tmem + (uint32_t)(t * BN), sdesc_k_sw128(a + t * L::A_BYTES + kk * 32),
                             sdesc_k_sw128(b + kk * 32), idesc, (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(empty + s);
        }
        mma_commit(done);  // also when stopped early: every issued MMA drains before dealloc
    }
    __syncwarp();
    // the accumulator is complete (or the MMA thread gave up) once `done` fires
    if (nkb > 0 && !mbar_wait(done, 0, args.err, 3)) failed = 1;  // no early exit: MMAs drain
    __syncthreads();
    const bool ok = nkb > 0 && !failed;  // block-uniform
    if (warp == 0 && lane == 0 && failed) {
        // let every TMA copy this CTA started land before its shared memory goes away
        for (int i = max(0, issued - STAGES); i < issued; ++i)
            mbar_wait(full + (i % STAGES), (uint32_t)(i / STAGES) & 1u, args.err, 4);
    }
    tc_fence_after();
#pragma unroll 1
    for (int t = 0; t < MT && ok; ++t) {
        const int row = m0 + t * BM + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * BN + c), v);
            if (row < args.M) {
                const int col0 = n0 + c;
                const bool full = args.vec && col0 + 16 <= args.N;  // 16-byte stores
                if (args.out_mode == GEMM_BF16) {
                    __nv_bfloat16* C = static_cast<__nv_bfloat16*>(args.C) + row * args.ldc;
                    if (full) {
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
                } else if (args.out_mode == GEMM_F32 || args.out_mode == GEMM_F32_SPLITS) {
                    // GEMM_F32_SPLITS: split z stores its partial tile in slice z
                    const long long slice =
                        args.out_mode == GEMM_F32_SPLITS ? (long long)blockIdx.z * args.M * args.ldc : 0;
                    float* C = static_cast<float*>(args.C) + slice + row * args.ldc;
                    if (full) {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            reinterpret_cast<float4*>(C + col0)[j] =
                                make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (col0 + j < args.N) C[col0 + j] = v[j];
                    }
                } else {
                    float* C = static_cast<float*>(args.C) + row * args.ldc;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (col0 + j < args.N) atomicAdd(C + col0 + j, v[j]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, L::TMEM_COLS);
}

// -------------------------------------------------------------------------------------
// host side
// -------------------------------------------------------------------------------------

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
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

// Row-major BF16 matrix [rows][cols] with row stride ld (elements), read in boxes of
// box_rows x 64 with the 128-byte swizzle.
static bool make_map(CUtensorMap* map, const void* base, int rows, int cols, long long ld,
                     int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int MT = 1>
static cudaError_t launch(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& a,
                          int splits, cudaStream_t st) {
    using L = GemmSmem<BN, MT>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(gemm_bf16_tn_kernel<BN, MT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES);
    });
    if (attr != cudaSuccess) return attr;
    const dim3 grid((a.M + BM * MT - 1) / (BM * MT), (a.N + BN - 1) / BN, splits);
    gemm_bf16_tn_kernel<BN, MT><<<grid, 128, L::BYTES, st>>>(ta, tb, a);
    return cudaGetLastError();
}

// The K blocks of one split (*per) and the number of splits actually launched: every
// split gets at least one K block.
static int split_count(int K, int splits, int* per) {
    const int kb_total = (K + BK - 1) / BK;
    splits = splits > kb_total ? kb_total : splits;
    *per = (kb_total + splits - 1) / splits;
    return (kb_total + *per - 1) / *per;
}

// Rows from which a 256-column GEMM takes two M tiles per CTA: from 160 pairs of tiles up,
// so that the CTAs still cover the 152 SMs (at 16384 rows the pairs would leave 88 idle).
#ifndef LBM_GEMM_TALL_ROWS
#define LBM_GEMM_TALL_ROWS 40960
#endif
constexpr int kTallRows = LBM_GEMM_TALL_ROWS;

cudaError_t gemm_bf16(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B,
                      long long ldb, void* C, long long ldc, int M, int N, int K, int out_mode,
                      int splits, int* err, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0 || (lda % 8) || (ldb % 8) || lda < K || ldb < K || splits < 1 ||
        ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || out_mode < GEMM_F32 || out_mode > GEMM_F32_SPLITS)
        return cudaErrorInvalidValue;
    const int BN = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
    int per;
    splits = split_count(K, splits, &per);
    if (splits > 1 && out_mode != GEMM_F32_ATOMIC && out_mode != GEMM_F32_SPLITS)
        return cudaErrorInvalidValue;
    CUtensorMap ta, tb;
    if (!make_map(&ta, A, M, K, lda, BM) || !make_map(&tb, B, N, K, ldb, BN))
        return cudaErrorInvalidValue;
    const long long esz = out_mode == GEMM_BF16 ? 2 : 4;
    const int vec = ((uintptr_t)C % 16 == 0) && ((ldc * esz) % 16 == 0);
    GemmArgs a{M, N, K, per, out_mode, C, ldc, err, vec, 2000000000ull, 0};
    switch (BN) {
    case 32: return launch<32>(ta, tb, a, splits, st);
    case 64: return launch<64>(ta, tb, a, splits, st);
    case 128: return launch<128>(ta, tb, a, splits, st);
    default:
        // a tall GEMM: two 128-row tiles per CTA share the B tile (half the L2 reads of B)
        if (a.M >= kTallRows) return launch<256, 2>(ta, tb, a, splits, st);
        return launch<256>(ta, tb, a, splits, st);
    }
}

// Diagnostic of the bounded waits: one 128 x 32 tile over one K block whose operand loads
// are withheld, so the MMA thread's wait for the first stage can only run out (after
// 10 ms).  The kernel then records code 2 in *err, issues no MMA, lets nothing drain
// (nothing was loaded), frees its TMEM and returns.  `operand` is any 16-byte aligned
// device buffer of 128 x 64 BF16 values; the tensor maps point at it, nothing reads it.
cudaError_t gemm_timeout_probe(const __nv_bfloat16* operand, float* C, int* err, cudaStream_t st) {
    CUtensorMap ta, tb;
    if (!make_map(&ta, operand, 128, 64, 64, BM) || !make_map(&tb, operand, 32, 64, 64, 32))
        return cudaErrorInvalidValue;
    GemmArgs a{128, 32, 64, 1, GEMM_F32, C, 32, err, 0, 10000000ull, 1};
    return launch<32>(ta, tb, a, 1, st);
}

// C[r][c] += ws[0][r][c] + ws[1][r][c] + ... in split order (slices of M * ldc floats).
__global__ void add_splits_kernel(const float* __restrict__ ws, int splits, int M, int N, long long ldc,
                                  float* __restrict__ C, int accumulate) {
    const int64_t total = (int64_t)M * N;
    const int64_t slice = (int64_t)M * ldc;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = (q / N) * ldc + q % N;
        float s = accumulate ? C[o] : 0.f;
        // unrolled so that the slices' loads are in flight together; added in split order
#pragma unroll 8
        for (int z = 0; z < splits; ++z) s += ws[z * slice + o];
        C[o] = s;
    }
}

cudaError_t add_splits(const float* ws, int splits, int M, int N, long long ldc, float* C, int accumulate,
                       cudaStream_t st) {
    const int64_t total = (int64_t)M * N;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
    add_splits_kernel<<<blocks, 256, 0, st>>>(ws, splits, M, N, ldc, C, accumulate);
    return cudaGetLastError();
}

cudaError_t gemm_bf16_add_splitk(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B,
                                 long long ldb, float* C, long long ldc, int M, int N, int K,
                                 int splits, float* ws, size_t ws_floats, int* err, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0 || splits < 1 || ldc < N) return cudaErrorInvalidValue;
    int per;
    const int used = split_count(K, splits, &per);
    if ((size_t)used * M * ldc > ws_floats) return cudaErrorInvalidValue;
    cudaError_t e = gemm_bf16(A, lda, B, ldb, ws, ldc, M, N, K, GEMM_F32_SPLITS, used, err, st);
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)M * N;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
    add_splits_kernel<<<blocks, 256, 0, st>>>(ws, used, M, N, ldc, C, 1);
    return cudaGetLastError();
}

size_t gemm_splitk_floats(int M, long long ldc, int K, int splits) {
    int per;
    return (size_t)split_count(K, splits, &per) * M * ldc;
}

}  // namespace nn
}  // namespace lbm
