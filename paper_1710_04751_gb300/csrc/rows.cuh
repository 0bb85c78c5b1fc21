// rows.cuh -- the staged row kernel of the 16-bit storage forms: a persistent grid whose
// blocks each advance a sequence of x-rows of the cavity, with the inputs of the next
// rows in flight while the current one is computed.
//
// Why: a 16-bit node update moves half the bytes of an FP32 one, so to keep HBM busy twice
// as many node updates must have their loads in flight; with loads into registers that is
// bounded by occupancy, and a warp has no loads in flight while it computes.  Here the
// loads are asynchronous bulk copies (cp.async.bulk, the TMA engine's untiled form) into a
// ring of shared-memory stages, each completing on an mbarrier, so the bytes in flight do
// not depend on registers and the copies of the rows ahead overlap the arithmetic.
//
// The update of an x-row (j, k) away from the y and z walls needs, per link a, the row
// (j - e_y, k - e_z) of population plane a -- one contiguous run of nx values, since a link
// whose source lies beyond an x face takes the node's own opposite population instead
// (Sec. 3) -- and the node temperatures (the references of the stored scalar deviations)
// of the 9 (D3Q15) or 5 (D3Q7) distinct source rows.  Those own opposite populations lie
// in the staged own row for the axis links; for the diagonal links they come as 16-byte
// chunks of the own row at x = 0 and x = nx - 8.  Per row: 15 + Q population rows, the
// temperature rows and the wall chunks, all copies with 16-byte aligned addresses and
// sizes (nx a multiple of 8).
//
// Warp 0 issues a row's copies (one copy per lane) into a free stage; both warps compute
// the row's node pairs from shared memory with pair.cuh's packed update and store to
// global memory directly.  Rows at a y or z wall use node.cuh's update from global memory.
// Every mbarrier wait is bounded: on a timeout the kernel records kStageTimeout in the
// context's error word, waits (bounded) for the copies it issued and returns.
#pragma once

#include "nn/tc.cuh"
#include "node.cuh"
#include "pair.cuh"

namespace lbm {

constexpr int kRowsThreads = 64;
constexpr int kRowsMaxNx = 512;
constexpr int kStagePad = 8;   // 16-bit values (16 bytes) around each staged population row
constexpr int kStagePadT = 4;  // floats (16 bytes) around each staged temperature row

// Untiled bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16),
// completing its bytes on the barrier.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            nn::smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(nn::smem_u32(bar))
        : "memory");
}

// Orders this thread's earlier shared-memory accesses (made visible to it by a barrier)
// before its later asynchronous-proxy writes to shared memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Staged temperature row of the links with (e_y, e_z): 0 own row, 1..4 the axis rows,
// 5..8 the diagonal rows (D3Q15 only).
__host__ __device__ constexpr int trow(int ey, int ez) {
    return (ey == 0 && ez == 0) ? 0
         : ez == 0              ? (ey > 0 ? 1 : 2)
         : ey == 0              ? (ez > 0 ? 3 : 4)
                                : 5 + (ey < 0) + 2 * (ez < 0);
}
__host__ __device__ constexpr int trow_ey(int r) {
    return r == 1 ? 1 : r == 2 ? -1 : r >= 5 ? (((r - 5) & 1) ? -1 : 1) : 0;
}
__host__ __device__ constexpr int trow_ez(int r) {
    return r == 3 ? 1 : r == 4 ? -1 : r >= 5 ? (((r - 5) >> 1) ? -1 : 1) : 0;
}

// Byte layout of one stage (every offset a multiple of 16).
struct RowLayout {
    int rw, rwt;           // staged row lengths (elements): populations, temperatures
    int offG, offT, offW;  // bytes: thermal rows, temperature rows, wall chunks
    int stage;             // bytes per stage (a multiple of 128)
    int ncopy;             // bulk copies per row
    uint32_t tx;           // bytes per row
};

template <int Q>
__host__ __device__ inline RowLayout row_layout(int nx) {
    constexpr int NT = Q == 15 ? 9 : 5;   // temperature rows
    constexpr int NW = Q == 15 ? 16 : 8;  // wall chunks: 8 flow (+ 8 scalar)
    RowLayout L;
    L.rw = nx + 2 * kStagePad;
    L.rwt = nx + 2 * kStagePadT;
    L.offG = 15 * L.rw * 2;
    L.offT = L.offG + Q * L.rw * 2;
    L.offW = L.offT + NT * L.rwt * 4;
    L.stage = (L.offW + NW * 16 + 127) / 128 * 128;
    L.ncopy = 15 + Q + NT + NW;
    L.tx = (uint32_t)((15 + Q) * nx * 2 + NT * nx * 4 + NW * 16);
    return L;
}

// Warp 0: the copies of row (j, k) into stage `st`, completing on `bar`.  Wall chunk w
// (0..7 flow, 8..15 scalar) holds the own row's population opp(a) at x = 0..7 for the
// +x diagonal a = 7 + 2w' (w' = w mod 8 < 4) and at x = nx-8..nx-1 for the -x diagonal
// a = 8 + 2(w' - 4).
template <typename S, int Q>
__device__ __forceinline__ void issue_row(unsigned char* st, uint64_t* bar, const RowLayout& L,
                                          const S* Fin, const S* Gin, const float* Tin, int nx,
                                          int nxy, int P, int j, int k, int lane) {
    constexpr int NT = Q == 15 ? 9 : 5;
    if (lane == 0) nn::mbar_expect_tx(bar, L.tx);
    __syncwarp();
    for (int cid = lane; cid < L.ncopy; cid += 32) {
        const void* src;
        void* dst;
        uint32_t bytes;
        if (cid < 15 + Q) {
            const bool flow = cid < 15;
            const int a = flow ? cid : cid - 15;
            src = (flow ? Fin : Gin) + (int64_t)a * P + (k - ez(a)) * nxy + (j - ey(a)) * nx;
            dst = st + (flow ? 0 : L.offG) + (a * L.rw + kStagePad) * 2;
            bytes = 2 * nx;
        } else if (cid < 15 + Q + NT) {
            const int r = cid - 15 - Q;
            src = Tin + (k - trow_ez(r)) * nxy + (j - trow_ey(r)) * nx;
            dst = st + L.offT + (r * L.rwt + kStagePadT) * 4;
            bytes = 4 * nx;
        } else {
            const int w = cid - 15 - Q - NT, ww = w & 7;
            const int a = ww < 4 ? 7 + 2 * ww : 8 + 2 * (ww - 4);
            src = (w < 8 ? Fin : Gin) + (int64_t)opp(a) * P + k * nxy + j * nx + (ww < 4 ? 0 : nx - 8);
            dst = st + L.offW + w * 16;
            bytes = 16;
        }
        bulk_copy(dst, src, bytes, bar);
    }
}

// Pull of the pair (2t, 2t+1) of a staged row: the same values pair_node loads from global
// memory (stored deviation + rest value; at an x face the own opposite population, with
// the anti-bounce-back of the scalar).
template <typename S, int Q>
__device__ __forceinline__ void stage_pull(const unsigned char* st, const RowLayout& L,
                                           const PairParams& q, int t, bool lo, bool hi, int nx,
                                           float2 (&f)[15], float2 (&g)[Q]) {
    using Pk = Pack<S>;
    using two = typename Pk::two;
    const S* sF = reinterpret_cast<const S*>(st) + kStagePad;
    const S* sG = reinterpret_cast<const S*>(st + L.offG) + kStagePad;
    const float* sT = reinterpret_cast<const float*>(st + L.offT) + kStagePadT;
    const S* sW = reinterpret_cast<const S*>(st + L.offW);
    const int i0 = 2 * t;
    const float Tlo = sT[0], Thi = sT[nx - 1];  // own row at the faces
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const S* s = sG + a * L.rw;
        const float* tr = sT + trow(ey(a), ez(a)) * L.rwt;
        const float2 Tc = *reinterpret_cast<const float2*>(tr + i0);
        if (ex(a) == 0) {
            g[a] = fma2(q.wg[a], Tc, Pk::to_float2(*reinterpret_cast<const two*>(s + i0)));
        } else if (ex(a) > 0) {
            // node 2t pulls from 2t - 1; at the cold face its own opposite population
            const S* w = a == 1 ? sG + 2 * L.rw : sW + (8 + (a - 7) / 2) * 8;
            const float2 Tm = *reinterpret_cast<const float2*>(tr + i0 - 2);
            const S* p0 = lo ? w : s + i0 - 1;
            float2 v = fma2(q.wg[a], make_float2(lo ? Tlo : Tm.y, Tc.x),
                            make_float2(Pk::to_float(*p0), Pk::to_float(s[i0])));
            v.x = lo ? q.wTc2[a] - v.x : v.x;
            g[a] = v;
        } else {
            // node 2t + 1 pulls from 2t + 2; at the hot face its own opposite population
            const S* w = a == 2 ? sG + L.rw + nx - 1 : sW + (12 + (a - 8) / 2) * 8 + 7;
            const float2 Tp = *reinterpret_cast<const float2*>(tr + i0 + 2);
            const S* p1 = hi ? w : s + i0 + 2;
            float2 v = fma2(q.wg[a], make_float2(Tc.y, hi ? Thi : Tp.x),
                            make_float2(Pk::to_float(s[i0 + 1]), Pk::to_float(*p1)));
            v.y = hi ? q.wTh2[a] - v.y : v.y;
            g[a] = v;
        }
    }
#pragma unroll
    for (int a = 0; a < 15; ++a) {
        const S* s = sF + a * L.rw;
        if (ex(a) == 0) {
            f[a] = add2(Pk::to_float2(*reinterpret_cast<const two*>(s + i0)), q.wf[a]);
        } else if (ex(a) > 0) {
            const S* w = a == 1 ? sF + 2 * L.rw : sW + ((a - 7) / 2) * 8;
            const S* p0 = lo ? w : s + i0 - 1;
            f[a] = add2(make_float2(Pk::to_float(*p0), Pk::to_float(s[i0])), q.wf[a]);
        } else {
            const S* w = a == 2 ? sF + L.rw + nx - 1 : sW + (4 + (a - 8) / 2) * 8 + 7;
            const S* p1 = hi ? w : s + i0 + 2;
            f[a] = add2(make_float2(Pk::to_float(s[i0 + 1]), Pk::to_float(*p1)), q.wf[a]);
        }
    }
}

// Blocks per SM the kernel is built for (its register budget); the stages' shared memory
// sets the actual residency.
#ifndef LBM_ROWS_STAGES
#define LBM_ROWS_STAGES 3
#endif
#ifndef LBM_ROWS_MIN_BLOCKS_Q15
#define LBM_ROWS_MIN_BLOCKS_Q15 4
#endif
#ifndef LBM_ROWS_MIN_BLOCKS_Q7
#define LBM_ROWS_MIN_BLOCKS_Q7 4
#endif
template <int Q>
constexpr int rows_min_blocks() { return Q == 15 ? LBM_ROWS_MIN_BLOCKS_Q15 : LBM_ROWS_MIN_BLOCKS_Q7; }

template <typename S, int Q, int NST>
__global__ void __launch_bounds__(kRowsThreads, (rows_min_blocks<Q>()))
    step_rows_kernel(const S* __restrict__ Fin, const S* __restrict__ Gin,
                     const float* __restrict__ Tin, S* __restrict__ Fout, S* __restrict__ Gout,
                     float* __restrict__ Tout, ParamsOf<S> p, PairParams q, int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int nx = p.nx, ny = p.ny, nz = p.nz, nxy = nx * ny, P = (int)p.plane;
    const RowLayout L = row_layout<Q>(nx);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NST * L.stage);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) nn::mbar_init(&bar[s], 1);
        nn::mbar_fence_init();
    }
    __syncthreads();
    const int ntask = ny * nz, G = gridDim.x;
    auto interior = [&](int n) {
        const int j = n % ny, k = n / ny;
        return j >= 1 && j + 1 < ny && k >= 1 && k + 1 < nz;
    };
    auto next_interior = [&](int n) {
        while (n < ntask && !interior(n)) n += G;
        return n;
    };
    // rows are taken in the order n = blockIdx.x + m G; interior rows go through the stages
    int issue_n = next_interior(blockIdx.x), issued = 0, cons = 0;
    for (int s = 0; s < NST && issue_n < ntask; ++s) {
        if (warp == 0)
            issue_row<S, Q>(smem + s * L.stage, &bar[s], L, Fin, Gin, Tin, nx, nxy, P, issue_n % ny,
                            issue_n / ny, lane);
        ++issued;
        issue_n = next_interior(issue_n + G);
    }
    for (int n = blockIdx.x; n < ntask; n += G) {
        const int j = n % ny, k = n / ny;
        if (!interior(n)) {
            for (int i = threadIdx.x; i < nx; i += kRowsThreads)
                cavity_node<S, Q, false>(Fin, Gin, Tin, Fout, Gout, Tout, p, i, j, k);
            continue;
        }
        const int s = cons % NST;
        const bool ok = nn::mbar_wait(&bar[s], (uint32_t)(cons / NST) & 1u, err, kStageTimeout);
        if (__syncthreads_or(!ok)) {
            // give the copies already issued a bounded time to land before the block exits
            for (int c = cons; c < issued; ++c)
                nn::mbar_wait(&bar[c % NST], (uint32_t)(c / NST) & 1u, err, kStageTimeout);
            return;
        }
        const unsigned char* st = smem + s * L.stage;
        const int c_row = k * nxy + j * nx;
        for (int t = threadIdx.x; t < (nx >> 1); t += kRowsThreads) {
            float2 f[15], g[Q];
            stage_pull<S, Q>(st, L, q, t, t == 0, 2 * t + 2 == nx, nx, f, g);
            pair_collide_store<S, Q>(f, g, Fout, Gout, Tout, q, P, c_row + 2 * t);
        }
        __syncthreads();  // stage s is read: refill it with the next row
        if (issue_n < ntask) {
            if (warp == 0) {
                fence_proxy_async_smem();
                issue_row<S, Q>(smem + s * L.stage, &bar[s], L, Fin, Gin, Tin, nx, nxy, P,
                                issue_n % ny, issue_n / ny, lane);
            }
            ++issued;
            issue_n = next_interior(issue_n + G);
        }
        ++cons;
    }
}

}  // namespace lbm
