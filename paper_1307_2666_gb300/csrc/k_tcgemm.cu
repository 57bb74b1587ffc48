// Batched FP32 matrix products on the tcgen05 tensor cores (sm_103a): the
// dense contractions of the large-box elimination, i.e. the blocks of
// Lemma 2.4 (B_sr = A_sr - A_ss T, B_rr = A_rr - T^T B_sr - A_rs T,
// B_rs = A_rs - T^T A_ss) and the Schur update S = -X Z of the skeletons.
//
//     C = beta C + alpha op(A) op(B),   beta in {0, 1},
//
// for a list of independent problems, column-major, op = identity or
// transpose.  FP32 values are split exactly into three BF16 pieces,
// x = x0 + x1 + x2 (each piece holds the next 8 significant bits, so the sum
// carries FP32's 24), and every product takes the six piece pairs with
// i + j <= 2, accumulated in FP32 in tensor memory: the pairs left out weigh
// at most ~3 * 2^-24 of |a b|, the rounding of FP32 itself.
//
// One CTA computes one 128 x 256 tile of one problem:
//   warps 0-3  load 128 x 32 blocks of op(A) and 256 x 32 blocks of op(B)
//              from global memory, split them and store the pieces in the
//              K-major core-matrix layout of the MMA operands (a 3-stage
//              ring); afterwards they read the accumulator out of tensor
//              memory and write C (one thread per row, coalesced along rows);
//   warp 4     allocates the 256 accumulator columns; one thread issues the
//              MMAs (6 pairs x 2 K-steps of 16 per stage, M = 128, N = 256).
// Every wait is bounded: on time-out the CTA ORs `flag` into *status, drains its own
// MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>

#include "hif_types.h"
#include "launch.h"
#include "tc_ptx.cuh"

namespace hif {
namespace {

constexpr int GM = 128;                          // rows per tile (TMEM lanes)
constexpr int GN = 256;                          // columns per tile (TMEM columns)
constexpr int GK = 32;                           // K per stage
constexpr int GST = 3;                           // ring depth
constexpr int A_PIECE = GM * GK * 2;             // bytes of one BF16 piece of the A block
constexpr int B_PIECE = GN * GK * 2;
constexpr int G_STAGE = 3 * A_PIECE + 3 * B_PIECE;
constexpr int SBO = (GK / 8) * 128;              // 8-row groups are 512 B apart
constexpr int NPROD = 128;                       // loader / epilogue threads
constexpr long long G_WAIT = 4000000000LL;       // ~2 s at GB300 clocks

static_assert(G_STAGE % 1024 == 0, "stage alignment");

struct GBars {
    uint64_t full[GST];        // stage stored (NPROD arrivals)
    uint64_t empty[GST];       // stage consumed by the MMAs (1 commit)
    uint64_t acc_full;         // accumulator complete (1 commit)
    uint64_t drain;
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ bool gwait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    const long long t0 = clock64();
    while (true) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > G_WAIT) {
            *abort = 1;
            return false;
        }
    }
}

// x = h0 + h1 + h2 exactly up to the last piece's rounding
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h0, __nv_bfloat16& h1, __nv_bfloat16& h2) {
    h0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h0);
    h1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(h1);
    h2 = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ uint32_t pk(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// 8 consecutive-K values of operand row `row` (k from k0) -> the three pieces
// at byte offset (row / 8) * SBO + kb * 128 + (row % 8) * 16 of each piece
__device__ __forceinline__ void store_row8(unsigned char* base, int piece_bytes, int row, int kb, const float (&v)[8]) {
    __nv_bfloat16 h[3][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) split3(v[e], h[0][e], h[1][e], h[2][e]);
    const int off = (row >> 3) * SBO + kb * 128 + (row & 7) * 16;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        uint4 w;
        w.x = pk(h[p][0], h[p][1]);
        w.y = pk(h[p][2], h[p][3]);
        w.z = pk(h[p][4], h[p][5]);
        w.w = pk(h[p][6], h[p][7]);
        *reinterpret_cast<uint4*>(base + p * piece_bytes + off) = w;
    }
}

// op(X)[r, l] for r < R, l < K (0 outside): X[r + ld l] or, transposed, X[l + ld r]
__device__ __forceinline__ void load8(const float* X, int64_t ld, int tr, int r, int R, int l0, int K, float (&v)[8]) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int l = l0 + e;
        v[e] = (r < R && l < K) ? __ldg(tr ? X + l + ld * r : X + r + ld * l) : 0.f;
    }
}

}  // namespace

__global__ void __launch_bounds__(160, 1) tc_gemm_kernel(const TcGemmProb* probs, int* status, int flag) {
    const TcGemmProb P = probs[blockIdx.z];
    const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
    if (m0 >= P.m || n0 >= P.n) return;             // uniform over the CTA, before any allocation
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)gsm_raw + 1023) & ~(uintptr_t)1023);
    GBars* bars = (GBars*)(smem + GST * G_STAGE);
    volatile int* abort = &bars->abort;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nk = (P.k + GK - 1) / GK;

    if (threadIdx.x == 0) {
        for (int i = 0; i < GST; ++i) {
            tc::mbar_init(&bars->full[i], NPROD);
            tc::mbar_init(&bars->empty[i], 1);
        }
        tc::mbar_init(&bars->acc_full, 1);
        tc::mbar_init(&bars->drain, 1);
        bars->abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == 4) tc::tmem_alloc(&bars->tmem, GN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = bars->tmem;

    if (warp == 4) {
        // ------------------------------------------------------------ issuer
        if (lane == 0) {
            bool ok = true;
            const uint32_t idesc = tc::idesc_bf16_f32(GM, GN);
            for (int it = 0; it < nk; ++it) {
                const int s = it % GST;
                if (!gwait(&bars->full[s], (uint32_t)((it / GST) & 1), abort)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t st = tc::smem_addr(smem + s * G_STAGE);
#pragma unroll
                for (int kk = 0; kk < GK / 16; ++kk) {
                    // piece pairs (i, j) with i + j <= 2
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        const int pi = q == 0 ? 0 : q == 1 ? 0 : q == 2 ? 1 : q == 3 ? 0 : q == 4 ? 1 : 2;
                        const int pj = q == 0 ? 0 : q == 1 ? 1 : q == 2 ? 0 : q == 3 ? 2 : q == 4 ? 1 : 0;
                        const uint64_t ad = tc::sdesc(st + pi * A_PIECE + kk * 256, 128, SBO);
                        const uint64_t bd = tc::sdesc(st + 3 * A_PIECE + pj * B_PIECE + kk * 256, 128, SBO);
                        tc::mma_bf16(tmem, ad, bd, idesc, !(it == 0 && kk == 0 && q == 0));
                    }
                }
                tc::mma_commit(&bars->empty[s]);
            }
            if (ok && nk > 0) tc::mma_commit(&bars->acc_full);
            tc::mma_commit(&bars->drain);
            const long long t0 = clock64();
            while (!tc::mbar_try_wait(&bars->drain, 0) && clock64() - t0 < G_WAIT) {}
            if (!ok) *abort = 1;
        }
    } else {
        // ------------------------------------------------- loaders, epilogue
        const int t = threadIdx.x;
        bool ok = true;
        for (int it = 0; it < nk; ++it) {
            const int s = it % GST;
            if (it >= GST && !gwait(&bars->empty[s], (uint32_t)((it / GST - 1) & 1), abort)) {
                ok = false;
                break;
            }
            unsigned char* st = smem + s * G_STAGE;
            const int k0 = it * GK;
            // A block: row t, the four 8-wide K groups
#pragma unroll
            for (int kb = 0; kb < GK / 8; ++kb) {
                float v[8];
                load8(P.A, P.lda, P.tA, m0 + t, P.m, k0 + 8 * kb, P.k, v);
                store_row8(st, A_PIECE, t, kb, v);
            }
            // B block: rows t and t + 128 (output columns n0 + row)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int kb = 0; kb < GK / 8; ++kb) {
                    float v[8];
                    load8(P.B, P.ldb, !P.tB, n0 + t + 128 * h, P.n, k0 + 8 * kb, P.k, v);
                    store_row8(st + 3 * A_PIECE, B_PIECE, t + 128 * h, kb, v);
                }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&bars->full[s]);
        }
        // epilogue: row m0 + t of the tile, 32 columns per TMEM load
        if (ok && nk > 0 && gwait(&bars->acc_full, 0, abort)) {
            tc::tc_fence_after();
            const int i = m0 + t;
            const uint32_t tb = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
            for (int cb = 0; cb < GN / 32; ++cb) {
                float v[32];
                tc::tmem_ld32(tb + 32 * cb, v);
                if (i < P.m) {
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int j = n0 + 32 * cb + q;
                        if (j < P.n) {
                            float* c = P.C + i + P.ldc * (int64_t)j;
                            *c = P.beta ? *c + P.alpha * v[q] : P.alpha * v[q];
                        }
                    }
                }
            }
        } else if (nk == 0 && !P.beta && m0 + t < P.m) {
            for (int j = n0; j < min(P.n, n0 + GN); ++j) P.C[m0 + t + P.ldc * (int64_t)j] = 0.f;
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && bars->abort) atomicOr(status, flag);
    if (warp == 4) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, GN);
    }
}

size_t tc_gemm_smem_bytes() { return (size_t)GST * G_STAGE + sizeof(GBars) + 1024; }

cudaError_t launch_tc_gemm(const TcGemmProb* dprobs, int nprob, int max_m, int max_n, int* status, int flag,
                           cudaStream_t st) {
    if (nprob <= 0 || max_m <= 0 || max_n <= 0) return cudaSuccess;
    static bool attr_set = false;
    const size_t smem = tc_gemm_smem_bytes();
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const dim3 grid((unsigned)((max_n + GN - 1) / GN), (unsigned)((max_m + GM - 1) / GM), (unsigned)nprob);
    note_launch();
    tc_gemm_kernel<<<grid, 160, smem, st>>>(dprobs, status, flag);
    return cudaGetLastError();
}

}  // namespace hif
