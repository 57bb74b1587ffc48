// Direct sum y = K v on a uniform grid (the residual operator of the
// refinement, Sec. 5; K as assembled in Sec. 3.1, Eq. (3.1)) on the tcgen05
// tensor cores, in exact integer digits.
//
// Every table entry t and every source value v is written as a short sum of
// signed 8-bit digits against a power-of-two scale,
//     t = 2^eT sum_s dT_s 2^-8(s+1),  v = 2^eX sum_t dX_t 2^-8(t+1),
// |dT_s|, |dX_t| <= 128 (round-to-nearest digit extraction in FP64, exact).
// Digits are BF16 integers, so dT_s * dX_t is exact in the tensor core and
// a sum of up to 1024 of them (<= 2^24) is exact in its FP32 accumulator.
// Products of digit pairs (s, t) are accumulated separately, converted to
// integers every 1024 sources and added into 64-bit integer class sums
// (class k = s + t, weight 2^(eT + eX - 8(k + 2))), so the only rounding is
// the dropped digits (below 2^-55 of max|t| max|v|) and the final FP64
// combination of eight class sums.  Table digits 0..6 and source digits 0..7
// are kept, and pairs with s + t >= 8 are not formed.
//
// On a grid K_ij depends only on the offset i - j, so the kernel block of a
// tile of 128 targets on one grid line against 128 sources on another line is
// a Toeplitz matrix in the last coordinate.  With the target rows taken in
// reverse order it is a Hankel matrix A[i][q] = v[i + q], whose 8 x 8 core
// matrices depend only on the sum of their block indices: the shared-memory
// operand stores the 31 distinct core matrices of each digit slice once and
// the MMA descriptor walks them with equal leading and stride offsets.
//
// CTA roles (256 threads, persistent, one CTA per SM, TMEM 512 columns):
//   warps 0-3  epilogue: TMEM -> integer class sums -> FP64 y (one thread
//              per target row),
//   warp 4     one thread: bulk copies of the source digits and the MMAs,
//   warps 5-7  builders of the Hankel operand from mirrored digit rows.
// Chunks of 128 sources flow through a 4-stage shared-memory ring; two TMEM
// accumulator buffers of 256 columns alternate between 1024-source groups so
// the epilogue of one group overlaps the MMAs of the next.  Every wait is
// bounded; on time-out the kernel sets *status = 1, drains its own MMAs and
// copies, frees TMEM and returns.
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>
#include "hif_types.h"
#include "launch.h"
#include "tc_ptx.cuh"

namespace hif {
namespace {

constexpr int TM = 128;                         // targets per tile (TMEM lanes)
constexpr int KC = 128;                         // sources per chunk
constexpr int ST = 7;                           // table digits
constexpr int SX = 8;                           // source digits
constexpr int NR = 8;                           // right-hand sides per launch
constexpr int NBLK = (TM + KC) / 8 - 1;         // distinct Hankel core matrices per slice (31)
constexpr int A_SLICE = NBLK * 128;             // bytes
constexpr int A_BYTES = ST * A_SLICE;
constexpr int B_BYTES = SX * NR * KC * 2;       // (digit, rhs) rows x KC sources, BF16
constexpr int STAGE = A_BYTES + B_BYTES;
constexpr int NST = 4;                          // ring depth
constexpr int GROUP = 8;                        // chunks per exact FP32 window (1024 sources)
constexpr int ACC = 256;                        // TMEM columns per accumulator buffer
constexpr int NBUILD = 96;                      // builder threads
constexpr int NPAIR = ST * NBLK;                // (slice, core matrix) build items per chunk
constexpr long long WAIT_CYCLES = 4000000000LL; // ~2 s at GB300 clocks

static_assert(STAGE % 128 == 0, "stage alignment");
static_assert(GROUP * KC * 128 * 128 <= (1 << 24), "exact FP32 window");

// accumulator columns of table digit s: (source digit t, rhs) rows of B, t
// limited so that s + t <= 7 (rounded up to the 16-column MMA granularity)
__host__ __device__ constexpr int ncols(int s) { return s == 0 ? 64 : s <= 2 ? 48 : s <= 4 ? 32 : 16; }
__host__ __device__ constexpr int coloff(int s) {
    return s == 0 ? 0 : s == 1 ? 64 : s == 2 ? 112 : s == 3 ? 160 : s == 4 ? 192 : s == 5 ? 224 : 240;
}
__host__ __device__ constexpr int col_slice(int c) {
    return c < 64 ? 0 : c < 112 ? 1 : c < 160 ? 2 : c < 192 ? 3 : c < 224 ? 4 : c < 240 ? 5 : 6;
}
__host__ __device__ constexpr int col_class(int c) { return col_slice(c) + (c - coloff(col_slice(c))) / 8; }
__host__ __device__ constexpr int col_rhs(int c) { return (c - coloff(col_slice(c))) % 8; }
static_assert(coloff(6) + ncols(6) == ACC, "column map");

__device__ __forceinline__ int scale_exp(unsigned long long maxbits) {
    const double m = __longlong_as_double((long long)maxbits);
    return m > 0.0 ? ilogb(m) + 2 : 0;             // |x| 2^-e < 1/2
}

// digits of u in [-1/2, 1/2): d_k = rint(256 r_k), r_{k+1} = 256 r_k - d_k
__device__ __forceinline__ void digits8(double u, float (&d)[8]) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const double x = u * 256.0;
        const double dk = rint(x);
        d[k] = (float)dk;
        u = x - dk;
    }
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&p);
}

struct Bars {
    uint64_t full[NST];
    uint64_t mma_done[NST];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t drain;
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort) {
    const long long t0 = clock64();
    while (true) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            *abort = 1;
            return false;
        }
    }
}

}  // namespace

// ---- digit tables ---------------------------------------------------------

__global__ void tc_maxabs_kernel(const double* x, int64_t n, int cols, int64_t ld,
                                 unsigned long long* out) {
    for (int c = 0; c < cols; ++c) {
        double m = 0.0;
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
            m = fmax(m, fabs(x[e + ld * c]));
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out + c, (unsigned long long)__double_as_longlong(m));
    }
}

// Mirrored table rows: R[s][dl][idx] = digit s of T(dl, |Z0 - idx|) (0 where
// |Z0 - idx| >= n), idx in [0, RL), Z0 = 128 nc - 1, RL = 256 nc; dl indexes
// the offsets of all but the last coordinate.
__global__ void tc_table_rows_kernel(const double* table, int n, int64_t lines, int nc,
                                     const unsigned long long* tmax, __nv_bfloat16* R) {
    const int64_t RL = 256LL * nc, Z0 = 128LL * nc - 1;
    const int eT = scale_exp(*tmax);
    const int64_t tot = lines * RL;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t dl = e / RL, idx = e % RL;
        const int64_t z = Z0 - idx, az = z < 0 ? -z : z;
        float d[8];
        if (az < n) {
            digits8(ldexp(table[dl + lines * az], -eT), d);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) d[k] = 0.f;
        }
#pragma unroll
        for (int s = 0; s < ST; ++s) R[((int64_t)s * lines + dl) * RL + idx] = __float2bfloat16_rn(d[s]);
    }
}

// Source digits in the K-major core-matrix layout of the B operand, chunk by
// chunk: element (digit t, rhs r, source q) of chunk ch at
// ((ch * SX + t) * (KC/8) + q/8) * 64 + r * 8 + q % 8 (BF16 units).
__global__ void tc_source_digits_kernel(const double* v, int64_t N, int n, int64_t lines, int nc, int r0, int nr,
                                        const unsigned long long* xmax, uint4* XB) {
    const int64_t tot = lines * nc * (KC / 8) * NR;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % NR);
        const int kb = (int)((e / NR) % (KC / 8));
        const int64_t ch = e / (NR * (KC / 8));
        const int64_t J = ch / nc;
        const int c = (int)(ch % nc);
        float d[8][8];                               // [source][digit]
        const int ex = r < nr ? scale_exp(xmax[r]) : 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t jl = (int64_t)KC * c + 8 * kb + q;
            if (r < nr && jl < n) {
                digits8(ldexp(v[J * n + jl + N * (r0 + r)], -ex), d[q]);
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) d[q][t] = 0.f;
            }
        }
#pragma unroll
        for (int t = 0; t < SX; ++t) {
            uint4 w;
            w.x = pack2(d[0][t], d[1][t]);
            w.y = pack2(d[2][t], d[3][t]);
            w.z = pack2(d[4][t], d[5][t]);
            w.w = pack2(d[6][t], d[7][t]);
            XB[((ch * SX + t) * (KC / 8) + kb) * 8 + r] = w;
        }
    }
}

// ---- the tensor-core sum ----------------------------------------------------

struct TcConvArgs {
    const __nv_bfloat16* R;     // mirrored table digit rows
    const uint4* XB;            // source digit chunks
    const unsigned long long* tmax;
    const unsigned long long* xmax;   // NR entries
    double* ybuf;               // N x nrhs, grid order
    int64_t N;
    int n;
    int64_t lines;              // n^(dim-1)
    int dim;
    int nb, nc;                 // target tiles / source chunks per line
    int64_t tiles;
    int r0, nr;
    int* status;
};

__global__ void __launch_bounds__(256, 1) tc_conv_kernel(TcConvArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    Bars* bars = (Bars*)(smem + NST * STAGE);
    volatile int* abort = &bars->abort;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NST; ++i) {
            tc::mbar_init(&bars->full[i], NBUILD + 1);
            tc::mbar_init(&bars->mma_done[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&bars->acc_full[i], 1);
            tc::mbar_init(&bars->acc_empty[i], 128);
        }
        tc::mbar_init(&bars->drain, 1);
        bars->abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&bars->tmem, 2 * ACC);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = bars->tmem;

    const int64_t cpt = a.lines * a.nc;                    // chunks per tile
    const int64_t my_tiles = a.tiles > blockIdx.x ? (a.tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t my_chunks = my_tiles * cpt;
    const int64_t Z0 = 128LL * a.nc - 1, RL = 256LL * a.nc;

    // line offset index of a (target line, source line) pair
    auto dline = [&](int64_t L, int64_t J) -> int64_t {
        if (a.dim == 2) return L > J ? L - J : J - L;
        const int64_t i0 = L / a.n, i1 = L % a.n, j0 = J / a.n, j1 = J % a.n;
        return (i0 > j0 ? i0 - j0 : j0 - i0) + (int64_t)a.n * (i1 > j1 ? i1 - j1 : j1 - i1);
    };

    if (warp == 4) {
        // ------------------------------------------------ issuer / B loader
        if (lane == 0) {
            int64_t issued_loads = 0, consumed = 0;
            auto load_B = [&](int64_t gc) {
                const int st = (int)(gc % NST);
                const int64_t ch = gc % cpt;                            // = J * nc + c
                unsigned char* dst = smem + st * STAGE + A_BYTES;
                tc::mbar_arrive_expect_tx(&bars->full[st], B_BYTES);
                tc::bulk_g2s(dst, (const unsigned char*)a.XB + ch * (int64_t)B_BYTES, B_BYTES, &bars->full[st]);
                ++issued_loads;
            };
            const int64_t pre = my_chunks < NST - 1 ? my_chunks : NST - 1;
            for (int64_t gc = 0; gc < pre; ++gc) load_B(gc);
            int64_t G = 0;
            uint32_t buf = 0;
            bool ok = true;
            for (int64_t gc = 0; gc < my_chunks && ok; ++gc) {
                const int st = (int)(gc % NST);
                const uint32_t use = (uint32_t)(gc / NST);
                const int64_t ci = gc % cpt;
                const bool first = ci % GROUP == 0;
                const bool last = ci % GROUP == GROUP - 1 || ci == cpt - 1;
                if (first) {
                    buf = (uint32_t)(G & 1);
                    if (G >= 2 && !wait_bounded(&bars->acc_empty[buf], (uint32_t)(((G >> 1) - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                }
                if (!wait_bounded(&bars->full[st], use & 1, abort)) {
                    ok = false;
                    break;
                }
                ++consumed;
                tc::tc_fence_after();
                // descriptors of the stage; moving the start address by 16 B
                // adds 1 to the descriptor (addresses stay below 256 KB)
                const uint32_t a_st = tc::smem_addr(smem + st * STAGE);
                const uint64_t a0 = tc::sdesc(a_st, 128, 128);
                const uint64_t b0 = tc::sdesc(a_st + A_BYTES, 128, (KC / 8) * 128);
#pragma unroll 1
                for (int kk = 0; kk < KC / 16; ++kk) {
                    const uint64_t bdesc = b0 + (uint64_t)(16 * kk);
                    const bool accum = !(first && kk == 0);
#pragma unroll
                    for (int s = 0; s < ST; ++s)
                        tc::mma_bf16(tmem + buf * ACC + coloff(s), a0 + (uint64_t)((s * A_SLICE) / 16 + 16 * kk), bdesc,
                                     tc::idesc_bf16_f32(TM, ncols(s)), accum);
                }
                tc::mma_commit(&bars->mma_done[st]);
                if (last) {
                    tc::mma_commit(&bars->acc_full[buf]);
                    ++G;
                }
                const int64_t nx = gc + NST - 1;
                if (nx < my_chunks) {
                    if (gc >= 1 && !wait_bounded(&bars->mma_done[(gc - 1) % NST], (uint32_t)(((gc - 1) / NST) & 1),
                                                 abort)) {
                        ok = false;
                        break;
                    }
                    load_B(nx);
                }
            }
            // drain: every MMA issued so far, then every bulk copy not consumed
            tc::mma_commit(&bars->drain);
            const long long t0 = clock64();
            while (!tc::mbar_try_wait(&bars->drain, 0) && clock64() - t0 < WAIT_CYCLES) {}
            for (int64_t gc = consumed; gc < issued_loads; ++gc) {
                const int st = (int)(gc % NST);
                const long long t1 = clock64();
                while (!tc::mbar_try_wait(&bars->full[st], (uint32_t)((gc / NST) & 1)) && clock64() - t1 < WAIT_CYCLES) {}
            }
            if (!ok) *abort = 1;
        }
    } else if (warp >= 5) {
        // ------------------------------------------------------- builders
        const int bt = threadIdx.x - 160;
        for (int64_t gc = 0; gc < my_chunks; ++gc) {
            const int st = (int)(gc % NST);
            const uint32_t use = (uint32_t)(gc / NST);
            if (use > 0 && !wait_bounded(&bars->mma_done[st], (use - 1) & 1, abort)) break;
            const int64_t tile = blockIdx.x + (gc / cpt) * gridDim.x;
            const int64_t L = tile / a.nb;
            const int b = (int)(tile % a.nb);
            const int64_t ci = gc % cpt;
            const int64_t J = ci / a.nc;
            const int c = (int)(ci % a.nc);
            const int64_t dl = dline(L, J);
            const int64_t base = (int64_t)TM * b + TM - 1 - (int64_t)KC * c;
            const int64_t idx0 = Z0 - base;                         // multiple of 8
            unsigned char* a_st = smem + st * STAGE;
            for (int pr = bt; pr < NPAIR; pr += NBUILD) {
                const int s = pr / NBLK, m = pr % NBLK;
                const uint4* src = reinterpret_cast<const uint4*>(a.R + ((int64_t)s * a.lines + dl) * RL + idx0 + 8 * m);
                const uint4 lo = __ldg(src), hi = __ldg(src + 1);
                const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
                uint4* dst = reinterpret_cast<uint4*>(a_st + s * A_SLICE + m * 128);
#pragma unroll
                for (int rho = 0; rho < 8; ++rho) {
                    uint32_t o[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        o[j] = (rho & 1) ? __funnelshift_r(w[rho / 2 + j], w[rho / 2 + j + 1], 16) : w[rho / 2 + j];
                    dst[rho] = make_uint4(o[0], o[1], o[2], o[3]);
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&bars->full[st]);
        }
    } else if (warp < 4) {
        // ------------------------------------------------------- epilogue
        long long acc[8][NR];
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[k][r] = 0;
        const int ngr = (int)((cpt + GROUP - 1) / GROUP);
        const int eT = scale_exp(*a.tmax);
        int64_t G = 0;
        bool ok = true;
        for (int64_t it = 0; it < my_tiles && ok; ++it) {
            const int64_t tile = blockIdx.x + it * gridDim.x;
            for (int g = 0; g < ngr; ++g, ++G) {
                const uint32_t buf = (uint32_t)(G & 1);
                if (!wait_bounded(&bars->acc_full[buf], (uint32_t)((G >> 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(32 * warp) << 16) + buf * ACC;
#pragma unroll
                for (int cb = 0; cb < ACC / 16; ++cb) {
                    float v[16];
                    tc::tmem_ld16(tbase + 16 * cb, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        acc[col_class(16 * cb + i)][col_rhs(16 * cb + i)] += (long long)__float2int_rn(v[i]);
                }
                tc::tc_fence_before();
                tc::mbar_arrive(&bars->acc_empty[buf]);
            }
            if (!ok) break;
            const int64_t L = tile / a.nb;
            const int b = (int)(tile % a.nb);
            const int il = TM * b + TM - 1 - (32 * warp + lane);
            if (il < a.n) {
                const int64_t gpos = L * a.n + il;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (r < a.nr) {
                        double y = 0.0, w = 1.0 / 72057594037927936.0;          // 2^-56
#pragma unroll
                        for (int k = 7; k >= 0; --k, w *= 256.0) y += (double)acc[k][r] * w;
                        a.ybuf[gpos + a.N * (a.r0 + r)] = ldexp(y, eT + scale_exp(a.xmax[r]) - 16);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[k][r] = 0;
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && bars->abort) atomicExch(a.status, 1);
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 2 * ACC);
    }
}

// ---- host side ----------------------------------------------------------------

size_t tc_table_rows_bytes(int n, int dim) {
    const int nc = (n + KC - 1) / KC;
    const int64_t lines = dim == 2 ? (int64_t)n : (int64_t)n * n;
    return sizeof(__nv_bfloat16) * (size_t)ST * lines * 256 * nc;
}

size_t tc_source_digits_bytes(int n, int dim) {
    const int nc = (n + KC - 1) / KC;
    const int64_t lines = dim == 2 ? (int64_t)n : (int64_t)n * n;
    return (size_t)lines * nc * B_BYTES;
}

cudaError_t launch_tc_table(const double* table, int n, int dim, unsigned long long* tmax, void* R,
                            cudaStream_t st) {
    const int nc = (n + KC - 1) / KC;
    const int64_t lines = dim == 2 ? (int64_t)n : (int64_t)n * n;
    const int64_t tot = lines * n;
    cudaError_t e = cudaMemsetAsync(tmax, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    note_launch();
    tc_maxabs_kernel<<<(int)std::min<int64_t>((tot + 255) / 256, 1024), 256, 0, st>>>(table, tot, 1, tot, tmax);
    note_launch();
    const int64_t rows = lines * 256LL * nc;
    tc_table_rows_kernel<<<(int)std::min<int64_t>((rows + 255) / 256, 152 * 16), 256, 0, st>>>(
        table, n, lines, nc, tmax, (__nv_bfloat16*)R);
    return cudaGetLastError();
}

cudaError_t launch_direct_grid_tc(const GridDirectArgs& a, const void* R, const unsigned long long* tmax,
                                  void* XB, unsigned long long* xmax, int* status, int num_sms, cudaStream_t st) {
    const int64_t N = a.dim == 2 ? (int64_t)a.n * a.n : (int64_t)a.n * a.n * a.n;
    if (N == 0) return cudaSuccess;
    const int nc = (a.n + KC - 1) / KC, nb = (a.n + TM - 1) / TM;
    const int64_t lines = a.dim == 2 ? (int64_t)a.n : (int64_t)a.n * a.n;
    const int eb = (int)std::min<int64_t>((N * a.nrhs + 255) / 256, 152 * 16);
    static bool attr_set = false;
    const size_t smem = (size_t)NST * STAGE + sizeof(Bars) + 1024;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tc_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    grid_scatter_kernel_launch(a, N, eb, st);
    for (int r0 = 0; r0 < a.nrhs; r0 += NR) {
        const int nr = std::min(NR, a.nrhs - r0);
        cudaError_t e = cudaMemsetAsync(xmax, 0, NR * sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        note_launch();
        tc_maxabs_kernel<<<(int)std::min<int64_t>((N + 255) / 256, 1024), 256, 0, st>>>(a.vbuf + N * r0, N, nr, N,
                                                                                       xmax);
        const int64_t items = lines * nc * (KC / 8) * NR;
        note_launch();
        tc_source_digits_kernel<<<(int)std::min<int64_t>((items + 255) / 256, 152 * 16), 256, 0, st>>>(
            a.vbuf, N, a.n, lines, nc, r0, nr, xmax, (uint4*)XB);
        TcConvArgs t{};
        t.R = (const __nv_bfloat16*)R;
        t.XB = (const uint4*)XB;
        t.tmax = tmax;
        t.xmax = xmax;
        t.ybuf = a.ybuf;
        t.N = N;
        t.n = a.n;
        t.lines = lines;
        t.dim = a.dim;
        t.nb = nb;
        t.nc = nc;
        t.tiles = lines * nb;
        t.r0 = r0;
        t.nr = nr;
        t.status = status;
        const int grid = (int)std::min<int64_t>(t.tiles, num_sms);
        note_launch();
        tc_conv_kernel<<<grid, 256, smem, st>>>(t);
    }
    grid_finish_kernel_launch(a, N, eb, st);
    return cudaGetLastError();
}

}  // namespace hif
