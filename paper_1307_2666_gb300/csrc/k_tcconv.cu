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
// Products of digit pairs (s, t) of the same class k = s + t carry the same
// weight 2^(eT + eX - 8(k + 2)), so they share one accumulator column: the
// MMA of table digit s writes the columns of classes s .. s + t_max.  A
// column then sums at most 8 pairs x 128 sources = 1024 products per slot
// (<= 2^24, exact in FP32); every slot's columns are converted to integers
// and added into 64-bit integer class sums, so the only rounding is the
// dropped digits (below 2^-55 of max|t| max|v|) and the final FP64
// combination of eight class sums.  Table digits 0..6 and source digits
// 0..7 are kept, and pairs with s + t >= 8 are not formed.
//
// Shorter digit sets serve the residuals of the refinement that are not the
// last one (their error only enters the next correction, which the last,
// full-digit residual then measures): with KD classes (4, 5 or 6) the kernel
// keeps table and source digits 0..KD-1 and the pairs with s + t < KD.  Per
// term the dropped part is below (KD + 1) 2^(-2 - 8 KD) of 2^(eT + eX) <= 16
// max|t| max|v|, and it behaves like a sum of independent terms of mean zero
// (round-to-nearest digits): on the 2D log-kernel grid with Gaussian sources
// the relative error of y is ~6e-9 with KD = 4, ~2e-11 with KD = 5 and ~1e-13
// with KD = 6, at every N from 4096 to 262144 (exact integer convolutions of
// the digits).
//
// On a grid K_ij depends only on the offset i - j, so the kernel block of a
// tile of 128 targets on one grid line against 128 sources on another line is
// a Toeplitz matrix in the last coordinate.  With the target rows taken in
// reverse order it is a Hankel matrix A[i][q] = v[i + q], whose 8 x 8 core
// matrices depend only on the sum of their block indices: the shared-memory
// operand stores the 31 distinct core matrices of each digit slice once and
// the MMA descriptor walks them with equal leading and stride offsets (144 B:
// a 16-B gap after every core matrix keeps the builders' stores free of
// shared-memory bank conflicts).
//
// The block also depends only on |offset| along the slowest axis, so the
// source lines at -d and +d from a target line share it, and so do the two
// target lines i0 and i0 + 1 of a tile with their sources at i0 +- d and
// i0 + 1 +- d: one MMA takes the four source chunks as the four quarters of
// its B operand (rows ordered digit, quarter, rhs), so N = 32 per source
// digit.  An M = 128 MMA reads its 4 KB A operand from shared memory whatever
// N is, and shared-memory bandwidth (128 B per clock) bounds the MMAs of
// small N: the four-chunk operand takes the A reads per target line to half
// those of one line with its mirror pair.  A missing source line reads a
// zero chunk.
//
// CTA roles (384 threads, persistent, one CTA per SM, TMEM 512 columns):
//   warps 0-7  epilogue: TMEM -> integer class sums -> FP64 y (one thread
//              per target row; warps 0-3 the first line, 4-7 the second),
//   warp 8     one thread: the MMAs,
//   warps 9-11 builders of the Hankel operand from mirrored digit rows; one
//              of them also issues the bulk copies of the source digits.
// Slots (one Hankel operand, four 128-source chunks) flow through a 2-stage
// shared-memory ring (3 stages for the short sums, whose stages are smaller)
// into two 256-column accumulators used in turn, so the
// MMAs of the next slot proceed while the epilogue drains one.  The class
// sums are kept as an int64 for class 0 and int32 for classes 1..7, and
// every 32 slots the carries of classes 7..1 move up (c = s_k >> 8, s_k -=
// 256 c, s_(k-1) += c), which keeps their value and their range.  Every wait
// is bounded; on time-out the kernel sets *status = 1, drains its own MMAs
// and copies, frees TMEM and returns.
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <utility>
#include <vector>
#include <cstdint>
#include "hif_types.h"
#include "launch.h"
#include "tc_ptx.cuh"

namespace hif {
namespace {

constexpr int TM = 128;                         // targets per tile (TMEM lanes)
constexpr int KC = 128;                         // sources per chunk
constexpr int ST = 7;                           // table digits stored
constexpr int SX = 8;                           // source digits stored per chunk
constexpr int NR = 8;                           // right-hand sides per launch
constexpr int NBLK = (TM + KC) / 8 - 1;         // distinct Hankel core matrices per slice (31)
constexpr int CM = 144;                         // core-matrix stride: 128 B + 16 B so that the
                                                // builders' 16-B row stores of consecutive core
                                                // matrices fall in different bank groups
constexpr int A_SLICE = NBLK * CM;              // bytes
constexpr int CHUNK = SX * NR * KC * 2;         // one source chunk: (digit, rhs) rows x KC, BF16
constexpr int TBLK = NR * KC * 2;               // the rows of one digit of one chunk
constexpr int NL = 2;                           // target lines per tile
constexpr int NQ = 2 * NL;                      // source chunks per slot (mirror pair per target line)
constexpr int NST_MAX = 3;                      // deepest ring of the variants below
constexpr int ACCB = 32 * 8;                    // TMEM columns of one accumulator: (class, quarter, rhs)
constexpr int NACC = 2;                         // accumulators, used slot by slot in turn
constexpr int ACC = ACCB * NACC;                // TMEM columns allocated
constexpr int NEPI = 256;                       // epilogue threads
constexpr int NBUILD = 96;                      // builder threads
constexpr int NTHR = NEPI + 32 + NBUILD;
constexpr int CARRY = 32;                       // slots between carry passes of the class sums
constexpr long long WAIT_CYCLES = 4000000000LL; // ~2 s at GB300 clocks

static_assert(8 * KC * 128 * 128 <= (1 << 24), "exact FP32 accumulation of one slot");
// a class sum gains at most 2 columns x 7 pairs x 128 sources x 2^14 per slot
static_assert(2.0 * 7 * KC * 16384 * CARRY + 2.0 * 16777216 < 2147483647.0, "int32 class sums between carries");

// The variant with KD digit classes (8: every class, the full sum; 4, 5 or
// 6: the short sums).  Columns of table digit s: B rows (source digit t,
// quarter, rhs) for t below nt(s) = ncols(s) / 32, written to the accumulator
// columns (class s + t, quarter, rhs), i.e. from column 32 s on; the full sum
// takes s + t <= 7 except for the odd counts rounded down, a short one every
// pair with s + t < KD.
template <int KD>
struct Digits {
    static constexpr int ST = KD == 8 ? 7 : KD;          // table digits read
    static constexpr int SX = KD;                        // source digits read
    static constexpr int A_BYTES = ST * A_SLICE;
    static constexpr int B_BYTES = NQ * SX * TBLK;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int NST = KD == 8 ? 2 : 3;         // ring depth within 227 KB of shared memory
    static constexpr int NPAIR = ST * NBLK;             // (slice, core matrix) build items per slot
    __host__ __device__ static constexpr int ncols(int s) {
        return KD == 8 ? (s == 0 ? 256 : s <= 2 ? 192 : s <= 4 ? 128 : 64) : 32 * (KD - s);
    }
    static_assert(STAGE % 16 == 0 && A_BYTES % 16 == 0 && TBLK % 16 == 0, "stage alignment");
    static_assert(NST <= NST_MAX && NST * STAGE + 1024 + 256 <= 232448, "shared memory");
    static_assert(ncols(0) == 32 * KD && ncols(ST - 1) >= 32, "column map");
};
__host__ __device__ constexpr int coloff(int s) { return 32 * s; }
static_assert(coloff(6) + Digits<8>::ncols(6) <= ACCB && Digits<8>::ncols(0) == ACCB, "column map");

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
    uint64_t full[NST_MAX];     // Hankel operand built (NBUILD arrivals)
    uint64_t bfull[NST_MAX];    // source digits landed (1 arrival + bytes)
    uint64_t mma_done[NST_MAX];
    uint64_t acc_full[NACC];    // accumulator written (1 commit)
    uint64_t acc_empty[NACC];   // accumulator drained (128 epilogue arrivals)
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
                                        int sx, const unsigned long long* xmax, uint4* XB) {
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
            if (t >= sx) break;
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
    const unsigned char* XB;    // source digit chunks, then one zero chunk
    const unsigned long long* tmax;
    const unsigned long long* xmax;   // NR entries
    double* ybuf;               // N x nrhs, grid order
    int64_t N;
    int n;
    int64_t lines;              // n^(dim-1)
    int dim;
    int nb, nc;                 // target chunks / source chunks per line
    int64_t tiles;              // (line pair, target chunk)
    int r0, nr;
    int* status;
    int stall;                  // test of the bounded waits: issue no MMA at all
};

namespace {

// The slot sequence of one CTA, identical in every role: its tiles
// (round-robin; a tile is the target lines i0 = 2 p and i0 + 1 along the
// slowest axis, the middle coordinate i1 in 3D, and one chunk b along the
// last), and per tile the offsets d0 = 0..dmax along the slowest axis, the
// middle source coordinate j1 (3D), the chunk c.
struct Walk {
    int n, dim, nb, nc;
    int64_t tiles, step, tile;
    int b, i0, i1, dmax, d0, j1, c;
    bool ok;

    __device__ void init(const TcConvArgs& a, int64_t first, int64_t stride) {
        n = a.n; dim = a.dim; nb = a.nb; nc = a.nc; tiles = a.tiles; step = stride; tile = first;
        ok = tile < tiles;
        if (ok) start();
    }
    __device__ void start() {
        const int64_t p = tile / nb;
        b = (int)(tile % nb);
        i0 = 2 * (dim == 2 ? (int)p : (int)(p / n));
        i1 = dim == 2 ? 0 : (int)(p % n);
        dmax = i0 > n - 1 - i0 ? i0 : n - 1 - i0;
        if (i0 + 1 < n && i0 + 1 > dmax) dmax = i0 + 1;
        d0 = 0; j1 = 0; c = 0;
    }
    // line index (all but the last coordinate) of target line l, -1 if none
    __device__ int64_t line(int l) const {
        const int il = i0 + l;
        if (il >= n) return -1;
        return dim == 2 ? (int64_t)il : (int64_t)il * n + i1;
    }
    __device__ int64_t slots() const { return (int64_t)(dmax + 1) * (dim == 3 ? n : 1) * nc; }
    __device__ void next() {
        if (++c < nc) return;
        c = 0;
        if (dim == 3 && ++j1 < n) return;
        j1 = 0;
        if (++d0 <= dmax) return;
        tile += step;
        ok = tile < tiles;
        if (ok) start();
    }
    // offset index of the line pair (all but the last coordinate)
    __device__ int64_t dl() const { return d0 + (dim == 3 ? (int64_t)n * (i1 > j1 ? i1 - j1 : j1 - i1) : 0); }
    // source line of quarter q = 2 l + h (target line i0 + l; h = 0: minus
    // d0, h = 1: plus d0), -1 if none
    __device__ int64_t src_line(int q) const {
        const int il = i0 + (q >> 1), h = q & 1;
        if (il >= n || (h == 1 && d0 == 0)) return -1;
        const int j0 = h == 0 ? il - d0 : il + d0;
        if (j0 < 0 || j0 >= n) return -1;
        return dim == 2 ? (int64_t)j0 : (int64_t)j0 * n + j1;
    }
};

}  // namespace

template <int KD>
__global__ void __launch_bounds__(NTHR, 1) tc_conv_kernel(TcConvArgs a) {
    using C = Digits<KD>;
    constexpr int NST = C::NST, STAGE = C::STAGE, A_BYTES = C::A_BYTES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    Bars* bars = (Bars*)(smem + NST * STAGE);
    volatile int* abort = &bars->abort;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NST; ++i) {
            tc::mbar_init(&bars->full[i], NBUILD);
            tc::mbar_init(&bars->bfull[i], 1);
            tc::mbar_init(&bars->mma_done[i], 1);
        }
        for (int i = 0; i < NACC; ++i) {
            tc::mbar_init(&bars->acc_full[i], 1);
            tc::mbar_init(&bars->acc_empty[i], NEPI);
        }
        tc::mbar_init(&bars->drain, 1);
        bars->abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&bars->tmem, ACC);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = bars->tmem;
    const int64_t Z0 = 128LL * a.nc - 1, RL = 256LL * a.nc;
    const int64_t zero_chunk = a.lines * a.nc;

    if (warp == NEPI / 32) {
        // ---------------------------------------------------------- issuer
        // (counters are stepped, not divided, and the thread does nothing
        // but wait and issue: its scalar work between MMA batches shows up
        // as tensor-pipe idle time)
        if (lane == 0) {
            Walk w;
            w.init(a, a.stall ? a.tiles : (int64_t)blockIdx.x, gridDim.x);
            int st = 0;
            uint32_t ph = 0;
            int64_t si = 0;                      // slots issued: accumulator si % NACC, use si / NACC
            bool ok = true;
            while (w.ok) {
                const int ab = (int)(si % NACC);
                const int64_t use = si / NACC;
                if (use >= 1 && !wait_bounded(&bars->acc_empty[ab], (uint32_t)((use - 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                if (!wait_bounded(&bars->full[st], ph, abort) || !wait_bounded(&bars->bfull[st], ph, abort)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                // descriptors of the stage; moving the start address by 16 B
                // adds 1 to the descriptor (addresses stay below 256 KB)
                const uint32_t a_st = tc::smem_addr(smem + st * STAGE);
                const uint64_t a0 = tc::sdesc(a_st, CM, CM);
                const uint64_t b0 = tc::sdesc(a_st + A_BYTES, 128, (KC / 8) * 128);
                // slice by slice: consecutive MMAs of one slice read
                // overlapping Hankel windows and keep N and D fixed, which
                // the tensor core streams faster than alternating slices
                // (the first MMA, slice 0 with N = 128, initializes all the
                // accumulator's columns; the others add into theirs)
#pragma unroll
                for (int s = 0; s < C::ST; ++s) {
                    const uint64_t as = a0 + (uint64_t)(s * A_SLICE / 16);
                    const uint32_t d = tmem + ACCB * ab + coloff(s);
#pragma unroll
                    for (int kk = 0; kk < KC / 16; ++kk)
                        tc::mma_bf16(d, as + (uint64_t)(2 * CM * kk / 16), b0 + (uint64_t)(16 * kk),
                                     tc::idesc_bf16_f32(TM, C::ncols(s)), !(s == 0 && kk == 0));
                }
                tc::mma_commit(&bars->mma_done[st]);
                tc::mma_commit(&bars->acc_full[ab]);
                ++si;
                w.next();
                if (++st == NST) {
                    st = 0;
                    ph ^= 1;
                }
            }
            // drain: every MMA issued so far
            tc::mma_commit(&bars->drain);
            const long long t0 = clock64();
            while (!tc::mbar_try_wait(&bars->drain, 0) && clock64() - t0 < WAIT_CYCLES) {}
            if (!ok) *abort = 1;
        }
    } else if (warp > NEPI / 32) {
        // ------------------------------------------------------- builders
        // each thread owns up to PPT (slice, core matrix) items per slot; the
        // 16 digits of every item are fetched one slot ahead, so the L2
        // latency overlaps the build of the current slot
        constexpr int NPAIR = C::NPAIR;
        constexpr int PPT = (NPAIR + NBUILD - 1) / NBUILD;
        const int bt = threadIdx.x - (NEPI + 32);
        uint4 cur[PPT][2], nxt[PPT][2];
        auto fetch = [&](const Walk& v, uint4 (&buf)[PPT][2]) {
            const int64_t dl = v.dl();
            const int64_t idx0 = Z0 - ((int64_t)TM * v.b + TM - 1 - (int64_t)KC * v.c);   // multiple of 8
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int pr = bt + NBUILD * j;
                if (pr < NPAIR) {
                    const int s = pr / NBLK, m = pr % NBLK;
                    const uint4* src =
                        reinterpret_cast<const uint4*>(a.R + ((int64_t)s * a.lines + dl) * RL + idx0 + 8 * m);
                    buf[j][0] = __ldg(src);
                    buf[j][1] = __ldg(src + 1);
                }
            }
        };
        Walk w, wn;
        w.init(a, blockIdx.x, gridDim.x);
        wn = w;
        if (w.ok) {
            fetch(w, cur);
            wn.next();
        }
        int st = 0;
        uint32_t ph = 0;
        int64_t gs = 0, issued = 0;
        while (w.ok) {
            if (wn.ok) fetch(wn, nxt);
            if (gs >= NST && !wait_bounded(&bars->mma_done[st], ph ^ 1, abort)) break;
            unsigned char* a_st = smem + st * STAGE;
            if (bt == 0) {
                // source digits of the four chunks, digit block by digit
                // block into rows (digit, quarter, rhs); a missing line reads zeros
                tc::mbar_arrive_expect_tx(&bars->bfull[st], C::B_BYTES);
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const int64_t J = w.src_line(q);
                    const int64_t chunk = J >= 0 ? J * a.nc + w.c : zero_chunk;
                    const unsigned char* src = a.XB + chunk * (int64_t)CHUNK;
#pragma unroll
                    for (int t = 0; t < C::SX; ++t)
                        tc::bulk_g2s(a_st + A_BYTES + (NQ * t + q) * TBLK, src + t * TBLK, TBLK, &bars->bfull[st]);
                }
                ++issued;
            }
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int pr = bt + NBUILD * j;
                if (pr < NPAIR) {
                    const int s = pr / NBLK, m = pr % NBLK;
                    const uint32_t wd[8] = {cur[j][0].x, cur[j][0].y, cur[j][0].z, cur[j][0].w,
                                            cur[j][1].x, cur[j][1].y, cur[j][1].z, cur[j][1].w};
                    uint4* dst = reinterpret_cast<uint4*>(a_st + s * A_SLICE + m * CM);
#pragma unroll
                    for (int rho = 0; rho < 8; ++rho) {
                        uint32_t o[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            o[q] = (rho & 1) ? __funnelshift_r(wd[rho / 2 + q], wd[rho / 2 + q + 1], 16)
                                             : wd[rho / 2 + q];
                        dst[rho] = make_uint4(o[0], o[1], o[2], o[3]);
                    }
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&bars->full[st]);
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                cur[j][0] = nxt[j][0];
                cur[j][1] = nxt[j][1];
            }
            w = wn;
            if (wn.ok) wn.next();
            ++gs;
            if (++st == NST) {
                st = 0;
                ph ^= 1;
            }
        }
        // drain: the latest copy into every stage has landed before exit
        if (bt == 0)
            for (int64_t i = issued > NST ? issued - NST : 0; i < issued; ++i) {
                const long long t1 = clock64();
                while (!tc::mbar_try_wait(&bars->bfull[i % NST], (uint32_t)((i / NST) & 1)) &&
                       clock64() - t1 < WAIT_CYCLES) {}
            }
    } else {
        // ------------------------------------------------------- epilogue
        // warp w: target line w / 4 of the tile, TMEM lane quarter w % 4
        const int ln = warp >> 2, quad = warp & 3;
        long long s0[NR];          // class 0
        int sk[KD - 1][NR];        // classes 1..KD-1
        auto carry = [&]() {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
#pragma unroll
                for (int k = KD - 2; k >= 1; --k) {
                    const int c = sk[k][r] >> 8;
                    sk[k][r] -= c * 256;
                    sk[k - 1][r] += c;
                }
                const int c = sk[0][r] >> 8;
                sk[0][r] -= c * 256;
                s0[r] += c;
            }
        };
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            s0[r] = 0;
#pragma unroll
            for (int k = 0; k < KD - 1; ++k) sk[k][r] = 0;
        }
        const int eT = scale_exp(*a.tmax);
        int64_t si = 0;                                        // slots drained
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < a.tiles && ok; tile += gridDim.x) {
            Walk w;
            w.init(a, tile, a.tiles);                          // this tile only
            const int64_t nsl = w.slots();
            for (int64_t g = 0; g < nsl; ++g, ++si) {
                const int ab = (int)(si % NACC);
                if (!wait_bounded(&bars->acc_full[ab], (uint32_t)((si / NACC) & 1), abort)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                // class k of this line: columns 32 k + 16 ln + (h, rhs)
                const uint32_t tbase = tmem + ACCB * ab + 16 * ln + ((uint32_t)(32 * quad) << 16);
#pragma unroll
                for (int k = 0; k < KD; ++k) {
                    float v[16];
                    tc::tmem_ld16(tbase + 32 * k, v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        if (k == 0) s0[e % 8] += (long long)__float2int_rn(v[e]);
                        else sk[k - 1][e % 8] += __float2int_rn(v[e]);
                    }
                }
                tc::tc_fence_before();
                tc::mbar_arrive(&bars->acc_empty[ab]);
                if (g % CARRY == CARRY - 1) carry();
            }
            if (!ok) break;
            carry();
            const int il = TM * w.b + TM - 1 - (32 * quad + lane);
            const int64_t L = w.line(ln);
            if (il < a.n && L >= 0) {
                const int64_t gpos = L * a.n + il;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (r < a.nr) {
                        double y = 0.0, wt = ldexp(1.0, -8 * (KD - 1));
#pragma unroll
                        for (int k = KD - 1; k >= 1; --k, wt *= 256.0) y += (double)sk[k - 1][r] * wt;
                        y += (double)s0[r];
                        a.ybuf[gpos + a.N * (a.r0 + r)] = ldexp(y, eT + scale_exp(a.xmax[r]) - 16);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                s0[r] = 0;
#pragma unroll
                for (int k = 0; k < KD - 1; ++k) sk[k][r] = 0;
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && bars->abort) atomicExch(a.status, 1);
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, ACC);
    }
}

// ---- host side ----------------------------------------------------------------

namespace {
std::mutex g_tm_mu;
bool g_tm_on = false;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_tm_ev;
}  // namespace

void tc_timing_set(bool enable) {
    std::lock_guard<std::mutex> lk(g_tm_mu);
    g_tm_on = enable;
}

cudaError_t tc_timing_collect(double* ms, int64_t* launches) {
    std::lock_guard<std::mutex> lk(g_tm_mu);
    double tot = 0.0;
    cudaError_t err = cudaSuccess;
    for (auto& e : g_tm_ev) {
        float t = 0.f;
        cudaError_t r = cudaEventSynchronize(e.second);
        if (r == cudaSuccess) r = cudaEventElapsedTime(&t, e.first, e.second);
        if (r != cudaSuccess && err == cudaSuccess) err = r;
        tot += t;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    if (ms) *ms = tot;
    if (launches) *launches = (int64_t)g_tm_ev.size();
    g_tm_ev.clear();
    return err;
}

size_t tc_table_rows_bytes(int n, int dim) {
    const int nc = (n + KC - 1) / KC;
    const int64_t lines = dim == 2 ? (int64_t)n : (int64_t)n * n;
    return sizeof(__nv_bfloat16) * (size_t)ST * lines * 256 * nc;
}

size_t tc_source_digits_bytes(int n, int dim) {
    const int nc = (n + KC - 1) / KC;
    const int64_t lines = dim == 2 ? (int64_t)n : (int64_t)n * n;
    return (size_t)(lines * nc + 1) * CHUNK;                 // + one zero chunk
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

namespace {
// the kernel variant of KD digit classes and its shared-memory size (the
// opt-in above 48 KB is set once per variant)
template <int KD>
cudaError_t tc_variant(void (**fn)(TcConvArgs), size_t* smem) {
    static bool attr_set = false;
    *fn = tc_conv_kernel<KD>;
    *smem = (size_t)Digits<KD>::NST * Digits<KD>::STAGE + sizeof(Bars) + 1024;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tc_conv_kernel<KD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)*smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t launch_direct_grid_tc(const GridDirectArgs& a, const void* R, const unsigned long long* tmax,
                                  void* XB, unsigned long long* xmax, int* status, int num_sms, int classes,
                                  cudaStream_t st) {
    const int64_t N = a.dim == 2 ? (int64_t)a.n * a.n : (int64_t)a.n * a.n * a.n;
    if (N == 0) return cudaSuccess;
    if (classes < 4 || classes == 7 || classes > 8) return cudaErrorInvalidValue;
    const int nc = (a.n + KC - 1) / KC, nb = (a.n + TM - 1) / TM;
    const int64_t lines = a.dim == 2 ? (int64_t)a.n : (int64_t)a.n * a.n;
    const int eb = (int)std::min<int64_t>((N * a.nrhs + 255) / 256, 152 * 16);
    void (*kfn)(TcConvArgs) = nullptr;
    size_t smem = 0;
    {
        cudaError_t e = classes == 8   ? tc_variant<8>(&kfn, &smem)
                        : classes == 6 ? tc_variant<6>(&kfn, &smem)
                        : classes == 5 ? tc_variant<5>(&kfn, &smem)
                                       : tc_variant<4>(&kfn, &smem);
        if (e != cudaSuccess) return e;
    }
    grid_scatter_kernel_launch(a, N, eb, st);
    {
        cudaError_t e = cudaMemsetAsync((unsigned char*)XB + lines * nc * (int64_t)CHUNK, 0, CHUNK, st);
        if (e != cudaSuccess) return e;
    }
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
            a.vbuf, N, a.n, lines, nc, r0, nr, classes, xmax, (uint4*)XB);
        TcConvArgs t{};
        t.R = (const __nv_bfloat16*)R;
        t.XB = (const unsigned char*)XB;
        t.tmax = tmax;
        t.xmax = xmax;
        t.ybuf = a.ybuf;
        t.N = N;
        t.n = a.n;
        t.lines = lines;
        t.dim = a.dim;
        t.nb = nb;
        t.nc = nc;
        t.tiles = (a.dim == 2 ? (int64_t)((a.n + 1) / 2) : (int64_t)((a.n + 1) / 2) * a.n) * nb;
        t.r0 = r0;
        t.nr = nr;
        t.status = status;
        {
            // test of the bounded waits (HIF_TC_TEST_STALL=1): the MMA thread
            // issues nothing, the builders' stage-reuse waits run out after
            // ~2 s and the call returns HIF_ETIMEOUT with the context intact
            const char* e = getenv("HIF_TC_TEST_STALL");
            t.stall = (e && atoi(e) != 0) ? 1 : 0;
        }
        const int grid = (int)std::min<int64_t>(t.tiles, num_sms);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_tm_mu);
            if (g_tm_on && classes == 8 && cudaEventCreate(&e0) == cudaSuccess &&
                cudaEventCreate(&e1) == cudaSuccess) {
                cudaEventRecord(e0, st);
                g_tm_ev.emplace_back(e0, e1);
            } else {
                e1 = nullptr;
            }
        }
        note_launch();
        kfn<<<grid, NTHR, smem, st>>>(t);
        if (e1) cudaEventRecord(e1, st);
    }
    grid_finish_kernel_launch(a, N, eb, st);
    return cudaGetLastError();
}

}  // namespace hif
