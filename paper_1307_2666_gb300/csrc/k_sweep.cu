// Apply / solve sweeps of the factorization in factored form (sm_103a).
//
// F^{-1} = V_0 ... V_last D^{-1} U_last^T ... U_0^T and F = U_0^{-T} ... D ...
// V_0^{-1} (Eqs. (3.2), (4.1), (4.2)).  One launch per sublevel and direction,
// one CTA per box: the box's skeleton and redundant entries of the working
// vectors are gathered into shared memory, the box's small factors (T, L, U,
// X, Y, D of Lemmas 2.1 and 2.3) are streamed once from HBM, and the result
// is scattered back.  Boxes of one sublevel touch disjoint DOFs.  The
// diagonal D^{-1} (or D) is fused into the sweep that last touches a box's
// redundant DOFs.
#include <algorithm>

#include "hif_common.cuh"
#include "launch.h"

namespace hif {

enum SweepMode {
    SOLVE_UP = 0, SOLVE_DOWN = 1, APPLY_UP = 2, APPLY_DOWN = 3,
    SOLVET_UP = 4, SOLVET_DOWN = 5, APPLYT_UP = 6, APPLYT_DOWN = 7
};

namespace {

// out (p x nr) += s * op(M) in, op(M) p x q; M column-major with leading dim ld.
template <typename T>
__device__ void mv(T* out, int p, const T* in, int q, const T* M, int64_t ld, bool trans, T s, int nr) {
    if (!trans) {
        for (int e = threadIdx.x; e < p * nr; e += blockDim.x) {
            const int i = e % p, c = e / p;
            T acc = T(0);
            for (int l = 0; l < q; ++l) acc += M[i + ld * l] * in[l + q * c];
            out[i + p * c] += s * acc;
        }
    } else {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int e = wid; e < p * nr; e += nw) {
            const int i = e % p, c = e / p;
            T acc = T(0);
            for (int l = lane; l < q; l += 32) acc += M[l + ld * i] * in[l + q * c];
            acc = warp_sum(acc);
            if (lane == 0) out[i + p * c] += s * acc;
        }
    }
    __syncthreads();
}

// out = (I + strict triangle of op(M)) in, n x nr.  lowerStore: the strict
// part sits in M's lower triangle (else upper); trans: op(M) = M^T.
template <typename T>
__device__ void tri(T* out, const T* in, int n, const T* M, int64_t ld, bool lowerStore, bool trans, int nr) {
    for (int e = threadIdx.x; e < n * nr; e += blockDim.x) {
        const int i = e % n, c = e / n;
        T acc = in[i + n * c];
        // op(M)[i,l] = trans ? M[l,i] : M[i,l]; nonzero for l<i if op is lower
        const bool opLower = lowerStore != trans;
        if (opLower) {
            for (int l = 0; l < i; ++l) acc += (trans ? M[l + ld * i] : M[i + ld * l]) * in[l + n * c];
        } else {
            for (int l = i + 1; l < n; ++l) acc += (trans ? M[l + ld * i] : M[i + ld * l]) * in[l + n * c];
        }
        out[i + n * c] = acc;
    }
    __syncthreads();
}

template <typename T>
__device__ void permute(T* out, const T* in, int n, const int* perm, bool inverse, int nr) {
    for (int e = threadIdx.x; e < n * nr; e += blockDim.x) {
        const int i = e % n, c = e / n;
        if (!inverse) out[i + n * c] = in[perm[i] + n * c];      // P x
        else out[perm[i] + n * c] = in[i + n * c];               // P^T x
    }
    __syncthreads();
}

template <typename T>
__device__ void copyv(T* out, const T* in, int cnt) {
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) out[e] = in[e];
    __syncthreads();
}

template <typename T>
__device__ void scale_rows(T* v, const T* D, int n, bool divide, int nr) {
    for (int e = threadIdx.x; e < n * nr; e += blockDim.x) {
        const int i = e % n;
        v[e] = divide ? v[e] / D[i] : v[e] * D[i];
    }
    __syncthreads();
}

}  // namespace

// For an LDL box (symmetric A, Sec. 5: P B_rr P^T = L D L^T, U = L^T P,
// Y = X^T) the box's factors are symmetric, so the transposed operation of a
// pass is the pass itself: solve_down = solve^T_down, solve^T_up = solve_up,
// apply_up = apply^T_up, apply^T_down = apply_down.  Those four bodies read
// only T, X, D, the permutation and L or L^{-1} (packed in one array: L in the
// strict lower triangle, L^{-1} transposed in the strict upper one).
__host__ __device__ constexpr int ldl_mode(int m) {
    return m == SOLVE_DOWN ? SOLVET_DOWN : m == SOLVET_UP ? SOLVE_UP : m == APPLY_UP ? APPLYT_UP
         : m == APPLYT_DOWN ? APPLY_DOWN : m;
}

template <typename T, int MODE>
__device__ void sweep_box(const BoxFac& bf, const T* pool, const int* perm, T* xs, T* xr, T* tmp, int nr) {
    const int k = bf.k, r = bf.r;
    const bool ldl = bf.ldl != 0;
    const T* Tm = pool + bf.T_off;
    const T* LU = pool + bf.LU_off;
    const T* LUi = pool + bf.LUi_off;
    const T* D = pool + bf.D_off;
    const T* X = pool + bf.X_off;
    const T* Y = pool + bf.Y_off;
    if (MODE == SOLVE_UP) {                 // U^T: Q^T then R^T
        mv<T>(xr, r, xs, k, Tm, k, true, T(-1), nr);
        permute<T>(tmp, xr, r, perm, false, nr);
        // L^{-1}: strict lower of LUi (LU box) or transposed in the upper (LDL box)
        tri<T>(xr, tmp, r, LUi, r, !ldl, ldl, nr);
        mv<T>(xs, k, xr, r, X, k, false, T(-1), nr);
    } else if (MODE == SOLVE_DOWN) {        // D^{-1} then V = Q S
        scale_rows<T>(xr, D, r, true, nr);
        mv<T>(xr, r, xs, k, Y, r, false, T(-1), nr);
        copyv<T>(tmp, xr, r * nr);
        tri<T>(xr, tmp, r, LUi, r, false, false, nr);
        mv<T>(xs, k, xr, r, Tm, k, false, T(-1), nr);
    } else if (MODE == APPLY_UP) {          // V^{-1} = S^{-1} Q^{-1}, then D
        mv<T>(xs, k, xr, r, Tm, k, false, T(1), nr);
        copyv<T>(tmp, xr, r * nr);
        tri<T>(xr, tmp, r, LU, r, false, false, nr);
        mv<T>(xr, r, xs, k, Y, r, false, T(1), nr);
        scale_rows<T>(xr, D, r, false, nr);
    } else if (MODE == APPLY_DOWN) {        // U^{-T} = Q^{-T} R^{-T}
        mv<T>(xs, k, xr, r, X, k, false, T(1), nr);
        tri<T>(tmp, xr, r, LU, r, true, false, nr);
        permute<T>(xr, tmp, r, perm, true, nr);
        mv<T>(xr, r, xs, k, Tm, k, true, T(1), nr);
    } else if (MODE == SOLVET_UP) {         // V^T = S^T Q^T
        mv<T>(xr, r, xs, k, Tm, k, true, T(-1), nr);
        copyv<T>(tmp, xr, r * nr);
        tri<T>(xr, tmp, r, LUi, r, false, true, nr);
        mv<T>(xs, k, xr, r, Y, r, true, T(-1), nr);
    } else if (MODE == SOLVET_DOWN) {       // D^{-T} then U = Q R
        scale_rows<T>(xr, D, r, true, nr);
        mv<T>(xr, r, xs, k, X, k, true, T(-1), nr);
        // L^{-T}: strict lower of LUi transposed (LU box) or the upper as stored (LDL box)
        tri<T>(tmp, xr, r, LUi, r, !ldl, !ldl, nr);
        permute<T>(xr, tmp, r, perm, true, nr);
        mv<T>(xs, k, xr, r, Tm, k, false, T(-1), nr);
    } else if (MODE == APPLYT_UP) {         // U^{-1} = R^{-1} Q^{-1}, then D
        mv<T>(xs, k, xr, r, Tm, k, false, T(1), nr);
        permute<T>(tmp, xr, r, perm, false, nr);
        tri<T>(xr, tmp, r, LU, r, true, true, nr);
        mv<T>(xr, r, xs, k, X, k, true, T(1), nr);
        scale_rows<T>(xr, D, r, false, nr);
    } else {                                // APPLYT_DOWN: V^{-T} = Q^{-T} S^{-T}
        mv<T>(xs, k, xr, r, Y, r, true, T(1), nr);
        copyv<T>(tmp, xr, r * nr);
        tri<T>(xr, tmp, r, LU, r, false, true, nr);
        mv<T>(xr, r, xs, k, Tm, k, true, T(1), nr);
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(512) sweep_kernel(SweepArgs a) {
    const BoxFac bf = a.boxes[blockIdx.x];
    const int k = bf.k, r = bf.r, nr = a.nrhs;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xs = a.gws ? static_cast<T*>(a.gws) + a.gws_off[blockIdx.x] * nr : reinterpret_cast<T*>(smem_raw);
    T* xr = xs + (size_t)k * nr;
    T* tmp = xr + (size_t)r * nr;
    T* x = static_cast<T*>(a.x);
    const int* sk = a.sk_ids + bf.sk_off;
    const int* rd = a.rd_ids + bf.rd_off;
    const T* pool = static_cast<const T*>(a.pool);
    const int* perm = a.perm + bf.piv_off;

    for (int e = threadIdx.x; e < k * nr; e += blockDim.x) xs[e] = x[sk[e % k] + a.ldx * (e / k)];
    for (int e = threadIdx.x; e < r * nr; e += blockDim.x) xr[e] = x[rd[e % r] + a.ldx * (e / r)];
    __syncthreads();

    if (bf.ldl) sweep_box<T, ldl_mode(MODE)>(bf, pool, perm, xs, xr, tmp, nr);
    else sweep_box<T, MODE>(bf, pool, perm, xs, xr, tmp, nr);

    for (int e = threadIdx.x; e < k * nr; e += blockDim.x) x[sk[e % k] + a.ldx * (e / k)] = xs[e];
    for (int e = threadIdx.x; e < r * nr; e += blockDim.x) x[rd[e % r] + a.ldx * (e / r)] = xr[e];
}

// Largest dynamic shared memory of any sweep launch: the callers batch the
// right-hand sides so that (k + 2 r) * nrhs * sizeof(T) <= 200 KB.
constexpr size_t kSweepSmemMax = 200 * 1024 + 64;

template <typename T, int MODE>
static cudaError_t launch_mode(const SweepArgs& a, int nbox, int threads, size_t smem, cudaStream_t st) {
    if (smem > kSweepSmemMax) return cudaErrorInvalidValue;
    // The kernel's dynamic shared-memory limit is only ever raised, to the
    // one fixed ceiling: launches captured in a CUDA graph keep their own
    // sizes, and no later launch may lower the limit below what a captured
    // node needs.
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(sweep_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSweepSmemMax);
        if (e != cudaSuccess) return e;
    }
    note_launch();
    sweep_kernel<T, MODE><<<nbox, threads, smem, st>>>(a);
    return cudaGetLastError();
}

// The caller sizes a.nrhs so that (k + 2r) * nrhs * sizeof(T) fits; the
// dynamic shared memory is passed through a.mode's high bits.
template <typename T>
cudaError_t launch_sweep(const SweepArgs& a, int nbox, int threads, cudaStream_t st) {
    if (nbox == 0) return cudaSuccess;
    if (threads < 32 || threads > 512 || threads % 32) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(a.mode >> 8);
    switch (a.mode & 0xff) {
        case SOLVE_UP: return launch_mode<T, SOLVE_UP>(a, nbox, threads, smem, st);
        case SOLVE_DOWN: return launch_mode<T, SOLVE_DOWN>(a, nbox, threads, smem, st);
        case APPLY_UP: return launch_mode<T, APPLY_UP>(a, nbox, threads, smem, st);
        case APPLY_DOWN: return launch_mode<T, APPLY_DOWN>(a, nbox, threads, smem, st);
        case SOLVET_UP: return launch_mode<T, SOLVET_UP>(a, nbox, threads, smem, st);
        case SOLVET_DOWN: return launch_mode<T, SOLVET_DOWN>(a, nbox, threads, smem, st);
        case APPLYT_UP: return launch_mode<T, APPLYT_UP>(a, nbox, threads, smem, st);
        case APPLYT_DOWN: return launch_mode<T, APPLYT_DOWN>(a, nbox, threads, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_sweep<double>(const SweepArgs&, int, int, cudaStream_t);
template cudaError_t launch_sweep<float>(const SweepArgs&, int, int, cudaStream_t);

// ---- wide boxes: the same passes spread over the GPU ------------------------
//
// A box with k + r in the thousands keeps one CTA busy for its whole pass
// while the other SMs idle, so the wide boxes of a sublevel take their pass as
// a sequence of stage launches over (box, 64-row tile): gather, matrix-vector
// products with T, X, Y, the triangular products (I + strict op(M)) with the
// unit factors or their inverses, permutations, scatter.  Each box keeps its
// three vectors in a global work space: B0 = skeleton part (k x nr), B1 =
// redundant part (r x nr), B2 = a second redundant vector.  Right-hand sides
// go 16 at a time.  The stage order of every mode is that of sweep_box.

namespace {

constexpr int WR = 16;      // right-hand sides per stage launch

template <typename T>
struct WideView {
    int k, r;
    T* B[3];
    int len[3];
    __device__ WideView(const WideArgs& a, int e, const BoxFac& bf) {
        k = bf.k;
        r = bf.r;
        T* base = static_cast<T*>(a.ws) + a.ws_off[e] * (int64_t)a.nr;
        B[0] = base;
        B[1] = base + (int64_t)k * a.nr;
        B[2] = B[1] + (int64_t)r * a.nr;
        len[0] = k;
        len[1] = r;
        len[2] = r;
    }
};

template <typename T>
__device__ __forceinline__ const T* wide_mat(const WideArgs& a, const BoxFac& bf, int mat, int64_t& ld) {
    const T* pool = static_cast<const T*>(a.pool);
    switch (mat) {
        case 0: ld = bf.k; return pool + bf.T_off;       // T: k x r
        case 1: ld = bf.k; return pool + bf.X_off;       // X: k x r
        case 2: ld = bf.r; return pool + bf.Y_off;       // Y: r x k
        case 3: ld = bf.r; return pool + bf.LU_off;      // unit factors, r x r
        default: ld = bf.r; return pool + bf.LUi_off;    // their inverses, r x r
    }
}

}  // namespace

template <typename T>
__global__ void wide_gather_kernel(WideArgs a, int div_d) {
    const int e = blockIdx.y;
    const BoxFac bf = a.boxes[e];
    WideView<T> v(a, e, bf);
    const T* x = static_cast<const T*>(a.x);
    const int* sk = a.sk_ids + bf.sk_off;
    const int* rd = a.rd_ids + bf.rd_off;
    const T* D = static_cast<const T*>(a.pool) + bf.D_off;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)(v.k + v.r) * a.nr; q += stride) {
        const int c = (int)(q / (v.k + v.r)), i = (int)(q % (v.k + v.r));
        if (i < v.k) v.B[0][i + (int64_t)v.k * c] = x[sk[i] + a.ldx * c];
        else {
            const int j = i - v.k;
            const T val = x[rd[j] + a.ldx * c];
            v.B[1][j + (int64_t)v.r * c] = div_d ? val / D[j] : val;
        }
    }
}

template <typename T>
__global__ void wide_scatter_kernel(WideArgs a, int xr_buf, int mul_d) {
    const int e = blockIdx.y;
    const BoxFac bf = a.boxes[e];
    WideView<T> v(a, e, bf);
    T* x = static_cast<T*>(a.x);
    const int* sk = a.sk_ids + bf.sk_off;
    const int* rd = a.rd_ids + bf.rd_off;
    const T* D = static_cast<const T*>(a.pool) + bf.D_off;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)(v.k + v.r) * a.nr; q += stride) {
        const int c = (int)(q / (v.k + v.r)), i = (int)(q % (v.k + v.r));
        if (i < v.k) x[sk[i] + a.ldx * c] = v.B[0][i + (int64_t)v.k * c];
        else {
            const int j = i - v.k;
            const T val = v.B[xr_buf][j + (int64_t)v.r * c];
            x[rd[j] + a.ldx * c] = mul_d ? val * D[j] : val;
        }
    }
}

// out = P in (inverse 0: out[i] = in[perm[i]]) or P^T in (out[perm[i]] = in[i])
template <typename T>
__global__ void wide_perm_kernel(WideArgs a, int out_buf, int in_buf, int inverse) {
    const int e = blockIdx.y;
    const BoxFac bf = a.boxes[e];
    WideView<T> v(a, e, bf);
    const int* perm = a.perm + bf.piv_off;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)v.r * a.nr; q += stride) {
        const int c = (int)(q / v.r), i = (int)(q % v.r);
        const int64_t o = (int64_t)v.r * c;
        if (!inverse) v.B[out_buf][i + o] = v.B[in_buf][perm[i] + o];
        else v.B[out_buf][perm[i] + o] = v.B[in_buf][i + o];
    }
}

// One product stage on rows [64 blockIdx.x, +64) of `out` for every wide box:
//   tri 0: out += s op(M) in                      (M = T, X or Y)
//   tri 1: out  = in' + strict op(M) in'          (M = LU or LUi; in' = P in
//          with perm_in, else in), opLower = lower_store != trans
// op(M)[i, l] = trans ? M[l + ld i] : M[i + ld l].  Not transposed: a thread
// per output row (coalesced column reads of M), the input staged in shared
// memory 64 rows at a time; transposed: a warp per output row (coalesced
// reads of column i of M) with warp reductions.
template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) wide_mv_kernel(WideArgs a, int out_buf, int in_buf, int mat, T s, int tri,
                                                      int lower_store, int perm_in) {
    const int e = blockIdx.y;
    const BoxFac bf = a.boxes[e];
    WideView<T> v(a, e, bf);
    const int p = v.len[out_buf], q = v.len[in_buf];
    const int i0 = blockIdx.x * 64;
    if (i0 >= p) return;
    int64_t ld;
    const T* M = wide_mat<T>(a, bf, mat, ld);
    const int* perm = a.perm + bf.piv_off;
    T* out = v.B[out_buf];
    const T* in = v.B[in_buf];
    const int nr = a.nr;
    const bool opLower = (lower_store != 0) != TRANS;
    auto inval = [&](int l, int c) -> T { return in[(perm_in ? perm[l] : l) + (int64_t)q * c]; };
    if (!TRANS) {
        __shared__ T ins[64][WR + 1];
        const int tx = threadIdx.x % 64, tc = threadIdx.x / 64;      // rhs tc, tc + 4, ...
        const int i = i0 + tx;
        T acc[WR / 4];
#pragma unroll
        for (int u = 0; u < WR / 4; ++u) acc[u] = T(0);
        // tri: only l < i (opLower) or l > i contribute
        const int lbeg = tri && !opLower ? i0 + 1 : 0;
        const int lend = tri && opLower ? min(q, i0 + 64) : q;
        for (int l0 = lbeg; l0 < lend; l0 += 64) {
            __syncthreads();
            for (int z = threadIdx.x; z < 64 * WR; z += 256) {
                const int ll = z % 64, c = z / 64;
                ins[ll][c] = (l0 + ll < lend && c < nr) ? inval(l0 + ll, c) : T(0);
            }
            __syncthreads();
            if (i < p) {
                const int cnt = min(64, lend - l0);
                for (int ll = 0; ll < cnt; ++ll) {
                    const int l = l0 + ll;
                    if (tri && (opLower ? l >= i : l <= i)) continue;
                    const T m = M[i + ld * l];
#pragma unroll
                    for (int u = 0; u < WR / 4; ++u) acc[u] += m * ins[ll][tc + 4 * u];
                }
            }
        }
        if (i < p)
#pragma unroll
            for (int u = 0; u < WR / 4; ++u) {
                const int c = tc + 4 * u;
                if (c >= nr) continue;
                T* o = out + i + (int64_t)p * c;
                if (tri) *o = inval(i, c) + acc[u];
                else *o += s * acc[u];
            }
    } else {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int ii = w; ii < 64; ii += 8) {
            const int i = i0 + ii;
            if (i >= p) break;
            const T* col = M + ld * i;
            T acc[WR];
#pragma unroll
            for (int c = 0; c < WR; ++c) acc[c] = T(0);
            const int lbeg = tri && !opLower ? i + 1 : 0;
            const int lend = tri && opLower ? i : q;
            for (int l = lbeg + lane; l < lend; l += 32) {
                const T m = col[l];
#pragma unroll
                for (int c = 0; c < WR; ++c)
                    if (c < nr) acc[c] += m * inval(l, c);
            }
#pragma unroll
            for (int c = 0; c < WR; ++c) acc[c] = warp_sum(acc[c]);
            if (lane < nr) {
                T val = T(0);
#pragma unroll
                for (int c = 0; c < WR; ++c)
                    if (c == lane) val = acc[c];
                T* o = out + i + (int64_t)p * lane;
                if (tri) *o = inval(i, lane) + val;
                else *o += s * val;
            }
        }
    }
}

template <typename T>
static cudaError_t wide_mv(const WideArgs& a, int nwide, int rows, int out_buf, int in_buf, int mat, bool trans,
                           T s, int tri, int lower_store, int perm_in, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const dim3 g((rows + 63) / 64, nwide);
    note_launch();
    if (trans) wide_mv_kernel<T, true><<<g, 256, 0, st>>>(a, out_buf, in_buf, mat, s, tri, lower_store, perm_in);
    else wide_mv_kernel<T, false><<<g, 256, 0, st>>>(a, out_buf, in_buf, mat, s, tri, lower_store, perm_in);
    return cudaGetLastError();
}

// The pass of `mode` for the wide boxes; a.nr <= 16 right-hand sides.
template <typename T>
cudaError_t launch_wide_sweep(const WideArgs& a, int nwide, int max_k, int max_r, int mode, cudaStream_t st) {
    if (nwide == 0) return cudaSuccess;
    if (a.nr < 1 || a.nr > WR) return cudaErrorInvalidValue;
    const dim3 ge((unsigned)std::min<int64_t>(((int64_t)(max_k + max_r) * a.nr + 255) / 256, 256), nwide);
    const dim3 gp((unsigned)std::min<int64_t>(((int64_t)max_r * a.nr + 255) / 256, 256), nwide);
    cudaError_t err = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (err == cudaSuccess) err = x; };
    auto mv = [&](int rows, int ob, int ib, int mat, bool tr, T sg) { chk(wide_mv<T>(a, nwide, rows, ob, ib, mat, tr, sg, 0, 0, 0, st)); };
    auto tri = [&](int ob, int ib, int mat, bool lower_store, bool tr, bool pin) {
        chk(wide_mv<T>(a, nwide, max_r, ob, ib, mat, tr, T(1), 1, lower_store ? 1 : 0, pin ? 1 : 0, st));
    };
    auto perm = [&](int ob, int ib, bool inv) {
        note_launch();
        wide_perm_kernel<T><<<gp, 256, 0, st>>>(a, ob, ib, inv ? 1 : 0);
        chk(cudaGetLastError());
    };
    auto gather = [&](bool divd) {
        note_launch();
        wide_gather_kernel<T><<<ge, 256, 0, st>>>(a, divd ? 1 : 0);
        chk(cudaGetLastError());
    };
    auto scatter = [&](int xr_buf, bool muld) {
        note_launch();
        wide_scatter_kernel<T><<<ge, 256, 0, st>>>(a, xr_buf, muld ? 1 : 0);
        chk(cudaGetLastError());
    };
    enum { MT = 0, MX = 1, MY = 2, MLU = 3, MLUI = 4 };
    switch (mode) {
        case SOLVE_UP:        // xr -= T^T xs; xr <- L^{-1} P xr; xs -= X xr
            gather(false);
            mv(max_r, 1, 0, MT, true, T(-1));
            tri(2, 1, MLUI, true, false, true);
            mv(max_k, 0, 2, MX, false, T(-1));
            scatter(2, false);
            break;
        case SOLVE_DOWN:      // xr /= D; xr -= Y xs; xr <- U'^{-1} xr; xs -= T xr
            gather(true);
            mv(max_r, 1, 0, MY, false, T(-1));
            tri(2, 1, MLUI, false, false, false);
            mv(max_k, 0, 2, MT, false, T(-1));
            scatter(2, false);
            break;
        case APPLY_UP:        // xs += T xr; xr <- U' xr; xr += Y xs; xr *= D
            gather(false);
            mv(max_k, 0, 1, MT, false, T(1));
            tri(2, 1, MLU, false, false, false);
            mv(max_r, 2, 0, MY, false, T(1));
            scatter(2, true);
            break;
        case APPLY_DOWN:      // xs += X xr; xr <- P^T L xr; xr += T^T xs
            gather(false);
            mv(max_k, 0, 1, MX, false, T(1));
            tri(2, 1, MLU, true, false, false);
            perm(1, 2, true);
            mv(max_r, 1, 0, MT, true, T(1));
            scatter(1, false);
            break;
        case SOLVET_UP:       // xr -= T^T xs; xr <- U'^{-T} xr; xs -= Y^T xr
            gather(false);
            mv(max_r, 1, 0, MT, true, T(-1));
            tri(2, 1, MLUI, false, true, false);
            mv(max_k, 0, 2, MY, true, T(-1));
            scatter(2, false);
            break;
        case SOLVET_DOWN:     // xr /= D; xr -= X^T xs; xr <- P^T L^{-T} xr; xs -= T xr
            gather(true);
            mv(max_r, 1, 0, MX, true, T(-1));
            tri(2, 1, MLUI, true, true, false);
            perm(1, 2, true);
            mv(max_k, 0, 1, MT, false, T(-1));
            scatter(1, false);
            break;
        case APPLYT_UP:       // xs += T xr; xr <- L^T P xr; xr += X^T xs; xr *= D
            gather(false);
            mv(max_k, 0, 1, MT, false, T(1));
            tri(2, 1, MLU, true, true, true);
            mv(max_r, 2, 0, MX, true, T(1));
            scatter(2, true);
            break;
        case APPLYT_DOWN:     // xs += Y^T xr; xr <- U'^T xr; xr += T^T xs
            gather(false);
            mv(max_k, 0, 1, MY, true, T(1));
            tri(2, 1, MLU, false, true, false);
            mv(max_r, 2, 0, MT, true, T(1));
            scatter(2, false);
            break;
        default: return cudaErrorInvalidValue;
    }
    return err;
}

template cudaError_t launch_wide_sweep<double>(const WideArgs&, int, int, int, int, cudaStream_t);
template cudaError_t launch_wide_sweep<float>(const WideArgs&, int, int, int, int, cudaStream_t);

// ---------------------------------------------------- precision moves ----

template <typename T>
__global__ void to_work_kernel(const double* src, int64_t lds, T* dst, int64_t ldd, int64_t N, int nrhs) {
    const int64_t tot = N * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % N, c = e / N;
        dst[i + ldd * c] = (T)src[i + lds * c];
    }
}

template <typename T>
__global__ void from_work_kernel(const T* src, int64_t lds, double* dst, int64_t ldd, int64_t N, int nrhs) {
    const int64_t tot = N * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % N, c = e / N;
        dst[i + ldd * c] = (double)src[i + lds * c];
    }
}

template <typename T>
cudaError_t launch_to_work(const double* src, int64_t lds, T* dst, int64_t ldd, int64_t N, int nrhs, cudaStream_t st) {
    const int64_t tot = N * nrhs;
    if (tot == 0) return cudaSuccess;
    const int blocks = (int)((tot + 255) / 256 < 152 * 16 ? (tot + 255) / 256 : 152 * 16);
    note_launch();
    to_work_kernel<T><<<blocks, 256, 0, st>>>(src, lds, dst, ldd, N, nrhs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_from_work(const T* src, int64_t lds, double* dst, int64_t ldd, int64_t N, int nrhs, cudaStream_t st) {
    const int64_t tot = N * nrhs;
    if (tot == 0) return cudaSuccess;
    const int blocks = (int)((tot + 255) / 256 < 152 * 16 ? (tot + 255) / 256 : 152 * 16);
    note_launch();
    from_work_kernel<T><<<blocks, 256, 0, st>>>(src, lds, dst, ldd, N, nrhs);
    return cudaGetLastError();
}

template cudaError_t launch_to_work<double>(const double*, int64_t, double*, int64_t, int64_t, int, cudaStream_t);
template cudaError_t launch_to_work<float>(const double*, int64_t, float*, int64_t, int64_t, int, cudaStream_t);
template cudaError_t launch_from_work<double>(const double*, int64_t, double*, int64_t, int64_t, int, cudaStream_t);
template cudaError_t launch_from_work<float>(const float*, int64_t, double*, int64_t, int64_t, int, cudaStream_t);

}  // namespace hif
