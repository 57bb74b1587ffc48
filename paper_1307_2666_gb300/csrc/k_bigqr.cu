// Unpivoted blocked Householder QR of the proxy matrices of large boxes
// (sm_103a), the first stage of their interpolative decomposition.
//
// The ID of Y_c[:, g] (Lemma 2.2, column-pivoted QR to tolerance rho_g eps)
// is the ID of R[:, g] for Y_c = Q R with Q orthonormal: column norms, pivots
// and T = R11^{-1} R12 are the same in exact arithmetic.  A large box's Y_c
// is tall (m = 2 (near-field + proxy) rows, often 10-30 x its n columns), so
// it is first reduced to its n x n factor R here, with BLAS-3 updates; the
// pivoted QR (k_large.cu) then works on R instead of Y_c.
//
// Opt-in (environment HIF_BIG_RFIRST=1).  Measured on GB300 it is slower than
// the per-pivot sweeps over the tall matrix (2D n = 1024 FP32 factorization
// 4.5 s against 2.5 s; 3D n = 64, eps 1e-3: 63 s against 44 s), although the
// FP32 factorization it gives is more accurate (one refinement step fewer):
// the full QR does m n^2 work where the pivoted QR stops at rank k ~ n / 2,
// the trailing updates run on the SIMT pipes, and the panel is one CTA per
// box, serial over its columns.  A multi-CTA panel and tensor-core trailing
// updates would be needed for it to pay.
//
// Panels of QB columns: the panel is factored column by column by one CTA
// per box (reductions accumulated in FP64), the compact-WY factor T of
// I - V T V^T is formed from the Gram matrix V^T V, and the trailing
// columns are updated as C -= V (T^T (V^T C)) in two row-split passes.  The
// row splits have a fixed size and their partial sums are added in a fixed
// order, so the result is reproducible and independent of the batch.  On
// return the upper triangle of Y[0:n, 0:n] holds R and its strict lower part
// is zero; boxes with m <= n are left untouched.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "hif_common.cuh"
#include "launch.h"

namespace hif {
namespace {

constexpr int QB = 16;          // panel width
constexpr int PT = 512;         // panel kernel threads
constexpr int WR = 64;          // rows per staged chunk (V^T C)
constexpr int WC = 64;          // columns per tile (V^T C, C -= V W)
constexpr int AR = 128;         // rows per tile (C -= V W)
constexpr int GROWS = 4096;     // rows per partial Gram (fixed, so sums do not depend on the batch)
constexpr int WROWS = 2048;     // rows per partial V^T C

// element (i, a) of the panel's reflectors: unit at row j0 + a, zero above
template <typename T>
__device__ __forceinline__ T vref(const T* Y, int64_t m, int j0, int i, int a) {
    const int c = j0 + a;
    return i == c ? T(1) : (i > c ? Y[i + m * c] : T(0));
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(PT) bqr_panel_kernel(BigQRArgs a, int j0) {
    const int b = blockIdx.x;
    const int m = a.m[b], n = a.n[b];
    if (m <= n || j0 >= n) return;
    const int nb = min(QB, n - j0);
    T* Y = static_cast<T*>(a.Y) + a.y_off[b];
    T* tau_out = static_cast<T*>(a.tau) + (int64_t)b * QB;
    __shared__ double part[PT / 32][QB];
    __shared__ double tot[QB];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = 0; c < nb; ++c) {
        const int jc = j0 + c;
        const int nq = nb - 1 - c;                 // panel columns right of jc
        T* v = Y + (int64_t)m * jc;
        // acc[0] = sum v_i^2, acc[1 + q] = sum v_i Y[i, jc + 1 + q], rows i > jc
        double acc[QB];
#pragma unroll
        for (int q = 0; q < QB; ++q) acc[q] = 0.0;
        for (int i = jc + 1 + threadIdx.x; i < m; i += PT) {
            const double vi = (double)v[i];
            acc[0] += vi * vi;
#pragma unroll
            for (int q = 0; q < QB - 1; ++q)
                if (q < nq) acc[1 + q] += vi * (double)Y[i + (int64_t)m * (jc + 1 + q)];
        }
#pragma unroll
        for (int q = 0; q < QB; ++q) {
            double s = acc[q];
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) part[wid][q] = s;
        }
        __syncthreads();
        if (threadIdx.x < QB) {
            double s = 0.0;
            for (int w = 0; w < PT / 32; ++w) s += part[w][threadIdx.x];
            tot[threadIdx.x] = s;
        }
        __syncthreads();
        const double ss = tot[0];
        const double alpha = (double)v[jc];
        double tau = 0.0, scal = 0.0, beta = alpha;
        if (ss != 0.0) {
            beta = -copysign(sqrt(alpha * alpha + ss), alpha);
            tau = (beta - alpha) / beta;
            scal = 1.0 / (alpha - beta);
        }
        // w_q = Y[jc, col] + scal * dot_q; column col -= tau w_q v
        for (int i = jc + 1 + threadIdx.x; i < m; i += PT) {
            const double vi = (double)v[i];
            v[i] = (T)(vi * scal);
#pragma unroll
            for (int q = 0; q < QB - 1; ++q)
                if (q < nq) {
                    T* col = Y + (int64_t)m * (jc + 1 + q);
                    const double wq = (double)col[jc] + scal * tot[1 + q];
                    col[i] = (T)((double)col[i] - tau * wq * scal * vi);
                }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 0; q < nq; ++q) {
                T* col = Y + (int64_t)m * (jc + 1 + q);
                const double wq = (double)col[jc] + scal * tot[1 + q];
                col[jc] = (T)((double)col[jc] - tau * wq);
            }
            v[jc] = (T)beta;
            tau_out[c] = (T)tau;
        }
        __syncthreads();
    }
}

// Partial G = V^T V of the panel's reflectors over rows [j0 + GROWS y,
// j0 + GROWS (y + 1)), FP64, one slot per (box, split); thread t handles the
// pair (t / QB, t % QB).  The slots are summed in order by bqr_gsum_kernel, so
// the result does not depend on how many boxes share the launch.
template <typename T>
__global__ void __launch_bounds__(QB * QB) bqr_gram_kernel(BigQRArgs a, int j0) {
    const int b = blockIdx.x;
    const int m = a.m[b], n = a.n[b];
    if (m <= n || j0 >= n) return;
    const int nb = min(QB, n - j0);
    const int r0 = j0 + blockIdx.y * GROWS;
    if (r0 >= m) return;
    const int r1 = min(m, r0 + GROWS);
    const T* Y = static_cast<const T*>(a.Y) + a.y_off[b];
    __shared__ T tile[QB * QB][QB + 1];
    const int pa = threadIdx.x / QB, pb = threadIdx.x % QB;
    double s = 0.0;
    for (int base = r0; base < r1; base += QB * QB) {
        __syncthreads();
        const int i = base + threadIdx.x;
#pragma unroll
        for (int q = 0; q < QB; ++q) tile[threadIdx.x][q] = (i < r1 && q < nb) ? vref(Y, m, j0, i, q) : T(0);
        __syncthreads();
        const int cnt = min(QB * QB, r1 - base);
        for (int r = 0; r < cnt; ++r) s += (double)tile[r][pa] * (double)tile[r][pb];
    }
    a.Gp[a.gp_off[b] + (int64_t)blockIdx.y * QB * QB + threadIdx.x] = s;
}

template <typename T>
__global__ void __launch_bounds__(QB * QB) bqr_gsum_kernel(BigQRArgs a, int j0) {
    const int b = blockIdx.x;
    const int m = a.m[b], n = a.n[b];
    if (m <= n || j0 >= n) return;
    const int ns = (m - j0 + GROWS - 1) / GROWS;
    double s = 0.0;
    for (int y = 0; y < ns; ++y) s += a.Gp[a.gp_off[b] + (int64_t)y * QB * QB + threadIdx.x];
    static_cast<double*>(a.G)[(int64_t)b * QB * QB + threadIdx.x] = s;
}

// T (upper triangular, column by column): T[c][c] = tau_c,
// T[0:c, c] = -tau_c T[0:c, 0:c] G[0:c, c].
template <typename T>
__global__ void bqr_tfac_kernel(BigQRArgs a, int j0) {
    const int b = blockIdx.x;
    const int m = a.m[b], n = a.n[b];
    if (m <= n || j0 >= n) return;
    const int nb = min(QB, n - j0);
    const double* G = static_cast<const double*>(a.G) + (int64_t)b * QB * QB;
    const T* tau = static_cast<const T*>(a.tau) + (int64_t)b * QB;
    T* Tf = static_cast<T*>(a.Tf) + (int64_t)b * QB * QB;
    __shared__ double Ts[QB][QB];
    const int r = threadIdx.x;
    if (r < QB)
        for (int c = 0; c < QB; ++c) Ts[r][c] = 0.0;
    __syncthreads();
    for (int c = 0; c < nb; ++c) {
        const double tc = (double)tau[c];
        double v = 0.0;
        if (r < c)
            for (int l = r; l < c; ++l) v += Ts[r][l] * G[l * QB + c];
        __syncthreads();
        if (r < c) Ts[r][c] = -tc * v;
        if (r == c) Ts[c][c] = tc;
        __syncthreads();
    }
    if (r < QB)
        for (int c = 0; c < QB; ++c) Tf[r * QB + c] = (T)Ts[r][c];
}

// W[a][col] += sum over this block's rows of V(i, a) Y[i, col], for the
// trailing columns col >= j0 + nb.
template <typename T>
__global__ void __launch_bounds__(256) bqr_w_kernel(BigQRArgs a, int j0) {
    const int b = blockIdx.x;
    const int m = a.m[b], n = a.n[b];
    if (m <= n || j0 >= n) return;
    const int nb = min(QB, n - j0);
    const int c0 = j0 + nb + blockIdx.y * WC;
    if (c0 >= n) return;
    const T* Y = static_cast<const T*>(a.Y) + a.y_off[b];
    const int r0 = j0 + blockIdx.z * WROWS;
    if (r0 >= m) return;
    const int r1 = min(m, r0 + WROWS);
    __shared__ T Vs[WR][QB + 1];
    __shared__ T Cs[WR][WC + 1];
    // thread t: reflector a = t / 16, columns (t % 16) + 16 k, k < 4
    const int ta = threadIdx.x / 16, tcol = threadIdx.x % 16;
    T acc[WC / 16] = {T(0), T(0), T(0), T(0)};     // in the factorization's precision
    for (int base = r0; base < r1; base += WR) {
        __syncthreads();
        for (int e = threadIdx.x; e < WR * QB; e += 256) {
            const int rr = e % WR, q = e / WR, i = base + rr;
            Vs[rr][q] = (i < r1 && q < nb) ? vref(Y, m, j0, i, q) : T(0);
        }
        for (int e = threadIdx.x; e < WR * WC; e += 256) {
            const int rr = e % WR, cc = e / WR, i = base + rr, col = c0 + cc;
            Cs[rr][cc] = (i < r1 && col < n) ? Y[i + (int64_t)m * col] : T(0);
        }
        __syncthreads();
        for (int rr = 0; rr < WR; ++rr) {
            const T va = Vs[rr][ta];
#pragma unroll
            for (int k = 0; k < WC / 16; ++k) acc[k] += va * Cs[rr][tcol + 16 * k];
        }
    }
    // slot of this row split: QB x n partial sums at wp_off[b] + split * QB * n
    double* Wp = a.Wp + a.wp_off[b] + (int64_t)blockIdx.z * QB * n;
#pragma unroll
    for (int k = 0; k < WC / 16; ++k) {
        const int col = c0 + tcol + 16 * k;
        if (col < n) Wp[(int64_t)ta * n + col] = ta < nb ? (double)acc[k] : 0.0;
    }
}

// W2 = T^T W for the trailing columns, W = the row-split slots summed in
// order; one thread per column.
template <typename T>
__global__ void bqr_wsum_kernel(BigQRArgs a, int j0) {
    const int b = blockIdx.y;
    const int m = a.m[b], n = a.n[b];
    if (m <= n || j0 >= n) return;
    const int nb = min(QB, n - j0);
    const int ns = (m - j0 + WROWS - 1) / WROWS;
    T* W2 = static_cast<T*>(a.W) + (int64_t)b * QB * a.wld;
    const double* Wp = a.Wp + a.wp_off[b];
    const T* Tf = static_cast<const T*>(a.Tf) + (int64_t)b * QB * QB;
    for (int col = j0 + nb + blockIdx.x * blockDim.x + threadIdx.x; col < n; col += gridDim.x * blockDim.x) {
        double w[QB];
#pragma unroll
        for (int q = 0; q < QB; ++q) w[q] = 0.0;
        for (int y = 0; y < ns; ++y)
#pragma unroll
            for (int q = 0; q < QB; ++q) w[q] += Wp[(int64_t)y * QB * n + (int64_t)q * n + col];
#pragma unroll
        for (int q = 0; q < QB; ++q) {
            double s = 0.0;
#pragma unroll
            for (int l = 0; l <= q; ++l) s += (double)Tf[l * QB + q] * w[l];
            W2[(int64_t)q * a.wld + col] = q < nb ? (T)s : T(0);
        }
    }
}

// C -= V (T^T W) on a tile of AR rows x WC trailing columns.
template <typename T>
__global__ void __launch_bounds__(256) bqr_apply_kernel(BigQRArgs a, int j0) {
    const int b = blockIdx.x;
    const int m = a.m[b], n = a.n[b];
    if (m <= n || j0 >= n) return;
    const int nb = min(QB, n - j0);
    const int c0 = j0 + nb + blockIdx.y * WC;
    const int r0 = j0 + blockIdx.z * AR;
    if (c0 >= n || r0 >= m) return;
    T* Y = static_cast<T*>(a.Y) + a.y_off[b];
    const T* W = static_cast<const T*>(a.W) + (int64_t)b * QB * a.wld;     // T^T V^T C
    __shared__ T W2[QB][WC];
    __shared__ T Vs[AR][QB + 1];
    for (int e = threadIdx.x; e < QB * WC; e += 256) {
        const int q = e / WC, cc = e % WC, col = c0 + cc;
        W2[q][cc] = (q < nb && col < n) ? W[(int64_t)q * a.wld + col] : T(0);
    }
    for (int e = threadIdx.x; e < AR * QB; e += 256) {
        const int rr = e % AR, q = e / AR, i = r0 + rr;
        Vs[rr][q] = (i < m && q < nb) ? vref(Y, m, j0, i, q) : T(0);
    }
    __syncthreads();
    const int rr = threadIdx.x % AR, i = r0 + rr;
    if (i >= m) return;
    for (int cc = threadIdx.x / AR; cc < WC; cc += 256 / AR) {
        const int col = c0 + cc;
        if (col >= n) break;
        T s = T(0);
#pragma unroll
        for (int q = 0; q < QB; ++q) s += Vs[rr][q] * W2[q][cc];
        Y[i + (int64_t)m * col] -= s;
    }
}

// zero the strict lower triangle of Y[0:n, 0:n] (it held reflectors)
template <typename T>
__global__ void bqr_clear_kernel(BigQRArgs a) {
    const int b = blockIdx.y;
    const int m = a.m[b], n = a.n[b];
    if (m <= n) return;
    T* Y = static_cast<T*>(a.Y) + a.y_off[b];
    const int64_t tot = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        if (i > j) Y[i + (int64_t)m * j] = T(0);
    }
}

size_t big_geqrf_partials(const int* m, const int* n, int nbox, std::vector<int64_t>& gp_off,
                          std::vector<int64_t>& wp_off, int64_t* wp_total) {
    int64_t g = 0, w = 0;
    gp_off.resize(nbox);
    wp_off.resize(nbox);
    for (int b = 0; b < nbox; ++b) {
        gp_off[b] = g;
        wp_off[b] = w;
        if (m[b] <= n[b]) continue;
        g += (int64_t)((m[b] + GROWS - 1) / GROWS) * QB * QB;
        w += (int64_t)((m[b] + WROWS - 1) / WROWS) * QB * n[b];
    }
    *wp_total = w;
    return (size_t)g;
}

template <typename T>
cudaError_t big_geqrf(const BigQRArgs& a, int nbox, int max_m, int max_n, cudaStream_t st) {
    if (nbox == 0) return cudaSuccess;
    const int gsplit = (max_m + GROWS - 1) / GROWS;
    const int wsplit = (max_m + WROWS - 1) / WROWS;
    for (int j0 = 0; j0 < max_n; j0 += QB) {
        note_launch();
        bqr_panel_kernel<T><<<nbox, PT, 0, st>>>(a, j0);
        note_launch();
        bqr_gram_kernel<T><<<dim3(nbox, gsplit), QB * QB, 0, st>>>(a, j0);
        note_launch();
        bqr_gsum_kernel<T><<<nbox, QB * QB, 0, st>>>(a, j0);
        note_launch();
        bqr_tfac_kernel<T><<<nbox, 32, 0, st>>>(a, j0);
        const int trail = max_n - j0 - QB;
        if (trail > 0) {
            const int ctiles = (trail + WC - 1) / WC;
            note_launch();
            bqr_w_kernel<T><<<dim3(nbox, ctiles, wsplit), 256, 0, st>>>(a, j0);
            note_launch();
            bqr_wsum_kernel<T><<<dim3(std::max(1, (trail + 127) / 128), nbox), 128, 0, st>>>(a, j0);
            const int rtiles = (max_m - j0 + AR - 1) / AR;
            note_launch();
            bqr_apply_kernel<T><<<dim3(nbox, ctiles, rtiles), 256, 0, st>>>(a, j0);
        }
    }
    note_launch();
    bqr_clear_kernel<T><<<dim3(std::min<int64_t>(((int64_t)max_n * max_n + 255) / 256, 1024), nbox), 256, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t big_geqrf<double>(const BigQRArgs&, int, int, int, cudaStream_t);
template cudaError_t big_geqrf<float>(const BigQRArgs&, int, int, int, cudaStream_t);

}  // namespace hif
