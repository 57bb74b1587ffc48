// Operator-level kernels (sm_103a): exact self-cell integrals, kernel-entry
// blocks, and the FP64 direct-sum matvec y = a.x + b.(K (c.x)) of Eq. (3.1)
// (and its transpose), plus the BLAS-1 helpers of the refinement loops.
//
// Two direct-sum variants, both exact sums over all N^2 pairs:
//  * general points: each CTA owns 128 targets and streams all sources
//    through shared memory; G(r) evaluated per pair.
//  * uniform tensor grids: K_ij = G(h |i - j|) w depends only on the integer
//    index offset, so the sum is a discrete convolution with a table of
//    n^dim values; each CTA owns a 256-target tile, stages a 256-source tile
//    and the matching window of the table in shared memory, and spends one
//    FP64 FMA per pair and right-hand side.
#include <algorithm>

#include "hif_common.cuh"
#include "launch.h"

namespace hif {

__global__ void kself_kernel(GeomDev g, double* kself) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N; i += (int64_t)gridDim.x * blockDim.x) {
        const double w = g.w[i];
        double v;
        if (g.kernel_id == 0) {
            // -(h^2 / 2 pi) (ln h - ln(2)/2 - 3/2 + pi/4), h = sqrt(w)
            const double h = sqrt(w);
            v = -(w / (2.0 * kPi)) * (log(h) - 0.5 * log(2.0) - 1.5 + 0.25 * kPi);
        } else {
            // (h^2 / 4 pi) (3 ln(2 + sqrt 3) - pi/2), h = w^(1/3)
            const double h = cbrt(w);
            v = (h * h / (4.0 * kPi)) * (3.0 * log(2.0 + sqrt(3.0)) - 0.5 * kPi);
        }
        kself[i] = v;
    }
}

cudaError_t launch_kself(const GeomDev& g, double* kself, cudaStream_t st) {
    if (g.N == 0) return cudaSuccess;
    note_launch();
    kself_kernel<<<(int)std::min<int64_t>((g.N + 255) / 256, 4096), 256, 0, st>>>(g, kself);
    return cudaGetLastError();
}

__global__ void kernel_block_kernel(GeomDev g, const int* rows, int64_t nr, const int* cols, int64_t nc,
                                    double* out, int64_t ldo) {
    const int64_t tot = nr * nc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e % nr, q = e / nr;
        const int i = rows[p], j = cols[q];
        double v;
        if (i == j) {
            v = g.a[i] + g.b[i] * g.kself[i] * g.c[i];
        } else {
            double r2 = 0.0;
            for (int d = 0; d < g.dim; ++d) {
                const double dd = g.x[(int64_t)g.dim * i + d] - g.x[(int64_t)g.dim * j + d];
                r2 += dd * dd;
            }
            v = g.b[i] * green_d(g.kernel_id, r2) * g.w[j] * g.c[j];
        }
        out[p + ldo * q] = v;
    }
}

cudaError_t launch_kernel_block(const GeomDev& g, const int* rows, int64_t nr, const int* cols, int64_t nc,
                                double* out, int64_t ldo, cudaStream_t st) {
    const int64_t tot = nr * nc;
    if (tot == 0) return cudaSuccess;
    note_launch();
    kernel_block_kernel<<<(int)std::min<int64_t>((tot + 255) / 256, 152 * 16), 256, 0, st>>>(g, rows, nr, cols, nc, out, ldo);
    return cudaGetLastError();
}

// ------------------------------------------------------- general points --

constexpr int DS_T = 128;   // targets per CTA (one per thread)
constexpr int DS_S = 256;   // sources per shared-memory tile
constexpr int DS_R = 8;     // right-hand sides per pass

__global__ void __launch_bounds__(DS_T) direct_general_kernel(DirectArgs a, int r0, int nr) {
    __shared__ double sx[DS_S * 3];
    __shared__ double sv[DS_S * DS_R];
    const GeomDev& g = a.g;
    const int dim = g.dim;
    const int64_t s_end = a.seg_off + a.seg_n;
    const int64_t i = a.seg_off + blockIdx.x * (int64_t)DS_T + threadIdx.x;
    const bool valid = i < s_end;
    double xi[3] = {0, 0, 0};
    if (valid)
        for (int d = 0; d < dim; ++d) xi[d] = g.x[(int64_t)dim * i + d];
    double acc[DS_R];
    for (int c = 0; c < DS_R; ++c) acc[c] = 0.0;
    for (int64_t j0 = a.seg_off; j0 < s_end; j0 += DS_S) {
        const int ns = (int)(s_end - j0 < DS_S ? s_end - j0 : DS_S);
        __syncthreads();
        for (int s = threadIdx.x; s < ns; s += DS_T) {
            const int64_t j = j0 + s;
            for (int d = 0; d < 3; ++d) sx[3 * s + d] = d < dim ? g.x[(int64_t)dim * j + d] : 0.0;
            const double sw = a.trans ? g.b[j] : g.w[j] * g.c[j];
            for (int c = 0; c < DS_R; ++c) sv[s * DS_R + c] = c < nr ? sw * a.x[j + a.ldx * (r0 + c)] : 0.0;
        }
        __syncthreads();
        if (valid) {
            for (int s = 0; s < ns; ++s) {
                const int64_t j = j0 + s;
                if (j == i) continue;
                const double d0 = xi[0] - sx[3 * s], d1 = xi[1] - sx[3 * s + 1], d2 = xi[2] - sx[3 * s + 2];
                const double gk = green_d(g.kernel_id, d0 * d0 + d1 * d1 + d2 * d2);
                for (int c = 0; c < DS_R; ++c) acc[c] += gk * sv[s * DS_R + c];
            }
        }
    }
    if (valid) {
        const double tf = a.trans ? g.c[i] * g.w[i] : g.b[i];
        const double self = g.b[i] * g.kself[i] * g.c[i] + g.a[i];
        for (int c = 0; c < nr; ++c)
            a.y[i + a.ldy * (r0 + c)] = tf * acc[c] + self * a.x[i + a.ldx * (r0 + c)];
    }
}

// Helmholtz kernel (kernel 2) on the real embedding: complex unknowns are the
// pairs of real DOFs (2p, 2p + 1), vectors interleave real and imaginary
// parts.  y = A x with A_pq = a_p delta_pq + b_p K_pq c_q, K_pq = G(r_pq) w_q
// (one-point rule), K_pp the self-cell integral; trans = 1 gives the adjoint
// A^H x (the transpose of the real embedding).  One thread per complex
// target, sources staged in shared memory; G is evaluated once per pair and
// used for every right-hand side.
constexpr int DH_R = 4;     // right-hand sides per pass

__global__ void __launch_bounds__(DS_T) direct_helmholtz_kernel(DirectArgs a, int r0, int nr) {
    __shared__ double sx[DS_S * 2];
    __shared__ double sv[DS_S * DH_R * 2];
    const GeomDev& g = a.g;
    const int64_t p_beg = a.seg_off / 2, p_end = (a.seg_off + a.seg_n) / 2;
    const int64_t p = p_beg + blockIdx.x * (int64_t)DS_T + threadIdx.x;
    const bool valid = p < p_end;
    const double conj_sign = a.trans ? -1.0 : 1.0;
    double xi0 = 0.0, xi1 = 0.0;
    if (valid) {
        xi0 = g.x[4 * p];
        xi1 = g.x[4 * p + 1];
    }
    double ar[DH_R], ai[DH_R];
    for (int c = 0; c < DH_R; ++c) ar[c] = ai[c] = 0.0;
    for (int64_t q0 = p_beg; q0 < p_end; q0 += DS_S) {
        const int ns = (int)(p_end - q0 < DS_S ? p_end - q0 : DS_S);
        __syncthreads();
        for (int s = threadIdx.x; s < ns; s += DS_T) {
            const int64_t q = q0 + s;
            sx[2 * s] = g.x[4 * q];
            sx[2 * s + 1] = g.x[4 * q + 1];
            const double sw = a.trans ? g.b[2 * q] : g.w[2 * q] * g.c[2 * q];
            for (int c = 0; c < DH_R; ++c) {
                const bool on = c < nr;
                sv[(s * DH_R + c) * 2] = on ? sw * a.x[2 * q + a.ldx * (r0 + c)] : 0.0;
                sv[(s * DH_R + c) * 2 + 1] = on ? sw * a.x[2 * q + 1 + a.ldx * (r0 + c)] : 0.0;
            }
        }
        __syncthreads();
        if (valid) {
            for (int s = 0; s < ns; ++s) {
                if (q0 + s == p) continue;
                const double d0 = xi0 - sx[2 * s], d1 = xi1 - sx[2 * s + 1];
                double gr, gi;
                green_helmholtz(g.wavenumber, d0 * d0 + d1 * d1, gr, gi);
                gi *= conj_sign;
                for (int c = 0; c < DH_R; ++c) {
                    const double vr = sv[(s * DH_R + c) * 2], vi = sv[(s * DH_R + c) * 2 + 1];
                    ar[c] += gr * vr - gi * vi;
                    ai[c] += gr * vi + gi * vr;
                }
            }
        }
    }
    if (valid) {
        const int64_t e = 2 * p;
        const double tf = a.trans ? g.c[e] * g.w[e] : g.b[e];
        const double sr = g.b[e] * g.kself[e] * g.c[e] + g.a[e];
        const double si = conj_sign * g.b[e] * g.kself_im[e] * g.c[e];
        for (int c = 0; c < nr; ++c) {
            const double xr = a.x[e + a.ldx * (r0 + c)], xim = a.x[e + 1 + a.ldx * (r0 + c)];
            a.y[e + a.ldy * (r0 + c)] = tf * ar[c] + sr * xr - si * xim;
            a.y[e + 1 + a.ldy * (r0 + c)] = tf * ai[c] + sr * xim + si * xr;
        }
    }
}

cudaError_t launch_direct_helmholtz(const DirectArgs& a, cudaStream_t st) {
    if (a.seg_n == 0) return cudaSuccess;
    const int blocks = (int)((a.seg_n / 2 + DS_T - 1) / DS_T);
    for (int r0 = 0; r0 < a.nrhs; r0 += DH_R) {
        note_launch();
        direct_helmholtz_kernel<<<blocks, DS_T, 0, st>>>(a, r0, std::min(DH_R, a.nrhs - r0));
    }
    return cudaGetLastError();
}

cudaError_t launch_direct_general(const DirectArgs& a, cudaStream_t st) {
    if (a.seg_n == 0) return cudaSuccess;
    const int blocks = (int)((a.seg_n + DS_T - 1) / DS_T);
    for (int r0 = 0; r0 < a.nrhs; r0 += DS_R) {
        note_launch();
        direct_general_kernel<<<blocks, DS_T, 0, st>>>(a, r0, std::min(DS_R, a.nrhs - r0));
    }
    return cudaGetLastError();
}

// --------------------------------------------------------- uniform grid --

__global__ void grid_table_kernel(double* table, int n, int dim, double h, int kernel_id, double k0) {
    const int64_t tot = dim == 2 ? (int64_t)n * n : (int64_t)n * n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t t = e;
        double r2 = 0.0;
        for (int d = 0; d < dim; ++d) {
            const double dd = (double)(t % n) * h;
            r2 += dd * dd;
            t /= n;
        }
        table[e] = e == 0 ? k0 : green_d(kernel_id, r2);
    }
}

cudaError_t launch_grid_table(double* table, int n, int dim, double h, int kernel_id, double kself_over_w,
                              cudaStream_t st) {
    const int64_t tot = dim == 2 ? (int64_t)n * n : (int64_t)n * n * n;
    note_launch();
    grid_table_kernel<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, st>>>(table, n, dim, h, kernel_id,
                                                                                 kself_over_w);
    return cudaGetLastError();
}

__global__ void grid_scatter_kernel(GridDirectArgs a, int64_t N) {
    // v (grid order) = source weight * x
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * a.nrhs; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gpos = e % N, c = e / N;
        const int j = a.dof_of[gpos];
        const double sw = a.trans ? a.b[j] : a.w[j] * a.c[j];
        a.vbuf[gpos + N * c] = sw * a.x[j + a.ldx * c];
    }
}

__global__ void grid_finish_kernel(GridDirectArgs a, int64_t N) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * a.nrhs; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gpos = e % N, c = e / N;
        const int i = a.dof_of[gpos];
        const double tf = a.trans ? a.c[i] * a.w[i] : a.b[i];
        a.y[i + a.ldy * c] = a.a[i] * a.x[i + a.ldx * c] + tf * a.ybuf[gpos + N * c];
    }
}

void grid_scatter_kernel_launch(const GridDirectArgs& a, int64_t N, int eb, cudaStream_t st) {
    note_launch();
    grid_scatter_kernel<<<eb, 256, 0, st>>>(a, N);
}

void grid_finish_kernel_launch(const GridDirectArgs& a, int64_t N, int eb, cudaStream_t st) {
    note_launch();
    grid_finish_kernel<<<eb, 256, 0, st>>>(a, N);
}

// Tile shapes: 2D 16 x 16, 3D 8 x 8 x 4 (256 points either way).
template <int DIM>
__global__ void __launch_bounds__(256) grid_conv_kernel(GridDirectArgs a, int r0, int nr) {
    constexpr int T0 = DIM == 2 ? 16 : 8, T1 = DIM == 2 ? 16 : 8, T2 = DIM == 2 ? 1 : 4;
    constexpr int W0 = 2 * T0 - 1, W1 = 2 * T1 - 1, W2 = 2 * T2 - 1;
    __shared__ double tw[W0 * W1 * W2];
    __shared__ double sv[256 * DS_R];
    const int n = a.n;
    const int nt0 = (n + T0 - 1) / T0, nt1 = (n + T1 - 1) / T1, nt2 = DIM == 2 ? 1 : (n + T2 - 1) / T2;
    int tb = blockIdx.x;
    const int tt2 = tb % nt2; tb /= nt2;
    const int tt1 = tb % nt1; tb /= nt1;
    const int tt0 = tb;
    const int l0 = threadIdx.x / (T1 * T2), l1 = (threadIdx.x / T2) % T1, l2 = threadIdx.x % T2;
    const int i0 = tt0 * T0 + l0, i1 = tt1 * T1 + l1, i2 = tt2 * T2 + l2;
    const bool valid = i0 < n && i1 < n && (DIM == 2 || i2 < n);
    const int64_t N = DIM == 2 ? (int64_t)n * n : (int64_t)n * n * n;
    double acc[DS_R];
    for (int c = 0; c < DS_R; ++c) acc[c] = 0.0;
    for (int s0 = 0; s0 < nt0; ++s0)
        for (int s1 = 0; s1 < nt1; ++s1)
            for (int s2 = 0; s2 < nt2; ++s2) {
                __syncthreads();
                // table window: offsets (tt - s) * T + [-(T-1), T-1] per axis
                for (int e = threadIdx.x; e < W0 * W1 * W2; e += 256) {
                    const int w2 = e % W2, w1 = (e / W2) % W1, w0 = e / (W1 * W2);
                    const int d0 = abs((tt0 - s0) * T0 + w0 - (T0 - 1));
                    const int d1 = abs((tt1 - s1) * T1 + w1 - (T1 - 1));
                    const int d2 = DIM == 2 ? 0 : abs((tt2 - s2) * T2 + w2 - (T2 - 1));
                    double v = 0.0;
                    if (d0 < n && d1 < n && d2 < n)
                        v = DIM == 2 ? a.table[(int64_t)d0 + (int64_t)n * d1]
                                     : a.table[(int64_t)d0 + (int64_t)n * (d1 + (int64_t)n * d2)];
                    tw[e] = v;
                }
                for (int e = threadIdx.x; e < 256; e += 256) {
                    const int m0 = e / (T1 * T2), m1 = (e / T2) % T1, m2 = e % T2;
                    const int j0 = s0 * T0 + m0, j1 = s1 * T1 + m1, j2 = s2 * T2 + m2;
                    const bool ok = j0 < n && j1 < n && (DIM == 2 || j2 < n);
                    const int64_t gpos = DIM == 2 ? (int64_t)j0 * n + j1 : ((int64_t)j0 * n + j1) * n + j2;
                    for (int c = 0; c < DS_R; ++c)
                        sv[e * DS_R + c] = (ok && c < nr) ? a.vbuf[gpos + N * (r0 + c)] : 0.0;
                }
                __syncthreads();
                if (valid) {
                    for (int m = 0; m < 256; ++m) {
                        const int m0 = m / (T1 * T2), m1 = (m / T2) % T1, m2 = m % T2;
                        const int w0 = l0 - m0 + (T0 - 1), w1 = l1 - m1 + (T1 - 1), w2 = l2 - m2 + (T2 - 1);
                        const double t = tw[(w0 * W1 + w1) * W2 + w2];
                        for (int c = 0; c < DS_R; ++c) acc[c] += t * sv[m * DS_R + c];
                    }
                }
            }
    if (valid) {
        const int64_t gpos = DIM == 2 ? (int64_t)i0 * n + i1 : ((int64_t)i0 * n + i1) * n + i2;
        for (int c = 0; c < nr; ++c) a.ybuf[gpos + N * (r0 + c)] = acc[c];
    }
}

cudaError_t launch_direct_grid(const GridDirectArgs& a, cudaStream_t st) {
    const int64_t N = a.dim == 2 ? (int64_t)a.n * a.n : (int64_t)a.n * a.n * a.n;
    if (N == 0) return cudaSuccess;
    const int eb = (int)std::min<int64_t>((N * a.nrhs + 255) / 256, 152 * 16);
    note_launch();
    grid_scatter_kernel<<<eb, 256, 0, st>>>(a, N);
    int tiles;
    if (a.dim == 2) tiles = ((a.n + 15) / 16) * ((a.n + 15) / 16);
    else tiles = ((a.n + 7) / 8) * ((a.n + 7) / 8) * ((a.n + 3) / 4);
    for (int r0 = 0; r0 < a.nrhs; r0 += DS_R) {
        const int nr = std::min(DS_R, a.nrhs - r0);
        note_launch();
        if (a.dim == 2) grid_conv_kernel<2><<<tiles, 256, 0, st>>>(a, r0, nr);
        else grid_conv_kernel<3><<<tiles, 256, 0, st>>>(a, r0, nr);
    }
    note_launch();
    grid_finish_kernel<<<eb, 256, 0, st>>>(a, N);
    return cudaGetLastError();
}


// ------------------------------------------- uniform grid, double-float --
//
// Same sum, in paired FP32 ("double-float") arithmetic: every table entry and
// every source value is split into hi + lo floats (hi = fl32(v), lo =
// fl32(v - hi)), each product T v is formed as an exact FP32 product of the
// hi parts (fma recovers its rounding error) plus the two cross terms, and the
// running sum is kept as an unevaluated pair updated with the error-free
// two-sum (Knuth).  Every operation is good to ~2^-48 relative, far below the
// 1e-10 residual the refinement certifies; the work runs on the FP32 pipes,
// which GB300 has 64x more of than FP64.

__global__ void split_df_kernel(const double* src, float2* dst, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = src[e];
        const float hi = (float)v;
        dst[e] = make_float2(hi, (float)(v - (double)hi));
    }
}

__global__ void grid_scatter_df_kernel(GridDirectArgs a, int64_t N, float2* vdf) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * a.nrhs; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gpos = e % N, c = e / N;
        const int j = a.dof_of[gpos];
        const double sw = a.trans ? a.b[j] : a.w[j] * a.c[j];
        const double v = sw * a.x[j + a.ldx * c];
        const float hi = (float)v;
        vdf[gpos + N * c] = make_float2(hi, (float)(v - (double)hi));
    }
}

template <int DIM, int NR>
__global__ void __launch_bounds__(256) grid_conv_df_kernel(GridDirectArgs a, const float2* tdf, const float2* vdf,
                                                           int r0) {
    constexpr int T0 = DIM == 2 ? 16 : 8, T1 = DIM == 2 ? 16 : 8, T2 = DIM == 2 ? 1 : 4;
    constexpr int W0 = 2 * T0 - 1, W1 = 2 * T1 - 1, W2 = 2 * T2 - 1;
    __shared__ float2 tw[W0 * W1 * W2];
    __shared__ float2 sv[256 * NR];
    const int n = a.n;
    const int nt0 = (n + T0 - 1) / T0, nt1 = (n + T1 - 1) / T1, nt2 = DIM == 2 ? 1 : (n + T2 - 1) / T2;
    int tb = blockIdx.x;
    const int tt2 = tb % nt2; tb /= nt2;
    const int tt1 = tb % nt1; tb /= nt1;
    const int tt0 = tb;
    const int l0 = threadIdx.x / (T1 * T2), l1 = (threadIdx.x / T2) % T1, l2 = threadIdx.x % T2;
    const int i0 = tt0 * T0 + l0, i1 = tt1 * T1 + l1, i2 = tt2 * T2 + l2;
    const bool valid = i0 < n && i1 < n && (DIM == 2 || i2 < n);
    const int64_t N = DIM == 2 ? (int64_t)n * n : (int64_t)n * n * n;
    float sh[NR], sl[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) { sh[c] = 0.f; sl[c] = 0.f; }
    for (int s0 = 0; s0 < nt0; ++s0)
        for (int s1 = 0; s1 < nt1; ++s1)
            for (int s2 = 0; s2 < nt2; ++s2) {
                __syncthreads();
                for (int e = threadIdx.x; e < W0 * W1 * W2; e += 256) {
                    const int w2 = e % W2, w1 = (e / W2) % W1, w0 = e / (W1 * W2);
                    const int d0 = abs((tt0 - s0) * T0 + w0 - (T0 - 1));
                    const int d1 = abs((tt1 - s1) * T1 + w1 - (T1 - 1));
                    const int d2 = DIM == 2 ? 0 : abs((tt2 - s2) * T2 + w2 - (T2 - 1));
                    float2 v = make_float2(0.f, 0.f);
                    if (d0 < n && d1 < n && d2 < n)
                        v = DIM == 2 ? tdf[(int64_t)d0 + (int64_t)n * d1]
                                     : tdf[(int64_t)d0 + (int64_t)n * (d1 + (int64_t)n * d2)];
                    tw[e] = v;
                }
                {
                    const int e = threadIdx.x;
                    const int m0 = e / (T1 * T2), m1 = (e / T2) % T1, m2 = e % T2;
                    const int j0 = s0 * T0 + m0, j1 = s1 * T1 + m1, j2 = s2 * T2 + m2;
                    const bool ok = j0 < n && j1 < n && (DIM == 2 || j2 < n);
                    const int64_t gpos = DIM == 2 ? (int64_t)j0 * n + j1 : ((int64_t)j0 * n + j1) * n + j2;
#pragma unroll
                    for (int c = 0; c < NR; ++c)
                        sv[e * NR + c] = ok ? vdf[gpos + N * (r0 + c)] : make_float2(0.f, 0.f);
                }
                __syncthreads();
                if (valid) {
#pragma unroll 4
                    for (int m = 0; m < 256; ++m) {
                        const int m0 = m / (T1 * T2), m1 = (m / T2) % T1, m2 = m % T2;
                        const int w0 = l0 - m0 + (T0 - 1), w1 = l1 - m1 + (T1 - 1), w2 = l2 - m2 + (T2 - 1);
                        const float2 t = tw[(w0 * W1 + w1) * W2 + w2];
#pragma unroll
                        for (int c = 0; c < NR; ++c) {
                            const float2 v = sv[m * NR + c];
                            const float p = t.x * v.x;
                            float e = fmaf(t.x, v.x, -p);
                            e = fmaf(t.x, v.y, e);
                            e = fmaf(t.y, v.x, e);
                            const float s = sh[c] + p;
                            const float bb = s - sh[c];
                            const float err = (sh[c] - (s - bb)) + (p - bb);
                            sh[c] = s;
                            sl[c] += err + e;
                        }
                    }
                }
            }
    if (valid) {
        const int64_t gpos = DIM == 2 ? (int64_t)i0 * n + i1 : ((int64_t)i0 * n + i1) * n + i2;
#pragma unroll
        for (int c = 0; c < NR; ++c) a.ybuf[gpos + N * (r0 + c)] = (double)sh[c] + (double)sl[c];
    }
}

template <int DIM>
static void launch_conv_df(const GridDirectArgs& a, const float2* tdf, const float2* vdf, int tiles, cudaStream_t st) {
    for (int r0 = 0; r0 < a.nrhs;) {
        const int left = a.nrhs - r0;
        note_launch();
        if (left >= 8) { grid_conv_df_kernel<DIM, 8><<<tiles, 256, 0, st>>>(a, tdf, vdf, r0); r0 += 8; }
        else if (left >= 4) { grid_conv_df_kernel<DIM, 4><<<tiles, 256, 0, st>>>(a, tdf, vdf, r0); r0 += 4; }
        else if (left >= 2) { grid_conv_df_kernel<DIM, 2><<<tiles, 256, 0, st>>>(a, tdf, vdf, r0); r0 += 2; }
        else { grid_conv_df_kernel<DIM, 1><<<tiles, 256, 0, st>>>(a, tdf, vdf, r0); r0 += 1; }
    }
}

cudaError_t launch_split_df(const double* src, float2* dst, int64_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    note_launch();
    split_df_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_direct_grid_df(const GridDirectArgs& a, const float2* tdf, float2* vdf, cudaStream_t st) {
    const int64_t N = a.dim == 2 ? (int64_t)a.n * a.n : (int64_t)a.n * a.n * a.n;
    if (N == 0) return cudaSuccess;
    const int eb = (int)std::min<int64_t>((N * a.nrhs + 255) / 256, 152 * 16);
    note_launch();
    grid_scatter_df_kernel<<<eb, 256, 0, st>>>(a, N, vdf);
    int tiles;
    if (a.dim == 2) tiles = ((a.n + 15) / 16) * ((a.n + 15) / 16);
    else tiles = ((a.n + 7) / 8) * ((a.n + 7) / 8) * ((a.n + 3) / 4);
    if (a.dim == 2) launch_conv_df<2>(a, tdf, vdf, tiles, st);
    else launch_conv_df<3>(a, tdf, vdf, tiles, st);
    note_launch();
    grid_finish_kernel<<<eb, 256, 0, st>>>(a, N);
    return cudaGetLastError();
}

// ------------------------------------------------------------- BLAS-1 ----

__global__ void axpby_kernel(int64_t N, int nrhs, double alpha, const double* x, int64_t ldx, double beta, double* y,
                             int64_t ldy) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % N, c = e / N;
        y[i + ldy * c] = beta == 0.0 ? alpha * x[i + ldx * c] : alpha * x[i + ldx * c] + beta * y[i + ldy * c];
    }
}

cudaError_t launch_axpby(int64_t N, int nrhs, double alpha, const double* x, int64_t ldx, double beta, double* y,
                         int64_t ldy, cudaStream_t st) {
    if (N * nrhs == 0) return cudaSuccess;
    note_launch();
    axpby_kernel<<<(int)std::min<int64_t>((N * nrhs + 255) / 256, 152 * 16), 256, 0, st>>>(N, nrhs, alpha, x, ldx, beta, y, ldy);
    return cudaGetLastError();
}

// The kernel part b K c u of A u from a residual r = f - A u: out = f - r - a u
// (ld = N everywhere).
__global__ void kpart_kernel(int64_t N, int nrhs, const double* f, const double* r, const double* a, const double* u,
                             double* out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * nrhs; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = f[e] - r[e] - a[e % N] * u[e];
}

cudaError_t launch_kpart(int64_t N, int nrhs, const double* f, const double* r, const double* a, const double* u,
                         double* out, cudaStream_t st) {
    if (N * nrhs == 0) return cudaSuccess;
    note_launch();
    kpart_kernel<<<(int)std::min<int64_t>((N * nrhs + 255) / 256, 152 * 16), 256, 0, st>>>(N, nrhs, f, r, a, u, out);
    return cudaGetLastError();
}

// Coefficient gradients of the adjoint method for L(u), A u = f, per DOF i and
// summed over the columns: ga_i = -sum lam u, gb_i = -sum lam (F u - a u)_i / b_i,
// gc_i = -sum u (F^T lam - a lam)_i / c_i (F u - a u stands for b K c u, F^T lam
// - a lam for c K^T b lam).  *bad is set when some b_i or c_i is zero.
__global__ void adjoint_coef_kernel(int64_t N, int nrhs, const double* a, const double* b, const double* c,
                                    const double* u, const double* lam, const double* Fu, const double* Ftl,
                                    double* ga, double* gb, double* gc, int* bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double ai = a[i], bi = b[i], ci = c[i];
        if (bi == 0.0 || ci == 0.0) {
            atomicOr(bad, 1);
            continue;
        }
        double sa = 0.0, sb = 0.0, sc = 0.0;
        for (int col = 0; col < nrhs; ++col) {
            const int64_t e = i + N * col;
            const double ui = u[e], li = lam[e];
            sa += li * ui;
            sb += li * (Fu[e] - ai * ui);
            sc += ui * (Ftl[e] - ai * li);
        }
        ga[i] = -sa;
        gb[i] = -sb / bi;
        gc[i] = -sc / ci;
    }
}

cudaError_t launch_adjoint_coef(int64_t N, int nrhs, const double* a, const double* b, const double* c,
                                const double* u, const double* lam, const double* Fu, const double* Ftl, double* ga,
                                double* gb, double* gc, int* bad, cudaStream_t st) {
    if (N == 0) return cudaSuccess;
    note_launch();
    adjoint_coef_kernel<<<(int)std::min<int64_t>((N + 255) / 256, 152 * 8), 256, 0, st>>>(N, nrhs, a, b, c, u, lam,
                                                                                           Fu, Ftl, ga, gb, gc, bad);
    return cudaGetLastError();
}

__global__ void col_dots_kernel(int64_t N, const double* x, int64_t ldx, const double* y, int64_t ldy, double* out) {
    // one CTA per column, deterministic tree reduction
    __shared__ double red[256];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += x[i + ldx * c] * y[i + ldy * c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

__global__ void seg_dots_kernel(const int64_t* off, const int64_t* cnt, const double* x, int64_t ldx, const double* y,
                                int64_t ldy, double* out) {
    // CTA (s, c): sum over rows of problem s of x[:, c] * y[:, c], tree reduction
    __shared__ double red[256];
    const int s = blockIdx.x, c = blockIdx.y;
    const int64_t o = off[s], n = cnt[s];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += x[o + i + ldx * c] * y[o + i + ldy * c];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[s + (int64_t)gridDim.x * c] = red[0];
}

cudaError_t launch_seg_dots(int nseg, const int64_t* off, const int64_t* cnt, int nrhs, const double* x, int64_t ldx,
                            const double* y, int64_t ldy, double* out, cudaStream_t st) {
    if (nseg == 0 || nrhs == 0) return cudaSuccess;
    note_launch();
    seg_dots_kernel<<<dim3(nseg, nrhs), 256, 0, st>>>(off, cnt, x, ldx, y, ldy, out);
    return cudaGetLastError();
}

cudaError_t launch_col_dots(int64_t N, int nrhs, const double* x, int64_t ldx, const double* y, int64_t ldy,
                            double* out, cudaStream_t st) {
    if (nrhs == 0) return cudaSuccess;
    note_launch();
    col_dots_kernel<<<nrhs, 256, 0, st>>>(N, x, ldx, y, ldy, out);
    return cudaGetLastError();
}

}  // namespace hif
