// Top block D_L = A_L restricted to s_L (Sec. 3.1, level L): assembly from
// kernel entries plus accumulated SCIs, blocked right-looking LU with partial
// pivoting, explicit inverse for the solve sweeps, and the dense products
// x_{s_L} <- M x_{s_L} used by apply / solve (sm_103a).
#include "cta_linalg.cuh"
#include <algorithm>

#include "hif_common.cuh"
#include "launch.h"

namespace hif {

template <typename T>
__global__ void top_assemble_kernel(TopArgs a) {
    const int n = a.n;
    T* A = static_cast<T*>(a.A);
    const int d = a.g.dim;
    const int ref = a.ids[0];
    const double r0 = a.g.x[(int64_t)d * ref], r1 = a.g.x[(int64_t)d * ref + 1];
    const double r2 = d == 3 ? a.g.x[(int64_t)d * ref + 2] : 0.0;
    const int64_t tot = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(e % n), q = (int)(e / n);
        A[e] = entry<T>(a.g, a.sci, a.ids[p], a.ids[q], r0, r1, r2);
    }
}

template <typename T>
cudaError_t launch_top_assemble(const TopArgs& a, cudaStream_t st) {
    if (a.n == 0) return cudaSuccess;
    const int64_t tot = (int64_t)a.n * a.n;
    const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 152 * 32);
    note_launch();
    top_assemble_kernel<T><<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ---- blocked LU: panel / row interchanges / TRSM / GEMM update ----------

constexpr int NB = 32;

template <typename T>
__global__ void __launch_bounds__(256) panel_kernel(T* A, int n, int64_t ld, int j0, int nb, int* piv, int* status) {
    __shared__ T redv[256];
    __shared__ int redi[256];
    for (int j = j0 + threadIdx.x; j < j0 + nb; j += blockDim.x) piv[j] = j;
    __syncthreads();
    for (int j = j0; j < j0 + nb; ++j) {
        const int p = cta_argmax_abs<T>(A + ld * j, j, n, redv, redi);
        if (threadIdx.x == 0) piv[j] = p;
        if (p != j) {
            for (int c = j0 + threadIdx.x; c < j0 + nb; c += blockDim.x) {
                const T t = A[j + ld * c];
                A[j + ld * c] = A[p + ld * c];
                A[p + ld * c] = t;
            }
        }
        __syncthreads();
        const T dgl = A[j + ld * j];
        if (dgl == T(0) || !isfinite((double)dgl)) {
            if (threadIdx.x == 0) atomicOr(status, (int)DEV_SINGULAR);
            return;
        }
        const T inv = T(1) / dgl;
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const T l = A[i + ld * j] * inv;
            A[i + ld * j] = l;
            for (int c = j + 1; c < j0 + nb; ++c) A[i + ld * c] -= l * A[j + ld * c];
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void swap_trsm_kernel(T* A, int n, int64_t ld, int j0, int nb, const int* piv) {
    // one thread per column outside the panel: row interchanges, then for
    // columns right of the panel U12 = L11^{-1} A12
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || (c >= j0 && c < j0 + nb)) return;
    for (int j = j0; j < j0 + nb; ++j) {
        const int p = piv[j];
        if (p != j) {
            const T t = A[j + ld * c];
            A[j + ld * c] = A[p + ld * c];
            A[p + ld * c] = t;
        }
    }
    if (c >= j0 + nb) {
        for (int i = j0; i < j0 + nb; ++i) {
            T v = A[i + ld * c];
            for (int l = j0; l < i; ++l) v -= A[i + ld * l] * A[l + ld * c];
            A[i + ld * c] = v;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) update_kernel(T* A, int n, int64_t ld, int j0, int nb) {
    // A22 -= L21 U12 on 64 x 64 tiles, K = nb <= 32
    __shared__ T Ls[64][NB + 1];
    __shared__ T Us[NB][64 + 1];
    const int s = j0 + nb;
    const int i0 = s + blockIdx.x * 64, c0 = s + blockIdx.y * 64;
    for (int e = threadIdx.x; e < 64 * nb; e += blockDim.x) {
        const int i = e % 64, l = e / 64;
        Ls[i][l] = (i0 + i < n) ? A[(i0 + i) + ld * (j0 + l)] : T(0);
    }
    for (int e = threadIdx.x; e < 64 * nb; e += blockDim.x) {
        const int l = e % nb, c = e / nb;
        Us[l][c] = (c0 + c < n) ? A[(j0 + l) + ld * (c0 + c)] : T(0);
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4] = {};
    for (int l = 0; l < nb; ++l) {
        T av[4], bv[4];
        for (int q = 0; q < 4; ++q) av[q] = Ls[tx + 16 * q][l];
        for (int q = 0; q < 4; ++q) bv[q] = Us[l][ty + 16 * q];
        for (int p = 0; p < 4; ++p)
            for (int q = 0; q < 4; ++q) acc[p][q] += av[p] * bv[q];
    }
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + tx + 16 * p, c = c0 + ty + 16 * q;
            if (i < n && c < n) A[i + ld * c] -= acc[p][q];
        }
}

template <typename T>
cudaError_t lu_blocked(T* A, int n, int64_t ld, int* piv, int* status, cudaStream_t st) {
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int nb = std::min(NB, n - j0);
        note_launch();
        panel_kernel<T><<<1, 256, 0, st>>>(A, n, ld, j0, nb, piv, status);
        note_launch();
        swap_trsm_kernel<T><<<(n + 127) / 128, 128, 0, st>>>(A, n, ld, j0, nb, piv);
        const int rest = n - j0 - nb;
        if (rest > 0) {
            dim3 grid((rest + 63) / 64, (rest + 63) / 64);
            note_launch();
            update_kernel<T><<<grid, 256, 0, st>>>(A, n, ld, j0, nb);
        }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t top_lu(T* A, int n, int* piv, int* status, cudaStream_t st) {
    return lu_blocked<T>(A, n, n, piv, status, st);
}

// ---- inverse from the LU factors: Ainv = U^{-1} L^{-1} P ------------------

template <typename T>
__global__ void __launch_bounds__(256) lu_inverse_kernel(const T* LU, const int* piv, int n, T* Ainv) {
    // each CTA solves A X = I for 8 consecutive columns, axpy form
    const int64_t ld = n;
    const int c0 = blockIdx.x * 8;
    const int nc = min(8, n - c0);
    T* X = Ainv + ld * c0;
    for (int e = threadIdx.x; e < n * nc; e += blockDim.x) {
        const int i = e % n, c = e / n;
        X[i + ld * c] = (i == c0 + c) ? T(1) : T(0);
    }
    __syncthreads();
    if (threadIdx.x < nc) {
        T* col = X + ld * threadIdx.x;
        for (int j = 0; j < n; ++j) {
            const int p = piv[j];
            if (p != j) { const T t = col[j]; col[j] = col[p]; col[p] = t; }
        }
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {            // L y = P e
        for (int e = threadIdx.x; e < (n - j - 1) * nc; e += blockDim.x) {
            const int i = j + 1 + e % (n - j - 1), c = e / (n - j - 1);
            X[i + ld * c] -= LU[i + ld * j] * X[j + ld * c];
        }
        __syncthreads();
    }
    for (int j = n - 1; j >= 0; --j) {       // U x = y
        if (threadIdx.x < nc) X[j + ld * threadIdx.x] /= LU[j + ld * j];
        __syncthreads();
        for (int e = threadIdx.x; e < j * nc; e += blockDim.x) {
            const int i = e % j, c = e / j;
            X[i + ld * c] -= LU[i + ld * j] * X[j + ld * c];
        }
        __syncthreads();
    }
}

template <typename T>
cudaError_t top_inverse(const T* LU, const int* piv, int n, T* Ainv, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    note_launch();
    lu_inverse_kernel<T><<<(n + 7) / 8, 256, 0, st>>>(LU, piv, n, Ainv);
    return cudaGetLastError();
}

// ---- x_{s_L} <- op(M) x_{s_L} ---------------------------------------------

template <typename T>
__global__ void gather_kernel(const T* x, int64_t ldx, const int* ids, int n, int nrhs, T* tmp) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * nrhs; e += gridDim.x * blockDim.x)
        tmp[e] = x[ids[e % n] + ldx * (e / n)];
}

template <typename T>
__global__ void top_mv_kernel(const T* M, int n, int trans, const int* ids, T* x, int64_t ldx, int nrhs, const T* tmp) {
    const int64_t ld = n;
    if (!trans) {
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * nrhs; e += gridDim.x * blockDim.x) {
            const int i = e % n, c = e / n;
            T acc = T(0);
            for (int l = 0; l < n; ++l) acc += M[i + ld * l] * tmp[l + (int64_t)n * c];
            x[ids[i] + ldx * c] = acc;
        }
    } else {
        const int lane = threadIdx.x & 31;
        const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int nw = (gridDim.x * blockDim.x) >> 5;
        for (int e = w; e < n * nrhs; e += nw) {
            const int i = e % n, c = e / n;
            T acc = T(0);
            for (int l = lane; l < n; l += 32) acc += M[l + ld * i] * tmp[l + (int64_t)n * c];
            acc = warp_sum(acc);
            if (lane == 0) x[ids[i] + ldx * c] = acc;
        }
    }
}

template <typename T>
cudaError_t launch_top_gemm(const T* M, int n, bool trans, const int* ids, T* x, int64_t ldx, int nrhs, T* tmp,
                            cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    note_launch();
    gather_kernel<T><<<std::min(1024, (n * nrhs + 255) / 256), 256, 0, st>>>(x, ldx, ids, n, nrhs, tmp);
    note_launch();
    top_mv_kernel<T><<<std::min(152 * 8, (n * nrhs * (trans ? 32 : 1) + 255) / 256), 256, 0, st>>>(M, n, trans ? 1 : 0,
                                                                                               ids, x, ldx, nrhs, tmp);
    return cudaGetLastError();
}

template cudaError_t launch_top_assemble<double>(const TopArgs&, cudaStream_t);
template cudaError_t launch_top_assemble<float>(const TopArgs&, cudaStream_t);
template cudaError_t top_lu<double>(double*, int, int*, int*, cudaStream_t);
template cudaError_t lu_blocked<double>(double*, int, int64_t, int*, int*, cudaStream_t);
template cudaError_t lu_blocked<float>(float*, int, int64_t, int*, int*, cudaStream_t);
template cudaError_t top_lu<float>(float*, int, int*, int*, cudaStream_t);
template cudaError_t top_inverse<double>(const double*, const int*, int, double*, cudaStream_t);
template cudaError_t top_inverse<float>(const float*, const int*, int, float*, cudaStream_t);
template cudaError_t launch_top_gemm<double>(const double*, int, bool, const int*, double*, int64_t, int, double*,
                                             cudaStream_t);
template cudaError_t launch_top_gemm<float>(const float*, int, bool, const int*, float*, int64_t, int, float*,
                                            cudaStream_t);

}  // namespace hif
