// CTA-cooperative dense linear algebra on small column-major blocks that sit
// in shared memory or in a per-box global workspace.  Every routine is
// called by all threads of the block and ends with __syncthreads().
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hif {

// C (m x n) += alpha * op(A) * op(B); op(A) is m x kk, op(B) is kk x n.
// tA/tB: false = as stored, true = transposed.
template <typename T>
__device__ void cta_gemm(int m, int n, int kk, T alpha, const T* A, int64_t lda, bool tA,
                         const T* B, int64_t ldb, bool tB, T* C, int64_t ldc) {
    const int tot = m * n;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int i = e % m, j = e / m;
        T acc = T(0);
        for (int l = 0; l < kk; ++l) {
            const T av = tA ? A[l + lda * i] : A[i + lda * l];
            const T bv = tB ? B[j + ldb * l] : B[l + ldb * j];
            acc += av * bv;
        }
        C[i + ldc * j] += alpha * acc;
    }
    __syncthreads();
}

// Block-wide argmax of |v| (ties: lowest index).  red: 2*blockDim scratch.
template <typename T>
__device__ int cta_argmax_abs(const T* col, int lo, int hi, T* redv, int* redi) {
    T best = T(-1);
    int bi = hi;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const T v = fabs(col[i]);
        if (v > best) { best = v; bi = i; }
    }
    redv[threadIdx.x] = best;
    redi[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const T v2 = redv[threadIdx.x + s];
            const int i2 = redi[threadIdx.x + s];
            if (v2 > redv[threadIdx.x] || (v2 == redv[threadIdx.x] && i2 < redi[threadIdx.x])) {
                redv[threadIdx.x] = v2;
                redi[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    int r = redi[0];
    __syncthreads();
    // no comparable entry (all NaN): keep the diagonal row; the caller's
    // pivot test then reports the block as singular
    if (r < lo || r >= hi) r = lo;
    return r;
}

// In-place LU with partial pivoting, P A = L U (L unit lower, U upper).
// piv[j] = row swapped with row j at step j (LAPACK style).  Returns false
// (on every thread) if a zero or non-finite pivot is met.
template <typename T>
__device__ bool cta_lu(int n, T* A, int64_t lda, int* piv, T* redv, int* redi) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        const int p = cta_argmax_abs(A + lda * j, j, n, redv, redi);
        if (threadIdx.x == 0) piv[j] = p;
        if (p != j) {
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                const T t = A[j + lda * c];
                A[j + lda * c] = A[p + lda * c];
                A[p + lda * c] = t;
            }
        }
        __syncthreads();
        const T d = A[j + lda * j];
        if (d == T(0) || !isfinite((double)d)) {
            if (threadIdx.x == 0) bad = 1;
            __syncthreads();
            break;
        }
        const T inv = T(1) / d;
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + lda * j] *= inv;
        __syncthreads();
        const int mm = n - j - 1;
        const int tot = mm * mm;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int i = j + 1 + e % mm, c = j + 1 + e / mm;
            A[i + lda * c] -= A[i + lda * j] * A[j + lda * c];
        }
        __syncthreads();
    }
    const bool ok = bad == 0;
    __syncthreads();
    return ok;
}

// Apply the LAPACK-style row interchanges piv[0..n) to B (n x ncols): P B.
template <typename T>
__device__ void cta_apply_piv(int n, const int* piv, T* B, int64_t ldb, int ncols) {
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        for (int j = 0; j < n; ++j) {
            const int p = piv[j];
            if (p != j) {
                const T t = B[j + ldb * c];
                B[j + ldb * c] = B[p + ldb * c];
                B[p + ldb * c] = t;
            }
        }
    }
    __syncthreads();
}

// B (n x ncols) <- L^{-1} B, L unit lower (strict part in A).
template <typename T>
__device__ void cta_trsm_lower_unit(int n, const T* A, int64_t lda, T* B, int64_t ldb, int ncols) {
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        for (int i = 0; i < n; ++i) {
            T v = B[i + ldb * c];
            for (int l = 0; l < i; ++l) v -= A[i + lda * l] * B[l + ldb * c];
            B[i + ldb * c] = v;
        }
    }
    __syncthreads();
}

// X (m x n) <- X U^{-1}, U upper with diagonal (stored in A).
template <typename T>
__device__ void cta_trsm_right_upper(int n, const T* A, int64_t lda, T* X, int64_t ldx, int m) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        for (int j = 0; j < n; ++j) {
            T v = X[i + ldx * j];
            for (int l = 0; l < j; ++l) v -= X[i + ldx * l] * A[l + lda * j];
            X[i + ldx * j] = v / A[j + lda * j];
        }
    }
    __syncthreads();
}

// Inverses of the unit triangular factors: Li = L^{-1} (strict lower part of
// out), Ui = U^{-1} (strict upper part of out), where L, U are the strict
// parts of A (U unit after scaling by the diagonal elsewhere).  Column-wise,
// one thread per column.
template <typename T>
__device__ void cta_unit_tri_inverses(int n, const T* A, int64_t lda, T* out, int64_t ldo) {
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        // column c of L^{-1}: solve L y = e_c (rows >= c)
        out[c + ldo * c] = T(0);
        for (int i = c + 1; i < n; ++i) {
            T v = -A[i + lda * c];
            for (int l = c + 1; l < i; ++l) v -= A[i + lda * l] * out[l + ldo * c];
            out[i + ldo * c] = v;
        }
        // column c of U^{-1}: solve U y = e_c (rows <= c), unit diagonal
        for (int i = c - 1; i >= 0; --i) {
            T v = -A[i + lda * c];
            for (int l = i + 1; l < c; ++l) v -= A[i + lda * l] * out[l + ldo * c];
            out[i + ldo * c] = v;
        }
    }
    __syncthreads();
}

}  // namespace hif
