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

namespace hif {

// Block-wide (max value, lowest index) reduction of v over the threads;
// idx = -1 marks "no candidate".  red: blockDim scratch each.
template <typename T>
__device__ inline void cta_max_lowest(T& v, int& idx, T* redv, int* redi) {
    redv[threadIdx.x] = v;
    redi[threadIdx.x] = idx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const T v2 = redv[threadIdx.x + s];
            const int i2 = redi[threadIdx.x + s];
            const T v1 = redv[threadIdx.x];
            const int i1 = redi[threadIdx.x];
            if (i2 >= 0 && (i1 < 0 || v2 > v1 || (v2 == v1 && i2 < i1))) {
                redv[threadIdx.x] = v2;
                redi[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    v = redv[0];
    idx = redi[0];
    __syncthreads();
}

// Symmetric factorization P A P^T = L D L^T of a symmetric n x n block with
// 1 x 1 pivots: at step j the remaining diagonal entry of largest magnitude
// (ties: lowest position), accepted if it is at least alpha times the
// largest other entry of its column in the remaining block (the
// Bunch-Kaufman test for a 1 x 1 pivot, alpha = (1 + sqrt 17) / 8 unless the
// caller passes another value).  The
// whole block is updated (it stays symmetric); on return the strict lower
// triangle holds L and the diagonal D.  piv[j] = position interchanged with
// j at step j.  The columns of B (kb x n, leading dimension ldb) follow the
// interchanges, giving B P^T.  Returns 0, 1 for a pivot that fails the test
// (the caller falls back to LU) or 2 for a zero or non-finite pivot.
template <typename T>
__device__ int cta_ldl_diag(int n, T* A, int64_t lda, int* piv, T* B, int64_t ldb, int kb, T* redv, int* redi,
                            T alpha) {
    for (int j = 0; j < n; ++j) {
        T best = T(-1);
        int p = -1;
        for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
            const T v = fabs(A[i + lda * i]);
            if (v > best || (v == best && (p < 0 || i < p))) { best = v; p = i; }
        }
        cta_max_lowest<T>(best, p, redv, redi);
        if (p < j || p >= n) p = j;
        T cm = T(0);
        int ci = -1;
        for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
            if (i == p) continue;
            const T v = fabs(A[i + lda * p]);
            if (ci < 0 || v > cm) { cm = v; ci = i; }
        }
        cta_max_lowest<T>(cm, ci, redv, redi);
        if (ci < 0) cm = T(0);
        const T dp = A[p + lda * p];
        __syncthreads();                         // every thread has read A[p][p] before the swaps
        if (dp == T(0) || !isfinite((double)dp)) return 2;
        if (!(fabs(dp) >= alpha * cm)) return 1;
        if (threadIdx.x == 0) piv[j] = p;
        if (p != j) {
            for (int c = threadIdx.x; c < n; c += blockDim.x) {        // rows j <-> p
                const T t = A[j + lda * c];
                A[j + lda * c] = A[p + lda * c];
                A[p + lda * c] = t;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) {        // columns j <-> p
                const T t = A[i + lda * j];
                A[i + lda * j] = A[i + lda * p];
                A[i + lda * p] = t;
            }
            for (int i = threadIdx.x; i < kb; i += blockDim.x) {
                const T t = B[i + ldb * j];
                B[i + ldb * j] = B[i + ldb * p];
                B[i + ldb * p] = t;
            }
        }
        __syncthreads();
        const T d = A[j + lda * j];
        const T inv = T(1) / d;
        const int mm = n - j - 1;
        const int tot = mm * mm;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int i = j + 1 + e % mm, c = j + 1 + e / mm;
            A[i + lda * c] -= A[i + lda * j] * A[c + lda * j] * inv;
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + lda * j] *= inv;
        __syncthreads();
    }
    return 0;
}

// X (m x n) <- X L^{-T}, L unit lower (strict part in A): row by row,
// X[i][j] -= sum_{l<j} X[i][l] L[j][l].
template <typename T>
__device__ void cta_trsm_right_unit_lower_t(int n, const T* A, int64_t lda, T* X, int64_t ldx, int m) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        for (int j = 0; j < n; ++j) {
            T v = X[i + ldx * j];
            for (int l = 0; l < j; ++l) v -= X[i + ldx * l] * A[j + lda * l];
            X[i + ldx * j] = v;
        }
    }
    __syncthreads();
}

// L^{-1} of the unit lower L whose strict part sits in the strict lower
// triangle of LL (n x n, leading dimension n), written transposed into the
// strict upper triangle: LL[c + n i] = (L^{-1})[i][c] for i > c.  One
// thread per column of L^{-1}.
template <typename T>
__device__ void cta_unit_lower_inverse_to_upper(int n, T* LL) {
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        for (int i = c + 1; i < n; ++i) {
            T v = -LL[i + (int64_t)n * c];
            for (int l = c + 1; l < i; ++l) v -= LL[i + (int64_t)n * l] * LL[c + (int64_t)n * l];
            LL[c + (int64_t)n * i] = v;
        }
    }
    __syncthreads();
}

}  // namespace hif
