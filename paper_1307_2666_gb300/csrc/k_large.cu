// Skeletonization of large boxes (sm_103a): boxes whose column count is too
// large for one CTA are spread over the whole GPU.
//
//  * big_ygen        materializes the proxy matrices Y_c of Eq. (3.3) of all
//                    large boxes of a sublevel in HBM (kernel and SCI parts
//                    apart when rho_g is needed, Sec. 4.4);
//  * big_pow_*       rho_g = min(1, |Y^K_g| / |Y^S_g|) by 8 power iterations
//                    from the all-ones vector, directly on Y_g;
//  * big_step /      column-pivoted Householder QR (Lemma 2.2), one pair of
//    big_update      launches per pivot step for all large groups at once: one
//                    CTA per group picks the pivot and forms the reflector, a
//                    warp per remaining column applies it and recomputes the
//                    column norm in FP64;
//  * big_T           T = R1^{-1} R2 and the skeleton / redundant order;
//  * gemm / trsm / elimination helpers: Lemma 2.4 blocks, Lemma 2.1 LU
//                    (blocked, multi-CTA) and the Schur update for one large
//                    box at a time.
#include <algorithm>

#include "hif_common.cuh"
#include "launch.h"

namespace hif {

// --------------------------------------------------------------- Y gen ----

template <typename T>
__global__ void big_ygen_kernel(BigArgs a) {
    const BigBox bb = a.bigboxes[blockIdx.y];
    const BoxDesc bx = a.boxes[bb.box];
    const int n = bx.n, npairs = bx.m_near + a.P;
    const int dim = a.g.dim;
    const bool scival = bx.has_sci && a.sci.nsub > 0;
    const bool split = scival && a.second_kind;
    const bool sym = bx.sym != 0;        // Y'_c: outgoing rows only (Sec. 5)
    T* YK = static_cast<T*>(a.YK) + bb.y_off;
    T* YS = split ? static_cast<T*>(a.YS) + bb.y_off : nullptr;
    const int64_t m = bb.m;
    const int* cols = a.cols + bx.col_off;
    const int* near = a.near + bx.near_off;
    const double c0 = bx.ctr[0], c1 = bx.ctr[1], c2 = dim == 3 ? bx.ctr[2] : 0.0;
    const int64_t tot = (int64_t)npairs * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(e % npairs), l = (int)(e / npairs);
        const int j = cols[l];
        const T cx0 = (T)(a.g.x[(int64_t)dim * j] - c0), cx1 = (T)(a.g.x[(int64_t)dim * j + 1] - c1);
        const T cx2 = dim == 3 ? (T)(a.g.x[(int64_t)dim * j + 2] - c2) : T(0);
        int rid, rcomp = 0;
        T rx0, rx1, rx2, rb, rwc;
        if (p < bx.m_near) {
            rid = near[p];
            if (a.g.ncomp == 2) rcomp = rid & 1;
            rx0 = (T)(a.g.x[(int64_t)dim * rid] - c0);
            rx1 = (T)(a.g.x[(int64_t)dim * rid + 1] - c1);
            rx2 = dim == 3 ? (T)(a.g.x[(int64_t)dim * rid + 2] - c2) : T(0);
            rb = (T)a.g.b[rid];
            rwc = (T)(a.g.w[rid] * a.g.c[rid]);
        } else {
            const int kx = p - bx.m_near;
            rid = -1;
            if (a.g.ncomp == 2) rcomp = kx & 1;
            rx0 = (T)(bx.radius * a.proxy[dim * kx]);
            rx1 = (T)(bx.radius * a.proxy[dim * kx + 1]);
            rx2 = dim == 3 ? (T)(bx.radius * a.proxy[dim * kx + 2]) : T(0);
            rb = T(1);
            rwc = T(1);
        }
        T k1, k2, s1, s2;
        y_pair<T>(a.g.kernel_id, rid, rx0, rx1, rx2, rb, rwc, j, cx0, cx1, cx2, (T)(a.g.w[j] * a.g.c[j]),
                  (T)a.g.b[j], (T)(a.g.b[j] * a.g.w[j]), scival, a.sci, k1, k2, s1, s2, rcomp,
                  (T)a.g.wavenumber);
        T* col = YK + m * l;
        if (sym) {
            col[p] = split ? k1 : k1 + s1;
            if (split) YS[m * l + p] = s1;
        } else if (split) {
            col[2 * p] = k1;
            col[2 * p + 1] = k2;
            YS[m * l + 2 * p] = s1;
            YS[m * l + 2 * p + 1] = s2;
        } else {
            col[2 * p] = k1 + s1;
            col[2 * p + 1] = k2 + s2;
        }
    }
}

// ------------------------------------------------------- rho_g (Sec 4.4) --

// t = Y_g v   (which: 0 = Y^K, 1 = Y^S), one thread per row
template <typename T>
__global__ void big_pow_tv_kernel(BigArgs a) {
    const BigGroup G = a.groups[blockIdx.y];
    if (!G.need_rho) return;
    const int which = blockIdx.z;
    const T* Y = static_cast<const T*>(which == 0 ? a.YK : a.YS) + G.y_off;
    const double* v = a.vec_v + 2 * G.vec_off + which * (int64_t)G.n;
    double* t = a.vec_t + 2 * G.row_off + which * (int64_t)G.m;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.m; i += gridDim.x * blockDim.x) {
        // rho_g needs only a rough norm ratio: FP32 data accumulate in FP32
        // (an FP64 FMA per entry binds the pass to the FP64 pipe)
        if constexpr (sizeof(T) == 4) {
            float acc = 0.f;
            for (int l = 0; l < G.n; ++l) acc = fmaf(Y[i + (int64_t)G.m * l], (float)v[l], acc);
            t[i] = acc;
        } else {
            double acc = 0.0;
            for (int l = 0; l < G.n; ++l) acc += (double)Y[i + (int64_t)G.m * l] * v[l];
            t[i] = acc;
        }
    }
}

// w = Y_g^T t, one warp per column
template <typename T>
__global__ void big_pow_w_kernel(BigArgs a) {
    const BigGroup G = a.groups[blockIdx.y];
    if (!G.need_rho) return;
    const int which = blockIdx.z;
    const T* Y = static_cast<const T*>(which == 0 ? a.YK : a.YS) + G.y_off;
    const double* t = a.vec_t + 2 * G.row_off + which * (int64_t)G.m;
    double* w = a.vec_w + 2 * G.vec_off + which * (int64_t)G.n;
    const int lane = threadIdx.x & 31;
    const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (l >= G.n) return;
    double acc = 0.0;
    if constexpr (sizeof(T) == 4) {
        float af = 0.f;
        for (int i = lane; i < G.m; i += 32) af = fmaf(Y[i + (int64_t)G.m * l], (float)t[i], af);
        acc = (double)af;
    } else {
        for (int i = lane; i < G.m; i += 32) acc += (double)Y[i + (int64_t)G.m * l] * t[i];
    }
    acc = warp_sum(acc);
    if (lane == 0) w[l] = acc;
}

// mode 0: v = w / |w| (v = 0 when w = 0); mode 1: est = |t|; mode 2: v = 1/sqrt(n)
__global__ void big_pow_norm_kernel(BigArgs a, int mode) {
    const BigGroup G = a.groups[blockIdx.x];
    if (!G.need_rho) return;
    const int which = blockIdx.y;
    double* v = a.vec_v + 2 * G.vec_off + which * (int64_t)G.n;
    const double* w = a.vec_w + 2 * G.vec_off + which * (int64_t)G.n;
    const double* t = a.vec_t + 2 * G.row_off + which * (int64_t)G.m;
    __shared__ double red[256];
    if (mode == 2) {
        for (int l = threadIdx.x; l < G.n; l += blockDim.x) v[l] = 1.0 / sqrt((double)G.n);
        return;
    }
    const double* src = mode == 0 ? w : t;
    const int len = mode == 0 ? G.n : G.m;
    double s = 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) s += src[i] * src[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    const double tot = red[0];
    if (mode == 1) {
        if (threadIdx.x == 0) a.est[2 * blockIdx.x + which] = sqrt(tot);
        return;
    }
    const double inv = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
    for (int l = threadIdx.x; l < G.n; l += blockDim.x) v[l] = w[l] * inv;
}

// tolerance per group and Y = Y^K + Y^S
__global__ void big_tol_kernel(BigArgs a, int ngroups) {
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ngroups) return;
    BigGroup& G = a.groups[gi];
    double rho = 1.0;
    if (G.need_rho) {
        const double eK = a.est[2 * gi], eS = a.est[2 * gi + 1];
        if (eS > 0.0) rho = fmin(1.0, eK / eS);
    }
    double tol = rho * a.eps;
    if (tol < a.tol_floor) tol = a.tol_floor;
    G.tol = tol;
}

template <typename T>
__global__ void big_add_kernel(T* YK, const T* YS, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        YK[e] += YS[e];
}

// --------------------------------------------------- pivoted QR steps ----

template <typename T>
__global__ void big_norm_init_kernel(BigArgs a) {
    const BigGroup G = a.groups[blockIdx.y];
    const T* Y = static_cast<const T*>(a.YK) + G.y_off;
    const int lane = threadIdx.x & 31;
    const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        BigState& S = a.state[blockIdx.y];
        S.k = 0;
        S.stop = 0;
        S.nu0 = 0.0;
        S.tau = 0.0;
        S.j0 = 0;
        S.pend = 0;
        S.last_step = -1;
    }
    if (l >= G.n) return;
    double s = 0.0;
    for (int i = lane; i < G.m; i += 32) {
        const double v = (double)Y[i + (int64_t)G.ld * l];
        s += v * v;
    }
    s = warp_sum(s);
    if (lane == 0) {
        a.nrm[G.vec_off + l] = s;
        if (a.nrm0) a.nrm0[G.vec_off + l] = s;
        a.perm[G.vec_off + l] = l;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) big_step_kernel(BigArgs a, int j) {
    const BigGroup G = a.groups[blockIdx.x];
    BigState* S = a.state + blockIdx.x;
    if (S->stop) return;
    T* W = static_cast<T*>(a.YK) + G.y_off;
    const int64_t ld = G.ld;
    double* nrm = a.nrm + G.vec_off;
    int* perm = a.perm + G.vec_off;
    __shared__ double redv[256];
    __shared__ int redi[256];
    __shared__ T hs[256];
    const int kmax = min(G.m, G.n);
    if (j >= kmax) {
        if (threadIdx.x == 0) S->stop = 1;
        return;
    }
    double best = -1.0;
    int bl = -1, bo = 1 << 30;
    for (int l = j + threadIdx.x; l < G.n; l += blockDim.x) {
        const double v = nrm[l];
        if (v > best || (v == best && perm[l] < bo)) { best = v; bo = perm[l]; bl = l; }
    }
    redv[threadIdx.x] = best;
    redi[threadIdx.x] = bl;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double v2 = redv[threadIdx.x + s], v1 = redv[threadIdx.x];
            const int l2 = redi[threadIdx.x + s], l1 = redi[threadIdx.x];
            if (l2 >= 0 && (l1 < 0 || v2 > v1 || (v2 == v1 && perm[l2] < perm[l1]))) {
                redv[threadIdx.x] = v2;
                redi[threadIdx.x] = l2;
            }
        }
        __syncthreads();
    }
    const double bnorm = sqrt(fmax(redv[0], 0.0));
    const int p = redi[0];
    const double nu0 = j == 0 ? bnorm : S->nu0;
    __syncthreads();
    if (bnorm <= G.tol * nu0 || bnorm == 0.0 || p < j) {
        if (threadIdx.x == 0) {
            S->stop = 1;
            if (j == 0) S->nu0 = bnorm;
        }
        return;
    }
    if (p != j) {
        for (int i = threadIdx.x; i < G.m; i += blockDim.x) {
            const T t = W[i + ld * j];
            W[i + ld * j] = W[i + ld * p];
            W[i + ld * p] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && p != j) {
        const int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
        const double tn = nrm[j]; nrm[j] = nrm[p]; nrm[p] = tn;
    }
    // reflector for W[j:, j]
    T s = T(0);
    for (int i = j + 1 + threadIdx.x; i < G.m; i += blockDim.x) {
        const T v = W[i + ld * j];
        s += v * v;
    }
    hs[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) hs[threadIdx.x] += hs[threadIdx.x + k];
        __syncthreads();
    }
    const T ss = hs[0];
    const T alpha = W[j + ld * j];
    T tau = T(0), scal = T(0);
    if (ss != T(0)) {
        const T beta = -copysign(sqrt(alpha * alpha + ss), alpha);
        tau = (beta - alpha) / beta;
        scal = T(1) / (alpha - beta);
    }
    __syncthreads();
    if (tau != T(0)) {
        for (int i = j + 1 + threadIdx.x; i < G.m; i += blockDim.x) W[i + ld * j] *= scal;
        if (threadIdx.x == 0) W[j + ld * j] = -copysign(sqrt(alpha * alpha + ss), alpha);
    }
    if (threadIdx.x == 0) {
        if (j == 0) S->nu0 = bnorm;
        S->tau = (double)tau;
        S->k = j + 1;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) big_update_kernel(BigArgs a, int j) {
    const BigGroup G = a.groups[blockIdx.y];
    const BigState S = a.state[blockIdx.y];
    if (S.k != j + 1 || S.stop) return;
    const int lane = threadIdx.x & 31;
    const int l = j + 1 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (l >= G.n) return;
    T* W = static_cast<T*>(a.YK) + G.y_off;
    const int64_t ld = G.ld;
    T* col = W + ld * l;
    const T* v = W + ld * j;
    const T tau = (T)S.tau;
    T w = T(0);
    if (tau != T(0)) {
        for (int i = j + 1 + lane; i < G.m; i += 32) w += v[i] * col[i];
        w = warp_sum(w);
        w = (w + col[j]) * tau;
        __syncwarp();
        if (lane == 0) col[j] -= w;
    }
    double s = 0.0;
    if constexpr (sizeof(T) == 4) {
        // FP32 factorization: the update and the new norm in one pass, each
        // lane's share of the norm summed in FP32 (its ~m/32 squares are FP32
        // data) and the lanes in FP64 -- a warp-wide FP64 FMA in the loop
        // would bind the step to the FP64 pipe
        float sf = 0.f;
        for (int i = j + 1 + lane; i < G.m; i += 32) {
            const float c = tau != T(0) ? col[i] - w * v[i] : col[i];
            if (tau != T(0)) col[i] = c;
            sf = fmaf(c, c, sf);
        }
        s = (double)sf;
    } else {
        if (tau != T(0))
            for (int i = j + 1 + lane; i < G.m; i += 32) col[i] -= w * v[i];
        // FP64: the new norm in its own pass
        for (int i = j + 1 + lane; i < G.m; i += 32) {
            const double c = (double)col[i];
            s += c * c;
        }
    }
    s = warp_sum(s);
    if (lane == 0) a.nrm[G.vec_off + l] = s;
}

// ---------------------------------------- blocked pivoted QR (panels) ----
//
// The pivoted QR of Lemma 2.2 with delayed trailing updates: within a panel
// of nb pivots only the pivot column and the pivot row are brought up to
// date; every trailing column l keeps F[l, q] = tau_q (W^T v_q)_l minus the
// earlier reflectors' share, so that W_updated = W - V F^T, and the panel
// ends with one product W[rows below the panel, trailing] -= V F^T.  The
// pivot choice and the rank test use the squared column norms downdated by
// the new pivot row's entries (in FP64); when a norm falls below
// sqrt(eps_T) of its value at the last exact computation the group ends its
// panel early, and every panel ends with the norms recomputed from the
// updated columns.  Per pivot the trailing columns are read once (for F),
// instead of read twice and written once.

constexpr int QPB = 32;   // maximum panel width

// start of a panel for every group still pivoting
__global__ void bqp_start_kernel(BigArgs a, int ngroups) {
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ngroups) return;
    BigState& S = a.state[gi];
    if (S.stop) return;
    S.j0 = S.k;
    S.pend = 0;
}

// one pivot of the panel (one CTA per group): argmax of the downdated norms,
// column swap, the pivot column brought up to date, its reflector, and
// g = V_panel^T v
constexpr int QPT = 512;   // threads of the pivot kernel

template <typename T>
__global__ void __launch_bounds__(QPT) bqp_pivot_kernel(BigArgs a, int step) {
    const BigGroup G = a.groups[blockIdx.x];
    BigState* S = a.state + blockIdx.x;
    if (S->stop || S->pend) return;
    const int j = S->k, j0 = S->j0, jj = j - j0;
    const int nb = a.nb;
    if (jj >= nb) return;
    const int kmax = min(G.m, G.n);
    if (j >= kmax) {
        if (threadIdx.x == 0) S->stop = 1;
        return;
    }
    T* W = static_cast<T*>(a.YK) + G.y_off;
    const int64_t ld = G.ld;
    const int n = G.n;
    double* nrm = a.nrm + G.vec_off;
    double* nrm0 = a.nrm0 + G.vec_off;
    int* perm = a.perm + G.vec_off;
    T* F = static_cast<T*>(a.F) + G.vec_off * nb;
    T* gq = static_cast<T*>(a.gv) + (int64_t)blockIdx.x * QPB;
    __shared__ double redv[QPT];
    __shared__ int redi[QPT];
    __shared__ T hs[QPT];
    __shared__ T fj[QPB];
    __shared__ T part[QPT / 32][QPB];
    // pivot: largest downdated norm, ties to the lowest original column
    double best = -1.0;
    int bl = -1, bo = 1 << 30;
    for (int l = j + threadIdx.x; l < n; l += blockDim.x) {
        const double v = nrm[l];
        if (v > best || (v == best && perm[l] < bo)) { best = v; bo = perm[l]; bl = l; }
    }
    redv[threadIdx.x] = best;
    redi[threadIdx.x] = bl;
    __syncthreads();
    for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) {
            const double v2 = redv[threadIdx.x + s2], v1 = redv[threadIdx.x];
            const int l2 = redi[threadIdx.x + s2], l1 = redi[threadIdx.x];
            if (l2 >= 0 && (l1 < 0 || v2 > v1 || (v2 == v1 && perm[l2] < perm[l1]))) {
                redv[threadIdx.x] = v2;
                redi[threadIdx.x] = l2;
            }
        }
        __syncthreads();
    }
    const double bnorm = sqrt(fmax(redv[0], 0.0));
    const int p = redi[0];
    const double nu0 = j == 0 ? bnorm : S->nu0;
    __syncthreads();
    // the rank test decides on exact norms: within a panel (downdated norms,
    // relative error up to ~sqrt(eps_T) in the square) a maximum near the
    // threshold ends the panel instead, and the next panel's first pivot,
    // on the recomputed norms, decides
    const double margin = sizeof(T) == 4 ? 1e-3 : 1e-7;
    if (jj > 0 && bnorm <= G.tol * nu0 * (1.0 + margin) && p >= j) {
        if (threadIdx.x == 0) S->pend = 1;
        return;
    }
    if (bnorm <= G.tol * nu0 || bnorm == 0.0 || p < j) {
        if (threadIdx.x == 0) {
            S->stop = 1;
            if (j == 0) S->nu0 = bnorm;
        }
        return;
    }
    if (p != j) {
        for (int i = threadIdx.x; i < G.m; i += blockDim.x) {
            const T t = W[i + ld * j];
            W[i + ld * j] = W[i + ld * p];
            W[i + ld * p] = t;
        }
        for (int q = threadIdx.x; q < jj; q += blockDim.x) {
            const T t = F[j + (int64_t)n * q];
            F[j + (int64_t)n * q] = F[p + (int64_t)n * q];
            F[p + (int64_t)n * q] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && p != j) {
        const int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
        double tn = nrm[j]; nrm[j] = nrm[p]; nrm[p] = tn;
        tn = nrm0[j]; nrm0[j] = nrm0[p]; nrm0[p] = tn;
    }
    for (int q = threadIdx.x; q < jj; q += blockDim.x) fj[q] = F[j + (int64_t)n * q];
    __syncthreads();
    // rows j.. of the pivot column: W[i, j] -= sum_q W[i, j0 + q] F[j, q]
    if (jj > 0)
        for (int i = j + threadIdx.x; i < G.m; i += blockDim.x) {
            T acc = W[i + ld * j];
            for (int q = 0; q < jj; ++q) acc -= W[i + ld * (j0 + q)] * fj[q];
            W[i + ld * j] = acc;
        }
    __syncthreads();
    // reflector for W[j:, j]
    T ssum = T(0);
    for (int i = j + 1 + threadIdx.x; i < G.m; i += blockDim.x) {
        const T v = W[i + ld * j];
        ssum += v * v;
    }
    hs[threadIdx.x] = ssum;
    __syncthreads();
    for (int k2 = blockDim.x / 2; k2 > 0; k2 >>= 1) {
        if (threadIdx.x < k2) hs[threadIdx.x] += hs[threadIdx.x + k2];
        __syncthreads();
    }
    const T ss = hs[0];
    const T alpha = W[j + ld * j];
    T tau = T(0), scal = T(0), beta = alpha;
    if (ss != T(0)) {
        beta = -copysign(sqrt(alpha * alpha + ss), alpha);
        tau = (beta - alpha) / beta;
        scal = T(1) / (alpha - beta);
    }
    __syncthreads();
    if (tau != T(0)) {
        for (int i = j + 1 + threadIdx.x; i < G.m; i += blockDim.x) W[i + ld * j] *= scal;
        if (threadIdx.x == 0) W[j + ld * j] = beta;
    }
    __syncthreads();
    // g[q] = sum_{i >= j} W[i, j0 + q] v_i, v_j = 1, v_i = W[i, j] below
    if (jj > 0) {
        T acc[QPB];
#pragma unroll
        for (int q = 0; q < QPB; ++q) acc[q] = T(0);
        for (int i = j + threadIdx.x; i < G.m; i += blockDim.x) {
            const T vi = i == j ? T(1) : W[i + ld * j];
#pragma unroll
            for (int q = 0; q < QPB; ++q)
                if (q < jj) acc[q] += W[i + ld * (j0 + q)] * vi;
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int q = 0; q < QPB; ++q) {
            const T v = warp_sum(acc[q]);
            if (lane == 0) part[wid][q] = v;
        }
        __syncthreads();
        if (threadIdx.x < jj) {
            T v = T(0);
            for (int w = 0; w < QPT / 32; ++w) v += part[w][threadIdx.x];
            gq[threadIdx.x] = v;
        }
    }
    if (threadIdx.x == 0) {
        if (j == 0) S->nu0 = bnorm;
        S->tau = (double)tau;
        S->k = j + 1;
        S->last_step = step;
    }
}

// F[l, jj] for the trailing columns (a warp per column), the pivot row's
// entry brought up to date, and the norm downdated
template <typename T>
__global__ void __launch_bounds__(256) bqp_f_kernel(BigArgs a, int step) {
    const BigGroup G = a.groups[blockIdx.y];
    const BigState S = a.state[blockIdx.y];
    if (S.stop || S.last_step != step) return;
    const int j = S.k - 1, j0 = S.j0, jj = j - j0;
    const int nb = a.nb;
    const int lane = threadIdx.x & 31;
    const int l = j + 1 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (l >= G.n) return;
    T* W = static_cast<T*>(a.YK) + G.y_off;
    const int64_t ld = G.ld;
    const int n = G.n;
    T* F = static_cast<T*>(a.F) + G.vec_off * nb;
    const T* gq = static_cast<const T*>(a.gv) + (int64_t)blockIdx.y * QPB;
    const T tau = (T)S.tau;
    T* col = W + ld * l;
    const T* v = W + ld * j;
    T dot = T(0);
    for (int i = j + 1 + lane; i < G.m; i += 32) dot += v[i] * col[i];
    dot = warp_sum(dot);
    if (lane == 0) {
        dot += col[j];
        T corr = T(0);
        for (int q = 0; q < jj; ++q) corr += F[l + (int64_t)n * q] * gq[q];
        const T f = tau * (dot - corr);
        F[l + (int64_t)n * jj] = f;
        // pivot row: W[j, l] -= sum_{q < jj} W[j, j0 + q] F[l, q] + F[l, jj]
        T r = col[j] - f;
        for (int q = 0; q < jj; ++q) r -= W[j + ld * (j0 + q)] * F[l + (int64_t)n * q];
        col[j] = r;
        double* nrm = a.nrm + G.vec_off;
        const double* nrm0 = a.nrm0 + G.vec_off;
        const double nn = fmax(nrm[l] - (double)r * (double)r, 0.0);
        nrm[l] = nn;
        // the downdated norm keeps ~sqrt(eps_T) relative accuracy only while
        // it stays above sqrt(eps_T) of the last exact value
        const double tol3z = sizeof(T) == 4 ? 3.4526698e-4 : 1.4901161e-8;
        if (nn <= tol3z * nrm0[l]) atomicExch(&a.state[blockIdx.y].pend, 1);
    }
}

// end of a panel: rows below the panel of the trailing columns, W -= V F^T
// (64 x 64 tiles, K = the panel's pivots)
template <typename T>
__global__ void __launch_bounds__(256) bqp_update_kernel(BigArgs a) {
    const BigGroup G = a.groups[blockIdx.z];
    const BigState S = a.state[blockIdx.z];
    if (S.stop) return;
    const int j0 = S.j0, kb = S.k - S.j0, r0 = S.k;
    if (kb <= 0) return;
    const int i0 = r0 + blockIdx.x * 64, c0 = r0 + blockIdx.y * 64;
    if (i0 >= G.m || c0 >= G.n) return;
    T* W = static_cast<T*>(a.YK) + G.y_off;
    const int64_t ld = G.ld;
    const int n = G.n;
    const T* F = static_cast<const T*>(a.F) + G.vec_off * a.nb;
    __shared__ T Vs[QPB][64 + 1];
    __shared__ T Fs[QPB][64 + 1];
    for (int q = threadIdx.x; q < 64 * QPB; q += 256) {
        const int rr = q % 64, c = q / 64;
        const int i = i0 + rr, l = c0 + rr;
        Vs[c][rr] = (c < kb && i < G.m) ? W[i + ld * (j0 + c)] : T(0);
        Fs[c][rr] = (c < kb && l < n) ? F[l + (int64_t)n * c] : T(0);
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4] = {};
    for (int c = 0; c < kb; ++c) {
        T av[4], bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) av[q] = Vs[c][tx + 16 * q];
#pragma unroll
        for (int q = 0; q < 4; ++q) bv[q] = Fs[c][ty + 16 * q];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[u][w] += av[u] * bv[w];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int i = i0 + tx + 16 * u, l = c0 + ty + 16 * w;
            if (i < G.m && l < n) W[i + ld * l] -= acc[u][w];
        }
}

// exact norms of rows k.. of the trailing columns (a warp per column)
template <typename T>
__global__ void __launch_bounds__(256) bqp_norm_kernel(BigArgs a) {
    const BigGroup G = a.groups[blockIdx.y];
    const BigState S = a.state[blockIdx.y];
    if (S.stop) return;
    const int r0 = S.k;
    const int lane = threadIdx.x & 31;
    const int l = r0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (l >= G.n) return;
    const T* col = static_cast<const T*>(a.YK) + G.y_off + G.ld * l;
    double s = 0.0;
    if constexpr (sizeof(T) == 4) {
        float sf = 0.f;
        for (int i = r0 + lane; i < G.m; i += 32) sf = fmaf(col[i], col[i], sf);
        s = (double)sf;
    } else {
        for (int i = r0 + lane; i < G.m; i += 32) s += (double)col[i] * (double)col[i];
    }
    s = warp_sum(s);
    if (lane == 0) {
        a.nrm[G.vec_off + l] = s;
        a.nrm0[G.vec_off + l] = s;
    }
}

template <typename T>
cudaError_t big_qp_panel(const BigArgs& a, int ngroups, int max_n, int max_m, int& step, cudaStream_t st) {
    if (ngroups == 0) return cudaSuccess;
    if (a.nb < 1 || a.nb > QPB) return cudaErrorInvalidValue;
    note_launch();
    bqp_start_kernel<<<(ngroups + 127) / 128, 128, 0, st>>>(a, ngroups);
    for (int jj = 0; jj < a.nb; ++jj, ++step) {
        note_launch();
        bqp_pivot_kernel<T><<<ngroups, QPT, 0, st>>>(a, step);
        note_launch();
        bqp_f_kernel<T><<<dim3((max_n + 7) / 8, ngroups), 256, 0, st>>>(a, step);
    }
    note_launch();
    bqp_update_kernel<T><<<dim3((max_m + 63) / 64, (max_n + 63) / 64, ngroups), 256, 0, st>>>(a);
    note_launch();
    bqp_norm_kernel<T><<<dim3((max_n + 7) / 8, ngroups), 256, 0, st>>>(a);
    return cudaGetLastError();
}

// T = R1^{-1} R2 (redundant columns in ascending original order), outputs
template <typename T>
__global__ void big_T_kernel(BigArgs a) {
    const BigGroup G = a.groups[blockIdx.y];
    const GroupDesc gd = a.gdesc[G.group];
    const int k = a.state[blockIdx.y].k;
    const int n = G.n, r = n - k;
    const T* W = static_cast<const T*>(a.YK) + G.y_off;
    const int64_t ld = G.ld;
    const int* perm = a.perm + G.vec_off;
    T* Tout = static_cast<T*>(a.Tws) + gd.T_off;
    int* pout = a.perm_out + gd.perm_off;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.k_out[G.group] = k;
    if (l < k) pout[l] = perm[l];
    if (l >= r) return;
    const int o = perm[k + l];
    int pos = 0;
    for (int q = 0; q < r; ++q) pos += perm[k + q] < o;
    pout[k + pos] = o;
    // back substitution in a local copy held in the T output column
    T* tcol = Tout + (int64_t)k * pos;
    const T* rcol = W + ld * (k + l);
    for (int i = k - 1; i >= 0; --i) {
        T v = rcol[i];
        for (int q = i + 1; q < k; ++q) v -= W[i + ld * q] * tcol[q];
        tcol[i] = v / W[i + ld * i];
    }
}

// ---------------------------------------------------------- launchers ----

template <typename T>
cudaError_t big_ygen(const BigArgs& a, int nbig, int64_t max_entries, cudaStream_t st) {
    if (nbig == 0) return cudaSuccess;
    dim3 grid((unsigned)std::min<int64_t>((max_entries + 255) / 256, 4096), nbig);
    note_launch();
    big_ygen_kernel<T><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t big_rho(const BigArgs& a, int ngroups, int max_m, int max_n, cudaStream_t st) {
    if (ngroups == 0) return cudaSuccess;
    dim3 gn(ngroups, 2);
    dim3 gtv((max_m + 255) / 256, ngroups, 2);
    dim3 gw((max_n + 7) / 8, ngroups, 2);
    note_launch();
    big_pow_norm_kernel<<<gn, 256, 0, st>>>(a, 2);
    for (int it = 0; it < 8; ++it) {
        note_launch();
        big_pow_tv_kernel<T><<<gtv, 256, 0, st>>>(a);
        note_launch();
        big_pow_w_kernel<T><<<gw, 256, 0, st>>>(a);
        note_launch();
        big_pow_norm_kernel<<<gn, 256, 0, st>>>(a, 0);
    }
    note_launch();
    big_pow_tv_kernel<T><<<gtv, 256, 0, st>>>(a);
    note_launch();
    big_pow_norm_kernel<<<gn, 256, 0, st>>>(a, 1);
    note_launch();
    big_tol_kernel<<<(ngroups + 127) / 128, 128, 0, st>>>(a, ngroups);
    return cudaGetLastError();
}

template <typename T>
cudaError_t big_add(void* YK, const void* YS, int64_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    note_launch();
    big_add_kernel<T><<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32), 256, 0, st>>>(
        static_cast<T*>(YK), static_cast<const T*>(YS), n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t big_qr_init(const BigArgs& a, int ngroups, int max_n, cudaStream_t st) {
    if (ngroups == 0) return cudaSuccess;
    dim3 g((max_n + 7) / 8, ngroups);
    note_launch();
    big_norm_init_kernel<T><<<g, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t big_qr_step(const BigArgs& a, int ngroups, int max_n, int j, cudaStream_t st) {
    note_launch();
    big_step_kernel<T><<<ngroups, 256, 0, st>>>(a, j);
    const int cols = max_n - j - 1;
    if (cols > 0) {
        dim3 g((cols + 7) / 8, ngroups);
        note_launch();
        big_update_kernel<T><<<g, 256, 0, st>>>(a, j);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t big_finish(const BigArgs& a, int ngroups, int max_n, cudaStream_t st) {
    if (ngroups == 0) return cudaSuccess;
    dim3 g((max_n + 127) / 128, ngroups);
    note_launch();
    big_T_kernel<T><<<g, 128, 0, st>>>(a);
    return cudaGetLastError();
}

// --------------------------------------------------- dense helpers ------

// C (m x n) += alpha op(A) op(B); 64 x 64 tiles, K staged 16 at a time.
template <typename T>
__global__ void __launch_bounds__(256) gemm_kernel(int m, int n, int kk, T alpha, const T* A, int64_t lda, int tA,
                                                   const T* B, int64_t ldb, int tB, T* C, int64_t ldc) {
    __shared__ T As[16][64 + 1];
    __shared__ T Bs[16][64 + 1];
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4] = {};
    for (int l0 = 0; l0 < kk; l0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            const int r = e % 64, l = e / 64;           // A tile: rows i0+r, k l0+l
            const int i = i0 + r, kx = l0 + l;
            T v = T(0);
            if (i < m && kx < kk) v = tA ? A[kx + lda * i] : A[i + lda * kx];
            As[l][r] = v;
            const int jj = j0 + r;                      // B tile: k l0+l, cols j0+r
            T u = T(0);
            if (jj < n && kx < kk) u = tB ? B[jj + ldb * kx] : B[kx + ldb * jj];
            Bs[l][r] = u;
        }
        __syncthreads();
        for (int l = 0; l < 16; ++l) {
            T av[4], bv[4];
            for (int q = 0; q < 4; ++q) av[q] = As[l][tx + 16 * q];
            for (int q = 0; q < 4; ++q) bv[q] = Bs[l][ty + 16 * q];
            for (int p = 0; p < 4; ++p)
                for (int q = 0; q < 4; ++q) acc[p][q] += av[p] * bv[q];
        }
        __syncthreads();
    }
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + tx + 16 * p, jj = j0 + ty + 16 * q;
            if (i < m && jj < n) C[i + ldc * jj] += alpha * acc[p][q];
        }
}

template <typename T>
cudaError_t gemm(int m, int n, int kk, T alpha, const T* A, int64_t lda, bool tA, const T* B, int64_t ldb, bool tB,
                 T* C, int64_t ldc, cudaStream_t st) {
    if (m == 0 || n == 0 || kk == 0) return cudaSuccess;
    dim3 g((m + 63) / 64, (n + 63) / 64);
    note_launch();
    gemm_kernel<T><<<g, 256, 0, st>>>(m, n, kk, alpha, A, lda, tA ? 1 : 0, B, ldb, tB ? 1 : 0, C, ldc);
    return cudaGetLastError();
}

template <typename T>
__global__ void big_gather_kernel(GeomDev g, SciDev sci, const int* rd, int r, const int* sk, int k, T* A) {
    const int n = k + r;
    const int ref = r > 0 ? rd[0] : sk[0];
    const int d = g.dim;
    const double r0 = g.x[(int64_t)d * ref], r1 = g.x[(int64_t)d * ref + 1];
    const double r2 = d == 3 ? g.x[(int64_t)d * ref + 2] : 0.0;
    const int64_t tot = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(e % n), q = (int)(e / n);
        const int i = p < r ? rd[p] : sk[p - r];
        const int j = q < r ? rd[q] : sk[q - r];
        A[e] = entry<T>(g, sci, i, j, r0, r1, r2);
    }
}

template <typename T>
__global__ void big_T_assemble_kernel(const ElimGroup* eg, int ng, const T* Tws, int k, int r, T* Tm) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * r; e += gridDim.x * blockDim.x) Tm[e] = T(0);
    __syncthreads();   // single-CTA launch
    for (int gi = 0; gi < ng; ++gi) {
        const ElimGroup G = eg[gi];
        for (int e = threadIdx.x; e < G.kg * G.rg; e += blockDim.x) {
            const int i = e % G.kg, jj = e / G.kg;
            Tm[(G.ko + i) + (int64_t)k * (G.ro + jj)] = Tws[G.T_off + e];
        }
    }
}

// X (m x n) <- X U^{-1}, U upper with diagonal; one thread per row of X
template <typename T>
__global__ void trsm_right_upper_rows(int n, const T* U, int64_t ldu, T* X, int64_t ldx, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    for (int j = 0; j < n; ++j) {
        T v = X[i + ldx * j];
        for (int l = 0; l < j; ++l) v -= X[i + ldx * l] * U[l + ldu * j];
        X[i + ldx * j] = v / U[j + ldu * j];
    }
}

// B (n x m) <- L^{-1} P B with LAPACK interchanges piv; one thread per column
template <typename T>
__global__ void piv_lower_cols(int n, const T* L, int64_t ldl, const int* piv, T* B, int64_t ldb, int m) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    T* col = B + ldb * c;
    for (int j = 0; j < n; ++j) {
        const int p = piv[j];
        if (p != j) { const T t = col[j]; col[j] = col[p]; col[p] = t; }
    }
    for (int i = 0; i < n; ++i) {
        T v = col[i];
        for (int l = 0; l < i; ++l) v -= L[i + ldl * l] * col[l];
        col[i] = v;
    }
}

// outputs of one eliminated large box (same layout as the one-CTA path)
template <typename T>
__global__ void big_elim_out_kernel(int k, int r, const T* A, int64_t ld, const T* Tm, T* pool, ElimDesc ed) {
    const T* Arr = A;
    const T* Asr = A + r;
    const T* Ars = A + ld * r;
    T* Dv = pool + ed.D_out;
    T* LUo = pool + ed.LU_out;
    T* Xo = pool + ed.X_out;
    T* Yo = pool + ed.Y_out;
    T* To = pool + ed.T_out;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t e = t0; e < r; e += stride) Dv[e] = Arr[e + ld * e];
    for (int64_t e = t0; e < (int64_t)r * r; e += stride) {
        const int i = (int)(e % r), j = (int)(e / r);
        LUo[e] = i == j ? T(0) : (i < j ? Arr[i + ld * j] / Arr[i + ld * i] : Arr[i + ld * j]);
    }
    for (int64_t e = t0; e < (int64_t)k * r; e += stride) {
        const int i = (int)(e % k), j = (int)(e / k);
        Xo[e] = Asr[i + ld * j];
        To[e] = Tm[e];
    }
    for (int64_t e = t0; e < (int64_t)r * k; e += stride) {
        const int i = (int)(e % r), j = (int)(e / r);
        Yo[e] = Ars[i + ld * j] / Arr[i + ld * i];
    }
}

// inverses of the unit triangular factors stored in LU (one thread per column)
template <typename T>
__global__ void tri_inv_cols(int n, const T* A, T* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int64_t ld = n;
    out[c + ld * c] = T(0);
    for (int i = c + 1; i < n; ++i) {
        T v = -A[i + ld * c];
        for (int l = c + 1; l < i; ++l) v -= A[i + ld * l] * out[l + ld * c];
        out[i + ld * c] = v;
    }
    for (int i = c - 1; i >= 0; --i) {
        T v = -A[i + ld * c];
        for (int l = i + 1; l < c; ++l) v -= A[i + ld * l] * out[l + ld * c];
        out[i + ld * c] = v;
    }
}

__global__ void piv_to_perm_kernel(const int* piv, int r, int* pm) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int i = 0; i < r; ++i) pm[i] = i;
    for (int j = 0; j < r; ++j) {
        const int p = piv[j];
        const int t = pm[j]; pm[j] = pm[p]; pm[p] = t;
    }
}

// ---------------------------------------------- batched elimination ----
//
// All large boxes of a sublevel are eliminated together: every stage below is
// one launch whose last grid dimension runs over the boxes.  Box e works on
// its own workspace A_e (n x n, order (rd, sk)) and T_e (k x r).

template <typename T>
struct EBox {
    int k, r, n;
    T* A;
    T* Tm;
    __device__ EBox(const BatchElimArgs& a, int e) {
        const ElimDesc& d = a.ed[e];
        k = d.k;
        r = d.r;
        n = k + r;
        A = static_cast<T*>(a.ws) + d.ws_off;
        Tm = A + (int64_t)n * n;
    }
};

template <typename T>
__global__ void be_gather_kernel(BatchElimArgs a) {
    const int e = blockIdx.y;
    const ElimDesc d = a.ed[e];
    const EBox<T> B(a, e);
    const int* sk = a.sk + d.sk_off;
    const int* rd = a.rd + d.rd_off;
    const int ref = B.r > 0 ? rd[0] : sk[0];
    const int dm = a.g.dim;
    const double r0 = a.g.x[(int64_t)dm * ref], r1 = a.g.x[(int64_t)dm * ref + 1];
    const double r2 = dm == 3 ? a.g.x[(int64_t)dm * ref + 2] : 0.0;
    const int64_t tot = (int64_t)B.n * B.n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(q % B.n), c = (int)(q / B.n);
        const int i = p < B.r ? rd[p] : sk[p - B.r];
        const int j = c < B.r ? rd[c] : sk[c - B.r];
        B.A[q] = entry<T>(a.g, a.sci, i, j, r0, r1, r2);
    }
}

template <typename T>
__global__ void be_T_kernel(BatchElimArgs a) {
    const int e = blockIdx.x;
    const ElimDesc d = a.ed[e];
    const EBox<T> B(a, e);
    for (int q = threadIdx.x; q < B.k * B.r; q += blockDim.x) B.Tm[q] = T(0);
    __syncthreads();
    const T* Tws = static_cast<const T*>(a.Tws);
    for (int gi = 0; gi < d.ngroups; ++gi) {
        const ElimGroup G = a.groups[d.grp_off + gi];
        for (int q = threadIdx.x; q < G.kg * G.rg; q += blockDim.x) {
            const int i = q % G.kg, jj = q / G.kg;
            B.Tm[(G.ko + i) + (int64_t)B.k * (G.ro + jj)] = Tws[G.T_off + q];
        }
    }
}

// the GEMMs of Lemma 2.4 and the Schur update, one op per launch:
// 0: B_sr = A_sr - A_ss T     1: B_rr -= T^T B_sr     2: B_rr -= A_rs T
// 3: B_rs = A_rs - T^T A_ss   4: S = -X Z (into the SCI pool)
template <typename T>
__global__ void __launch_bounds__(256) be_gemm_kernel(BatchElimArgs a, int op) {
    __shared__ T As[16][64 + 1];
    __shared__ T Bs[16][64 + 1];
    const int e = blockIdx.z;
    const ElimDesc d = a.ed[e];
    const EBox<T> Bx(a, e);
    const int k = Bx.k, r = Bx.r;
    const int64_t ld = Bx.n;
    T* Arr = Bx.A;
    T* Asr = Bx.A + r;
    T* Ars = Bx.A + ld * r;
    T* Ass = Bx.A + ld * r + r;
    int m, n, kk;
    const T* A;
    const T* Bm;
    T* C;
    int64_t lda, ldb, ldc;
    bool tA = false, tB = false;
    switch (op) {
        case 0: m = k; n = r; kk = k; A = Ass; lda = ld; Bm = Bx.Tm; ldb = k; C = Asr; ldc = ld; break;
        case 1: m = r; n = r; kk = k; A = Bx.Tm; lda = k; tA = true; Bm = Asr; ldb = ld; C = Arr; ldc = ld; break;
        case 2: m = r; n = r; kk = k; A = Ars; lda = ld; Bm = Bx.Tm; ldb = k; C = Arr; ldc = ld; break;
        case 3: m = r; n = k; kk = k; A = Bx.Tm; lda = k; tA = true; Bm = Ass; ldb = ld; C = Ars; ldc = ld; break;
        default:
            if (k == 0 || d.sci_out < 0) return;
            m = k; n = k; kk = r; A = Asr; lda = ld; Bm = Ars; ldb = ld;
            C = static_cast<T*>(a.sci_pool) + d.sci_out; ldc = k;
            break;
    }
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    if (i0 >= m || j0 >= n || kk == 0) return;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4] = {};
    for (int l0 = 0; l0 < kk; l0 += 16) {
        for (int q = threadIdx.x; q < 64 * 16; q += 256) {
            const int rr = q % 64, l = q / 64;
            const int i = i0 + rr, kx = l0 + l;
            T v = T(0);
            if (i < m && kx < kk) v = tA ? A[kx + lda * i] : A[i + lda * kx];
            As[l][rr] = v;
            const int jj = j0 + rr;
            T u = T(0);
            if (jj < n && kx < kk) u = tB ? Bm[jj + ldb * kx] : Bm[kx + ldb * jj];
            Bs[l][rr] = u;
        }
        __syncthreads();
        for (int l = 0; l < 16; ++l) {
            T av[4], bv[4];
            for (int q = 0; q < 4; ++q) av[q] = As[l][tx + 16 * q];
            for (int q = 0; q < 4; ++q) bv[q] = Bs[l][ty + 16 * q];
            for (int p = 0; p < 4; ++p)
                for (int q = 0; q < 4; ++q) acc[p][q] += av[p] * bv[q];
        }
        __syncthreads();
    }
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + tx + 16 * p, jj = j0 + ty + 16 * q;
            if (i < m && jj < n) {
                if (op == 4) C[i + ldc * jj] = -acc[p][q];
                else C[i + ldc * jj] -= acc[p][q];
            }
        }
}

// The same products as tensor-core problems (FP32): one TcGemmProb per box
// for op, C -= op(A) op(B) (op 4: C = -X Z); a box without work gets m = 0.
__global__ void be_probs_kernel(BatchElimArgs a, int op, TcGemmProb* out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.nbox) return;
    const ElimDesc d = a.ed[e];
    const EBox<float> Bx(a, e);
    const int k = Bx.k, r = Bx.r;
    const int64_t ld = Bx.n;
    float* Arr = Bx.A;
    float* Asr = Bx.A + r;
    float* Ars = Bx.A + ld * r;
    float* Ass = Bx.A + ld * r + r;
    TcGemmProb p{};
    p.alpha = -1.f;
    p.beta = 1;
    switch (op) {
        case 0: p = TcGemmProb{Ass, Bx.Tm, Asr, ld, k, ld, k, r, k, 0, 0, -1.f, 1}; break;
        case 1: p = TcGemmProb{Bx.Tm, Asr, Arr, k, ld, ld, r, r, k, 1, 0, -1.f, 1}; break;
        case 2: p = TcGemmProb{Ars, Bx.Tm, Arr, ld, k, ld, r, r, k, 0, 0, -1.f, 1}; break;
        case 3: p = TcGemmProb{Bx.Tm, Ass, Ars, k, ld, ld, r, k, k, 1, 0, -1.f, 1}; break;
        default: {
            const float* pool = static_cast<const float*>(a.pool);
            p = TcGemmProb{pool + d.X_out, pool + d.Y_out,
                           static_cast<float*>(a.sci_pool) + (d.sci_out < 0 ? 0 : d.sci_out), k, r, k, k, k, r, 0,
                           0, -1.f, 0};
            }
            if (k == 0 || d.sci_out < 0) p.m = 0;
            break;
    }
    if (k == 0 && op < 4) p.m = 0;
    out[e] = p;
}

// blocked LU of B_rr (Lemma 2.1), panel / interchange+TRSM / update stages
constexpr int PNT = 512;   // threads of the LU panel kernel (the pivot search spans all rows)

template <typename T>
__global__ void __launch_bounds__(PNT) be_panel_kernel(BatchElimArgs a, int j0) {
    const int e = blockIdx.x;
    const ElimDesc d = a.ed[e];
    const EBox<T> Bx(a, e);
    const int n = Bx.r;
    if (j0 >= n) return;
    const int nb = min(32, n - j0);
    const int64_t ld = Bx.n;
    T* A = Bx.A;
    int* piv = a.piv + d.piv_out;
    __shared__ T redv[PNT];
    __shared__ int redi[PNT];
    for (int j = j0 + threadIdx.x; j < j0 + nb; j += blockDim.x) piv[j] = j;
    __syncthreads();
    for (int j = j0; j < j0 + nb; ++j) {
        T best = T(-1);
        int bi = j;
        for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
            const T v = fabs(A[i + ld * j]);
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
        int p = redi[0];
        if (p < j || p >= n) p = j;
        __syncthreads();
        if (threadIdx.x == 0) piv[j] = p;
        if (p != j)
            for (int c = j0 + threadIdx.x; c < j0 + nb; c += blockDim.x) {
                const T t = A[j + ld * c];
                A[j + ld * c] = A[p + ld * c];
                A[p + ld * c] = t;
            }
        __syncthreads();
        const T dg = A[j + ld * j];
        if (dg == T(0) || !isfinite((double)dg)) {
            if (threadIdx.x == 0) atomicOr(a.status, (int)DEV_SINGULAR);
            return;
        }
        const T inv = T(1) / dg;
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const T l = A[i + ld * j] * inv;
            A[i + ld * j] = l;
            for (int c = j + 1; c < j0 + nb; ++c) A[i + ld * c] -= l * A[j + ld * c];
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void be_swap_trsm_kernel(BatchElimArgs a, int j0) {
    const int e = blockIdx.y;
    const ElimDesc d = a.ed[e];
    const EBox<T> Bx(a, e);
    const int n = Bx.r;
    if (j0 >= n) return;
    const int nb = min(32, n - j0);
    const int64_t ld = Bx.n;
    T* A = Bx.A;
    const int* piv = a.piv + d.piv_out;
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
    if (c >= j0 + nb)
        for (int i = j0; i < j0 + nb; ++i) {
            T v = A[i + ld * c];
            for (int l = j0; l < i; ++l) v -= A[i + ld * l] * A[l + ld * c];
            A[i + ld * c] = v;
        }
}

template <typename T>
__global__ void __launch_bounds__(256) be_update_kernel(BatchElimArgs a, int j0) {
    const int e = blockIdx.z;
    const EBox<T> Bx(a, e);
    const int n = Bx.r;
    if (j0 >= n) return;
    const int nb = min(32, n - j0);
    const int s = j0 + nb;
    const int i0 = s + blockIdx.x * 64, c0 = s + blockIdx.y * 64;
    if (i0 >= n || c0 >= n) return;
    const int64_t ld = Bx.n;
    T* A = Bx.A;
    __shared__ T Ls[64][33];
    __shared__ T Us[32][65];
    for (int q = threadIdx.x; q < 64 * nb; q += blockDim.x) {
        const int i = q % 64, l = q / 64;
        Ls[i][l] = (i0 + i < n) ? A[(i0 + i) + ld * (j0 + l)] : T(0);
    }
    for (int q = threadIdx.x; q < 64 * nb; q += blockDim.x) {
        const int l = q % nb, c = q / nb;
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

// ---- after the LU of B_rr: the factor outputs by blocked products --------
//
// With P B_rr = L U = L D U' (L, U' unit triangular), Lemma 2.4's blocks
// are X = B_sr U^{-1}, Z = L^{-1} P B_rs, the Schur update S = -X Z, and the
// sweeps keep Y = D^{-1} Z and the unit triangular inverses L^{-1}, U'^{-1}.
// The inverses are formed by IB x IB blocks: the diagonal blocks by
// substitution, then every block column J below the diagonal as
// X_IJ = -inv(F_II) sum_{K=J..I-1} F_IK X_KJ (F = L, or U'^T for the upper
// factor).  X and Z are blocked substitutions (only the IB x IB diagonal
// blocks enter through their inverses: multiplying by the whole explicit
// inverse measured a less accurate FP32 factor), S a tiled product.

// D, the unit factors (LU_out: L strictly below, U' strictly above, zero
// diagonal) and the row permutation P of the pivots
template <typename T>
__global__ void be_lu_out_kernel(BatchElimArgs a) {
    const int e = blockIdx.y;
    const ElimDesc d = a.ed[e];
    const EBox<T> Bx(a, e);
    const int r = Bx.r;
    const int64_t ld = Bx.n;
    const T* Arr = Bx.A;
    T* pool = static_cast<T*>(a.pool);
    T* Dv = pool + d.D_out;
    T* LUo = pool + d.LU_out;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t q = t0; q < r; q += stride) Dv[q] = Arr[q + ld * q];
    for (int64_t q = t0; q < (int64_t)r * r; q += stride) {
        const int i = (int)(q % r), j = (int)(q / r);
        LUo[q] = i == j ? T(0) : (i < j ? Arr[i + ld * j] / Arr[i + ld * i] : Arr[i + ld * j]);
    }
    if (t0 == 0) {
        int* pm = a.perm + d.piv_out;
        const int* piv = a.piv + d.piv_out;
        for (int i = 0; i < r; ++i) pm[i] = i;
        for (int j = 0; j < r; ++j) {
            const int p = piv[j];
            const int t = pm[j]; pm[j] = pm[p]; pm[p] = t;
        }
    }
}

constexpr int IB = 32;   // block size of the triangular inverses

// Unit lower factor F(i, l), i > l: L itself (UP false) or U'^T (UP true);
// its inverse's entries (i > j) go to LUi_out at (i, j) or, transposed, (j, i).
template <typename T, bool UP>
__device__ __forceinline__ T tri_f(const T* F, int64_t r, int i, int l) {
    return UP ? F[l + r * i] : F[i + r * l];
}
template <typename T, bool UP>
__device__ __forceinline__ T* tri_x(T* X, int64_t r, int i, int j) {
    return UP ? X + j + r * i : X + i + r * j;
}

// inverses of the IB x IB diagonal blocks (one warp per block and box)
template <typename T, bool UP>
__global__ void be_dinv_kernel(BatchElimArgs a) {
    const int e = blockIdx.y;
    const ElimDesc d = a.ed[e];
    const int r = d.r;
    const int b0 = blockIdx.x * IB;
    if (b0 >= r) return;
    const int nbk = min(IB, r - b0);
    const T* F = static_cast<const T*>(a.pool) + d.LU_out;
    T* X = static_cast<T*>(a.pool) + d.LUi_out;
    __shared__ T Fs[IB][IB + 1];
    __shared__ T Xs[IB][IB + 1];
    const int t = threadIdx.x;
    for (int q = t; q < IB * IB; q += 32) {
        const int i = UP ? q / IB : q % IB, l = UP ? q % IB : q / IB;   // coalesced either way
        Fs[i][l] = (i < nbk && l < nbk && i > l) ? tri_f<T, UP>(F, r, b0 + i, b0 + l) : T(0);
    }
    __syncthreads();
    if (t < nbk) {
        for (int i = 0; i < IB; ++i) Xs[i][t] = T(0);
        for (int i = t + 1; i < nbk; ++i) {
            T v = -Fs[i][t];
            for (int l = t + 1; l < i; ++l) v -= Fs[i][l] * Xs[l][t];
            Xs[i][t] = v;
        }
    }
    __syncthreads();
    for (int q = t; q < IB * IB; q += 32) {
        const int i = UP ? q / IB : q % IB, j = UP ? q % IB : q / IB;
        if (i < nbk && j < nbk && i > j) *tri_x<T, UP>(X, r, b0 + i, b0 + j) = Xs[i][j];
    }
    if (t < nbk) X[(b0 + t) + (int64_t)r * (b0 + t)] = T(0);
}

// block column J of the inverse, blocks I = J+1.. in order (one CTA per
// block column and box; 256 threads, 4 entries of the 32 x 32 block each)
template <typename T, bool UP>
__global__ void __launch_bounds__(256) be_binv_kernel(BatchElimArgs a) {
    const int e = blockIdx.y;
    const ElimDesc d = a.ed[e];
    const int r = d.r;
    const int nb = (r + IB - 1) / IB;
    const int J = blockIdx.x;
    if (J >= nb - 1) return;
    const T* F = static_cast<const T*>(a.pool) + d.LU_out;
    T* X = static_cast<T*>(a.pool) + d.LUi_out;
    __shared__ T Fs[IB][IB + 1];
    __shared__ T Xs[IB][IB + 1];
    const int t = threadIdx.x;
    const int ti = t % IB, tj = t / IB;          // entries (ti, tj + 8 q)
    for (int I = J + 1; I < nb; ++I) {
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int K = J; K < I; ++K) {
            __syncthreads();
            for (int q = t; q < IB * IB; q += 256) {
                const int i = UP ? q / IB : q % IB, l = UP ? q % IB : q / IB;
                const int gi = I * IB + i, gl = K * IB + l;
                Fs[i][l] = (gi < r && gl < r) ? tri_f<T, UP>(F, r, gi, gl) : T(0);
                // X_KJ (unit diagonal, zero above)
                const int xk = UP ? q / IB : q % IB, xj = UP ? q % IB : q / IB;
                const int gk = K * IB + xk, gj = J * IB + xj;
                T xv = T(0);
                if (gk < r && gj < r) xv = gk == gj ? T(1) : (gk > gj ? *tri_x<T, UP>(X, r, gk, gj) : T(0));
                Xs[xk][xj] = xv;
            }
            __syncthreads();
#pragma unroll 8
            for (int l = 0; l < IB; ++l) {
                const T f = Fs[ti][l];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] += f * Xs[l][tj + 8 * q];
            }
        }
        // X_IJ = -(I + S_II) acc, S_II the stored strict part of inv(F_II)
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) Xs[ti][tj + 8 * q] = acc[q];
        for (int q = t; q < IB * IB; q += 256) {
            const int i = UP ? q / IB : q % IB, l = UP ? q % IB : q / IB;
            const int gi = I * IB + i, gl = I * IB + l;
            Fs[i][l] = (i > l && gi < r && gl < r) ? *tri_x<T, UP>(X, r, gi, gl) : T(0);
        }
        __syncthreads();
        const int gi = I * IB + ti;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jj = tj + 8 * q, gj = J * IB + jj;
            T v = Xs[ti][jj];
            for (int l = 0; l < ti; ++l) v += Fs[ti][l] * Xs[l][jj];
            if (gi < r && gj < r) *tri_x<T, UP>(X, r, gi, gj) = -v;
        }
    }
}

// X = B_sr U^{-1} by block columns: X_J = (B_J - sum_{K<J} X_K U_KJ) inv(U_JJ),
// inv(U_JJ) = (I + S_JJ) D_J^{-1} with S_JJ the stored strict upper part of
// the diagonal block of U'^{-1}.  One CTA per 64 rows of X and box; thread
// (tx, ty) holds entries (tx, ty + 4 q), q < 8, of the 64 x 32 block.
template <typename T>
__global__ void __launch_bounds__(256) be_trsm_x_kernel(BatchElimArgs a) {
    const int e = blockIdx.y;
    const ElimDesc d = a.ed[e];
    const EBox<T> Bx(a, e);
    const int k = Bx.k, r = Bx.r;
    const int i0 = blockIdx.x * 64;
    if (i0 >= k) return;
    const int64_t ld = Bx.n;
    const T* Arr = Bx.A;
    const T* Asr = Bx.A + r;
    T* X = static_cast<T*>(a.pool) + d.X_out;
    const T* Si = static_cast<const T*>(a.pool) + d.LUi_out;
    const T* Dv = static_cast<const T*>(a.pool) + d.D_out;
    __shared__ T Xs[64][IB + 1];
    __shared__ T Us[IB][IB + 1];
    const int tx = threadIdx.x % 64, ty = threadIdx.x / 64;
    const int i = i0 + tx;
    const int rb = (r + IB - 1) / IB;
    for (int J = 0; J < rb; ++J) {
        T acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = J * IB + ty + 4 * q;
            acc[q] = (i < k && c < r) ? Asr[i + ld * c] : T(0);
        }
        for (int K = 0; K < J; ++K) {
            __syncthreads();
            for (int q = threadIdx.x; q < 64 * IB; q += 256) {
                const int rr = q % 64, l = q / 64, gl = K * IB + l;
                Xs[rr][l] = (i0 + rr < k && gl < r) ? X[(i0 + rr) + (int64_t)k * gl] : T(0);
            }
            for (int q = threadIdx.x; q < IB * IB; q += 256) {
                const int l = q % IB, c = q / IB, gl = K * IB + l, gc = J * IB + c;
                Us[l][c] = (gl < r && gc < r) ? Arr[gl + ld * gc] : T(0);
            }
            __syncthreads();
#pragma unroll 8
            for (int l = 0; l < IB; ++l) {
                const T xv = Xs[tx][l];
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] -= xv * Us[l][ty + 4 * q];
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; ++q) Xs[tx][ty + 4 * q] = acc[q];
        for (int q = threadIdx.x; q < IB * IB; q += 256) {
            const int l = q % IB, c = q / IB, gl = J * IB + l, gc = J * IB + c;
            Us[l][c] = (l < c && gc < r) ? Si[gl + (int64_t)r * gc] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = ty + 4 * q, gc = J * IB + c;
            T v = Xs[tx][c];
            for (int l = 0; l < c; ++l) v += Xs[tx][l] * Us[l][c];
            if (i < k && gc < r) X[i + (int64_t)k * gc] = v / Dv[gc];
        }
    }
}

// Z = L^{-1} P B_rs by block rows: Z_I = (I + S_II) (PB_I - sum_{K<I} L_IK Z_K),
// S_II the stored strict lower part of the diagonal block of L^{-1}.  Z goes
// to Y_out (scaled by D^{-1} later).  One CTA per 64 columns of Z and box;
// thread (tr, tc) holds entries (tr, tc + 8 q), q < 8, of the 32 x 64 block.
template <typename T>
__global__ void __launch_bounds__(256) be_trsm_z_kernel(BatchElimArgs a) {
    const int e = blockIdx.y;
    const ElimDesc d = a.ed[e];
    const EBox<T> Bx(a, e);
    const int k = Bx.k, r = Bx.r;
    const int j0 = blockIdx.x * 64;
    if (j0 >= k) return;
    const int64_t ld = Bx.n;
    const T* Arr = Bx.A;
    const T* Ars = Bx.A + ld * r;
    T* Z = static_cast<T*>(a.pool) + d.Y_out;
    const T* Si = static_cast<const T*>(a.pool) + d.LUi_out;
    const int* pm = a.perm + d.piv_out;
    __shared__ T Ls[IB][IB + 1];
    __shared__ T Zs[IB][64 + 1];
    const int tr = threadIdx.x % IB, tc = threadIdx.x / IB;
    const int rb = (r + IB - 1) / IB;
    for (int I = 0; I < rb; ++I) {
        const int gi = I * IB + tr;
        T acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = j0 + tc + 8 * q;
            acc[q] = (gi < r && j < k) ? Ars[pm[gi] + ld * j] : T(0);
        }
        for (int K = 0; K < I; ++K) {
            __syncthreads();
            for (int q = threadIdx.x; q < IB * IB; q += 256) {
                const int rr = q % IB, l = q / IB, g1 = I * IB + rr, g2 = K * IB + l;
                Ls[rr][l] = (g1 < r && g2 < r) ? Arr[g1 + ld * g2] : T(0);
            }
            for (int q = threadIdx.x; q < IB * 64; q += 256) {
                const int l = q % IB, c = q / IB, gl = K * IB + l;
                Zs[l][c] = (gl < r && j0 + c < k) ? Z[gl + (int64_t)r * (j0 + c)] : T(0);
            }
            __syncthreads();
#pragma unroll 8
            for (int l = 0; l < IB; ++l) {
                const T lv = Ls[tr][l];
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] -= lv * Zs[l][tc + 8 * q];
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; ++q) Zs[tr][tc + 8 * q] = acc[q];
        for (int q = threadIdx.x; q < IB * IB; q += 256) {
            const int rr = q % IB, l = q / IB, g1 = I * IB + rr, g2 = I * IB + l;
            Ls[rr][l] = (rr > l && g1 < r) ? Si[g1 + (int64_t)r * g2] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = tc + 8 * q;
            T v = Zs[tr][c];
            for (int l = 0; l < tr; ++l) v += Ls[tr][l] * Zs[l][c];
            if (gi < r && j0 + c < k) Z[gi + (int64_t)r * (j0 + c)] = v;
        }
    }
}

// S = -X Z into the SCI pool (64 x 64 tiles, K = r by 16)
template <typename T>
__global__ void __launch_bounds__(256) be_schur_kernel(BatchElimArgs a) {
    __shared__ T As[16][64 + 1];
    __shared__ T Bs[16][64 + 1];
    const int e = blockIdx.z;
    const ElimDesc d = a.ed[e];
    const int k = d.k, r = d.r;
    if (k == 0 || d.sci_out < 0) return;
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    if (i0 >= k || j0 >= k) return;
    const T* X = static_cast<const T*>(a.pool) + d.X_out;
    const T* Z = static_cast<const T*>(a.pool) + d.Y_out;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[4][4] = {};
    for (int l0 = 0; l0 < r; l0 += 16) {
        for (int q = threadIdx.x; q < 64 * 16; q += 256) {
            const int rr = q % 64, l = q / 64;
            const int i = i0 + rr, kx = l0 + l, jj = j0 + rr;
            As[l][rr] = (i < k && kx < r) ? X[i + (int64_t)k * kx] : T(0);
            Bs[l][rr] = (jj < k && kx < r) ? Z[kx + (int64_t)r * jj] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < 16; ++l) {
            T av[4], bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) av[q] = As[l][tx + 16 * q];
#pragma unroll
            for (int q = 0; q < 4; ++q) bv[q] = Bs[l][ty + 16 * q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] += av[p] * bv[q];
        }
        __syncthreads();
    }
    T* S = static_cast<T*>(a.sci_pool) + d.sci_out;
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + tx + 16 * p, jj = j0 + ty + 16 * q;
            if (i < k && jj < k) S[i + (int64_t)k * jj] = -acc[p][q];
        }
}

// Y = D^{-1} Z in place, and T
template <typename T>
__global__ void be_finish_kernel(BatchElimArgs a) {
    const int e = blockIdx.y;
    const ElimDesc d = a.ed[e];
    const EBox<T> Bx(a, e);
    const int k = Bx.k, r = Bx.r;
    T* pool = static_cast<T*>(a.pool);
    const T* Dv = pool + d.D_out;
    T* Yo = pool + d.Y_out;
    T* To = pool + d.T_out;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t q = t0; q < (int64_t)r * k; q += stride) Yo[q] /= Dv[q % r];
    for (int64_t q = t0; q < (int64_t)k * r; q += stride) To[q] = Bx.Tm[q];
}

template <typename T>
cudaError_t big_elim_batch(const BatchElimArgs& a, int max_n, int max_k, int max_r, cudaStream_t st) {
    const int nb = a.nbox;
    if (nb == 0) return cudaSuccess;
    note_launch();
    be_gather_kernel<T><<<dim3((unsigned)std::min<int64_t>(((int64_t)max_n * max_n + 255) / 256, 1024), nb), 256, 0, st>>>(a);
    note_launch();
    be_T_kernel<T><<<nb, 256, 0, st>>>(a);
    const int tk = (max_k + 63) / 64, tr = (max_r + 63) / 64;
    // FP32: the products of Lemma 2.4 and the Schur update on the tensor cores
    TcGemmProb* probs = static_cast<TcGemmProb*>(a.gemm_probs);
    const bool tcg = sizeof(T) == 4 && probs != nullptr;
    auto tc_op = [&](int op, int mm, int nn) -> cudaError_t {
        note_launch();
        be_probs_kernel<<<(nb + 127) / 128, 128, 0, st>>>(a, op, probs + (int64_t)op * nb);
        return launch_tc_gemm(probs + (int64_t)op * nb, nb, mm, nn, a.status, DEV_TIMEOUT, st);
    };
    if (max_k > 0 && tcg) {
        cudaError_t e;
        if ((e = tc_op(0, max_k, max_r)) != cudaSuccess) return e;
        if ((e = tc_op(1, max_r, max_r)) != cudaSuccess) return e;
        if ((e = tc_op(2, max_r, max_r)) != cudaSuccess) return e;
        if ((e = tc_op(3, max_r, max_k)) != cudaSuccess) return e;
    } else if (max_k > 0) {
        note_launch();
        be_gemm_kernel<T><<<dim3(tk, tr, nb), 256, 0, st>>>(a, 0);
        note_launch();
        be_gemm_kernel<T><<<dim3(tr, tr, nb), 256, 0, st>>>(a, 1);
        note_launch();
        be_gemm_kernel<T><<<dim3(tr, tr, nb), 256, 0, st>>>(a, 2);
        note_launch();
        be_gemm_kernel<T><<<dim3(tr, tk, nb), 256, 0, st>>>(a, 3);
    }
    for (int j0 = 0; j0 < max_r; j0 += 32) {
        note_launch();
        be_panel_kernel<T><<<nb, PNT, 0, st>>>(a, j0);
        note_launch();
        be_swap_trsm_kernel<T><<<dim3((max_r + 127) / 128, nb), 128, 0, st>>>(a, j0);
        const int rest = max_r - j0 - 32;
        if (rest > 0) {
            note_launch();
            be_update_kernel<T><<<dim3((rest + 63) / 64, (rest + 63) / 64, nb), 256, 0, st>>>(a, j0);
        }
    }
    note_launch();
    be_lu_out_kernel<T><<<dim3((unsigned)std::min<int64_t>(((int64_t)max_r * max_r + 255) / 256, 512), nb), 256, 0, st>>>(a);
    const int rb = (max_r + IB - 1) / IB;
    note_launch();
    be_dinv_kernel<T, false><<<dim3(rb, nb), 32, 0, st>>>(a);
    note_launch();
    be_dinv_kernel<T, true><<<dim3(rb, nb), 32, 0, st>>>(a);
    if (rb > 1) {
        note_launch();
        be_binv_kernel<T, false><<<dim3(rb - 1, nb), 256, 0, st>>>(a);
        note_launch();
        be_binv_kernel<T, true><<<dim3(rb - 1, nb), 256, 0, st>>>(a);
    }
    if (max_k > 0) {
        note_launch();
        be_trsm_x_kernel<T><<<dim3(tk, nb), 256, 0, st>>>(a);
        note_launch();
        be_trsm_z_kernel<T><<<dim3(tk, nb), 256, 0, st>>>(a);
        if (tcg) {
            const cudaError_t e = tc_op(4, max_k, max_k);
            if (e != cudaSuccess) return e;
        } else {
            note_launch();
            be_schur_kernel<T><<<dim3(tk, tk, nb), 256, 0, st>>>(a);
        }
    }
    note_launch();
    be_finish_kernel<T><<<dim3((unsigned)std::clamp<int64_t>(((int64_t)max_k * max_r + 255) / 256, 1, 512), nb), 256,
                           0, st>>>(a);
    return cudaGetLastError();
}

#define HIF_INST(T)                                                                                            \
    template cudaError_t big_ygen<T>(const BigArgs&, int, int64_t, cudaStream_t);                              \
    template cudaError_t big_rho<T>(const BigArgs&, int, int, int, cudaStream_t);                              \
    template cudaError_t big_add<T>(void*, const void*, int64_t, cudaStream_t);                                \
    template cudaError_t big_qr_init<T>(const BigArgs&, int, int, cudaStream_t);                               \
    template cudaError_t big_qr_step<T>(const BigArgs&, int, int, int, cudaStream_t);                          \
    template cudaError_t big_qp_panel<T>(const BigArgs&, int, int, int, int&, cudaStream_t);                   \
    template cudaError_t big_finish<T>(const BigArgs&, int, int, cudaStream_t);                                \
    template cudaError_t big_elim_batch<T>(const BatchElimArgs&, int, int, int, cudaStream_t);
HIF_INST(double)
HIF_INST(float)

}  // namespace hif
