// Skeletonization kernels of one sublevel (sm_103a).
//
//  fold_kernel   one CTA per box c: generates the proxy matrix Y_c of Eq. (3.3)
//                (near-field rows A_{cN,c}, A_{c,cN}^T and proxy rows of
//                Lemma 3.3; for symmetric A only A_{cN,c} and the outgoing
//                proxy rows, the Y'_c of Sec. 5, which has the same ID)
//                chunk by chunk in shared memory and folds every
//                chunk into the triangular factor R_c of Y_c = Q_c R_c by
//                Householder reflections; Y_c itself never reaches HBM.  In
//                second-kind mode it also accumulates the Gram matrices of the
//                kernel part Y^K and the SCI part Y^S (Sec. 4.4).
//  id_kernel     one CTA per column group g: rho_g = min(1, |Y^K_g|/|Y^S_g|)
//                by power iteration, then the column-pivoted QR interpolative
//                decomposition (Lemma 2.2) of R_c[:, g] -- equal to the ID of
//                Y_c[:, g] because Q_c has orthonormal columns.
//  elim_kernel   one CTA per box: the B blocks of Lemma 2.4, LU with partial
//                pivoting of B_rr (Lemma 2.1), X, Y and the Schur update
//                B_ss - B_sr B_rr^{-1} B_rs recorded as a new SCI block.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <vector>

#include "cta_linalg.cuh"
#include "hif_common.cuh"
#include "launch.h"

namespace hif {

namespace {

template <typename T>
__device__ inline T* align_ptr(unsigned char*& p, size_t count) {
    uintptr_t v = reinterpret_cast<uintptr_t>(p);
    v = (v + 15) & ~uintptr_t(15);
    T* out = reinterpret_cast<T*>(v);
    p = reinterpret_cast<unsigned char*>(v + count * sizeof(T));
    return out;
}

}  // namespace

// ------------------------------------------------------------- fold ------
//
// One CTA per box; thread t owns the columns l = t + q * blockDim.x
// (q < CPT) of Y_c.  Y_c is generated RC rows at a time; each thread holds its
// columns' RC entries in registers and folds them into its columns of R by
// Householder reflections of [R; C]: at step j the owner of column j forms
// the reflector from its registers and publishes it (RC values and tau) in
// shared memory, then every column l > j applies it to its registers and to
// R[j][l].  Column l of R is touched by its owner only, so one CTA barrier
// per step suffices (the reflector buffer is double-buffered), and the next
// step's R[j + 1][l] is loaded a step ahead.  R lives in shared memory as a
// packed upper triangle, column l at l (l + 1) / 2 (triangular numbers are
// distinct modulo 32, so a warp's accesses of one row are free of bank
// conflicts), or, when it does not fit, row-major in global memory.  In
// second-kind mode the chunk's kernel and SCI parts also pass through shared
// memory for the Gram matrices of Y^K and Y^S inside each column group
// (Sec. 4.4), stored diagonal-major: G[l][l + t] at t * n + l.
template <typename T, int RC, int CPT>
__global__ void __launch_bounds__(256, CPT == 1 ? 2 : 1) fold_kernel(FoldArgs args) {
    const BoxDesc bx = args.boxes[args.box_list[blockIdx.x]];
    const int n = bx.n;
    const int NT = blockDim.x;
    const bool sym = bx.sym != 0;               // one row per pair: Y'_c
    const int ppc = sym ? RC : RC / 2;          // pairs per chunk
    const int nsub = args.sci.nsub;
    const bool scival = bx.has_sci && nsub > 0;
    const bool grams = scival && args.second_kind;
    const int dim = args.g.dim;
    const int kid = args.g.kernel_id;

    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* sp = smem;
    T* rxl = align_ptr<T>(sp, (size_t)RC * 3);
    T* rb = align_ptr<T>(sp, RC);
    T* rwc = align_ptr<T>(sp, RC);
    int* rid = align_ptr<int>(sp, RC);
    int* rcm = align_ptr<int>(sp, RC);           // row component (real embedding, kernel 2)
    T* vbuf = align_ptr<T>(sp, 2 * RC);
    T* taub = align_ptr<T>(sp, 2);
    T* CK = align_ptr<T>(sp, (size_t)RC * n);    // the chunk (its kernel part in second-kind mode)
    T* CS = grams ? align_ptr<T>(sp, (size_t)RC * n) : nullptr;
    T* const Rglob = static_cast<T*>(args.Rws) + bx.R_off;
    T* const Rpack = args.R_in_smem ? align_ptr<T>(sp, (size_t)n * (n + 1) / 2) : nullptr;
    T* GK = grams ? static_cast<T*>(args.GKws) + bx.R_off : nullptr;
    T* GS = grams ? static_cast<T*>(args.GSws) + bx.R_off : nullptr;

    const double c0 = bx.ctr[0], c1 = bx.ctr[1], c2 = dim == 3 ? bx.ctr[2] : 0.0;
    // column data of this thread's columns
    int jid[CPT], lend[CPT];
    T xj0[CPT], xj1[CPT], xj2[CPT], cwc[CPT], cb[CPT], cbw[CPT];
    T* Rcol[CPT];                               // R[j][l] at Rcol[q][j * rstride]
    const int64_t rstride = args.R_in_smem ? 1 : n;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int l = threadIdx.x + q * NT;
        jid[q] = 0;
        lend[q] = 0;
        xj0[q] = xj1[q] = xj2[q] = cwc[q] = cb[q] = cbw[q] = T(0);
        Rcol[q] = args.R_in_smem ? Rpack + (size_t)l * (l + 1) / 2 : Rglob + l;
        if (l < n) {
            const int j = args.cols[bx.col_off + l];
            jid[q] = j;
            xj0[q] = (T)(args.g.x[(int64_t)dim * j + 0] - c0);
            xj1[q] = (T)(args.g.x[(int64_t)dim * j + 1] - c1);
            xj2[q] = dim == 3 ? (T)(args.g.x[(int64_t)dim * j + 2] - c2) : T(0);
            cwc[q] = (T)(args.g.w[j] * args.g.c[j]);
            cb[q] = (T)args.g.b[j];
            cbw[q] = (T)(args.g.b[j] * args.g.w[j]);
            for (int gi = 0; gi < bx.ngroups; ++gi) {
                const GroupDesc gd = args.groups[bx.grp_off + gi];
                if (l >= gd.col0 && l < gd.col0 + gd.n) lend[q] = gd.col0 + gd.n;
            }
            for (int j2 = 0; j2 < (args.R_in_smem ? l + 1 : n); ++j2) Rcol[q][j2 * rstride] = T(0);
            if (grams)
                for (int t = 0; t < n - l; ++t) {
                    GK[(int64_t)t * n + l] = T(0);
                    GS[(int64_t)t * n + l] = T(0);
                }
        }
    }

    const int* near = args.near + bx.near_off;
    const int npairs = bx.m_near + args.P;
    T c[CPT][RC];
    for (int p0 = 0; p0 < npairs; p0 += ppc) {
        const int np = min(ppc, npairs - p0);
        __syncthreads();                        // previous chunk's row data and Gram reads done
        for (int q = threadIdx.x; q < ppc; q += NT) {
            const int p = p0 + q;
            rcm[q] = 0;
            if (q >= np) {
                rid[q] = -2;
            } else if (p < bx.m_near) {
                const int i = near[p];
                rid[q] = i;
                rcm[q] = args.g.ncomp == 2 ? (i & 1) : 0;
                rxl[3 * q + 0] = (T)(args.g.x[(int64_t)dim * i + 0] - c0);
                rxl[3 * q + 1] = (T)(args.g.x[(int64_t)dim * i + 1] - c1);
                rxl[3 * q + 2] = dim == 3 ? (T)(args.g.x[(int64_t)dim * i + 2] - c2) : T(0);
                rb[q] = (T)args.g.b[i];
                rwc[q] = (T)(args.g.w[i] * args.g.c[i]);
            } else {
                const int kx = p - bx.m_near;
                rid[q] = -1;
                rcm[q] = args.g.ncomp == 2 ? (kx & 1) : 0;
                rxl[3 * q + 0] = (T)(bx.radius * args.proxy[dim * kx + 0]);
                rxl[3 * q + 1] = (T)(bx.radius * args.proxy[dim * kx + 1]);
                rxl[3 * q + 2] = dim == 3 ? (T)(bx.radius * args.proxy[dim * kx + 2]) : T(0);
                rb[q] = T(1);
                rwc[q] = T(1);
            }
        }
        __syncthreads();
        // ---- this thread's columns of the chunk, staged in shared memory:
        // rows (2q, 2q+1) = (outgoing, incoming) of pair q, or row q alone
        // for symmetric A; kernel and SCI parts apart when the Grams need them
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int l = threadIdx.x + q * NT;
            if (l < n) {
                for (int pq = 0; pq < ppc; ++pq) {
                    T k1, k2, s1, s2;
                    y_pair<T>(kid, rid[pq], rxl[3 * pq], rxl[3 * pq + 1], rxl[3 * pq + 2], rb[pq], rwc[pq], jid[q],
                              xj0[q], xj1[q], xj2[q], cwc[q], cb[q], cbw[q], scival, args.sci, k1, k2, s1, s2,
                              rcm[pq], (T)args.g.wavenumber);
                    const int i1 = sym ? pq : 2 * pq;
                    if (grams) {
                        CK[i1 * n + l] = k1;
                        CS[i1 * n + l] = s1;
                        if (!sym) {
                            CK[(i1 + 1) * n + l] = k2;
                            CS[(i1 + 1) * n + l] = s2;
                        }
                    } else {
                        CK[i1 * n + l] = k1 + s1;
                        if (!sym) CK[(i1 + 1) * n + l] = k2 + s2;
                    }
                }
#pragma unroll
                for (int i = 0; i < RC; ++i) c[q][i] = grams ? CK[i * n + l] + CS[i * n + l] : CK[i * n + l];
            } else {
#pragma unroll
                for (int i = 0; i < RC; ++i) c[q][i] = T(0);
            }
        }
        // ---- Gram matrices of Y^K_g and Y^S_g (row l, l <= l2 < group end)
        if (grams) {
            __syncthreads();
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const int l = threadIdx.x + q * NT;
                if (l >= n) continue;
                for (int l2 = l; l2 < lend[q]; ++l2) {
                    T gk = T(0), gs = T(0);
#pragma unroll 8
                    for (int i = 0; i < RC; ++i) {
                        gk += CK[i * n + l] * CK[i * n + l2];
                        gs += CS[i * n + l] * CS[i * n + l2];
                    }
                    GK[(int64_t)(l2 - l) * n + l] += gk;
                    GS[(int64_t)(l2 - l) * n + l] += gs;
                }
            }
        }
        // ---- fold the chunk into R: Householder QR of [R; C]
        T rcur[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) rcur[q] = threadIdx.x + q * NT < n ? Rcol[q][0] : T(0);
        for (int j = 0; j < n; ++j) {
            const int buf = j & 1;
            // the next step's R[j + 1][l], read a step ahead (only this thread writes it)
            T rnext[CPT];
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const int l = threadIdx.x + q * NT;
                rnext[q] = (l < n && j + 1 <= l) ? Rcol[q][(j + 1) * rstride] : T(0);
            }
            const int oq = j / NT;                   // the owner's slot
            if (threadIdx.x == j % NT) {
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    if (q != oq) continue;
                    T q0 = T(0), q1 = T(0), q2 = T(0), q3 = T(0);
#pragma unroll
                    for (int i = 0; i < RC; i += 4) {
                        q0 += c[q][i] * c[q][i];
                        if (i + 1 < RC) q1 += c[q][i + 1] * c[q][i + 1];
                        if (i + 2 < RC) q2 += c[q][i + 2] * c[q][i + 2];
                        if (i + 3 < RC) q3 += c[q][i + 3] * c[q][i + 3];
                    }
                    const T ss = (q0 + q1) + (q2 + q3);
                    T tau = T(0);
                    if (ss != T(0)) {
                        const T alpha = rcur[q];
                        const T beta = -copysign(sqrt(alpha * alpha + ss), alpha);
                        tau = (beta - alpha) / beta;
                        const T scal = T(1) / (alpha - beta);
                        Rcol[q][j * rstride] = beta;
#pragma unroll
                        for (int i = 0; i < RC; ++i) vbuf[buf * RC + i] = c[q][i] * scal;
                    }
                    taub[buf] = tau;
                }
            }
            __syncthreads();
            const T tau = taub[buf];
            if (tau != T(0)) {
                const T* v = vbuf + buf * RC;
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    const int l = threadIdx.x + q * NT;
                    if (l > j && l < n) {
                        T w0 = rcur[q], w1 = T(0), w2 = T(0), w3 = T(0);
#pragma unroll
                        for (int i = 0; i < RC; i += 4) {
                            w0 += v[i] * c[q][i];
                            if (i + 1 < RC) w1 += v[i + 1] * c[q][i + 1];
                            if (i + 2 < RC) w2 += v[i + 2] * c[q][i + 2];
                            if (i + 3 < RC) w3 += v[i + 3] * c[q][i + 3];
                        }
                        const T w = ((w0 + w1) + (w2 + w3)) * tau;
                        Rcol[q][j * rstride] = rcur[q] - w;
#pragma unroll
                        for (int i = 0; i < RC; ++i) c[q][i] -= w * v[i];
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < CPT; ++q) rcur[q] = rnext[q];
        }
    }
    if (args.R_in_smem)
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int l = threadIdx.x + q * NT;
            if (l < n)
                for (int j = 0; j < n; ++j) Rglob[(int64_t)j * n + l] = j <= l ? Rcol[q][j] : T(0);
        }
}

// Block-wide argmax of (v, original index o) over one candidate per thread:
// largest v, ties to the lowest o; candidates with pos < 0 are ignored.
// Returns the winner's pos on every thread (-1 if none).  Two barriers.
__device__ inline int cta_argmax_v_o(double v, int o, int pos, double* wv, int* wo, int* wp) {
    for (int off = 16; off > 0; off >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, off);
        const int o2 = __shfl_xor_sync(0xffffffffu, o, off);
        const int p2 = __shfl_xor_sync(0xffffffffu, pos, off);
        if (p2 >= 0 && (pos < 0 || v2 > v || (v2 == v && o2 < o))) { v = v2; o = o2; pos = p2; }
    }
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) { wv[warp] = v; wo[warp] = o; wp[warp] = pos; }
    __syncthreads();
    if (warp == 0) {
        const int lane = threadIdx.x & 31;
        v = lane < nw ? wv[lane] : -1.0;
        o = lane < nw ? wo[lane] : (1 << 30);
        pos = lane < nw ? wp[lane] : -1;
        for (int off = 16; off > 0; off >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, v, off);
            const int o2 = __shfl_xor_sync(0xffffffffu, o, off);
            const int p2 = __shfl_xor_sync(0xffffffffu, pos, off);
            if (p2 >= 0 && (pos < 0 || v2 > v || (v2 == v && o2 < o))) { v = v2; o = o2; pos = p2; }
        }
        if (lane == 0) wp[32] = pos;
    }
    __syncthreads();
    return wp[32];
}

// Column-pivoted Householder QR of W (mrow x ng; element (i, l) at
// W[i * rs + l * cs], overwritten) to relative tolerance tol (Lemma 2.2 with
// the adaptive rank of Sec. 2.2): pivot = largest remaining column 2-norm
// (ties: lowest original index), norms recomputed exactly in FP64 after every
// step, stop at the first step whose pivot norm is <= tol times the first
// one.  Writes k, the column order (skeletons in pivot order, then
// redundants in ascending order) and T = R1^{-1} R2 (k x (ng-k),
// column-major, columns in the redundant order).  Row-major W (cs = 1) makes
// the per-column sweeps of the trailing update coalesced.  perm, rank_of: ng
// ints; wv/wo/wp: 33 entries of scratch each.
template <typename T>
__device__ void cpqr_id(T* W, int rs, int cs, int mrow, int ng, double tol, double* nrm, int* perm,
                        int* rank_of, double* wv, int* wo, int* wp, T* hh, T* Tout, int* pout, int* kout) {
    for (int l = threadIdx.x; l < ng; l += blockDim.x) perm[l] = l;
    // ---- column-pivoted Householder QR with exact norm recomputation
    for (int l = threadIdx.x; l < ng; l += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < mrow; ++i) {
            const double v = (double)W[i * rs + l * cs];
            s += v * v;
        }
        nrm[l] = s;
    }
    __syncthreads();
    const int kmax = min(mrow, ng);
    double nu0 = 0.0;
    int k = 0;
    for (int j = 0; j < kmax; ++j) {
        // pivot: largest remaining norm, ties to the lowest original column
        double best = -1.0;
        int bo = 1 << 30, bl = -1;
        for (int l = j + threadIdx.x; l < ng; l += blockDim.x) {
            const double v = nrm[l];
            if (v > best || (v == best && perm[l] < bo)) { best = v; bo = perm[l]; bl = l; }
        }
        const int p = cta_argmax_v_o(best, bo, bl, wv, wo, wp);
        if (p < j) break;                                  // no comparable norm left
        const double bnorm = sqrt(fmax(nrm[p], 0.0));
        if (j == 0) nu0 = bnorm;
        if (bnorm <= tol * nu0 || bnorm == 0.0) break;
        if (p != j) {
            for (int i = threadIdx.x; i < mrow; i += blockDim.x) {
                const T t = W[i * rs + j * cs];
                W[i * rs + j * cs] = W[i * rs + p * cs];
                W[i * rs + p * cs] = t;
            }
        }
        __syncthreads();
        if (p != j && threadIdx.x == 0) {
            const int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
            const double tn = nrm[j]; nrm[j] = nrm[p]; nrm[p] = tn;
        }
        // Householder reflector for W[j:, j]
        if (threadIdx.x < 32) {
            T s = T(0);
            for (int i = j + 1 + threadIdx.x; i < mrow; i += 32) {
                const T v = W[i * rs + j * cs];
                s += v * v;
            }
            s = warp_sum(s);
            if (threadIdx.x == 0) {
                const T alpha = W[j * rs + j * cs];
                if (s == T(0)) {
                    hh[0] = T(0);
                    hh[1] = T(0);
                } else {
                    const T beta = -copysign(sqrt(alpha * alpha + s), alpha);
                    hh[0] = (beta - alpha) / beta;
                    hh[1] = T(1) / (alpha - beta);
                    W[j * rs + j * cs] = beta;
                }
            }
        }
        __syncthreads();
        const T tau = hh[0];
        if (tau != T(0)) {
            const T scal = hh[1];
            for (int i = j + 1 + threadIdx.x; i < mrow; i += blockDim.x) W[i * rs + j * cs] *= scal;
        }
        __syncthreads();
        for (int l = j + 1 + threadIdx.x; l < ng; l += blockDim.x) {
            T* col = W + l * cs;
            const T* v = W + j * cs;
            if (tau != T(0)) {
                T w = col[j * rs];
                for (int i = j + 1; i < mrow; ++i) w += v[i * rs] * col[i * rs];
                w *= tau;
                col[j * rs] -= w;
                for (int i = j + 1; i < mrow; ++i) col[i * rs] -= w * v[i * rs];
            }
            double s = 0.0;
            for (int i = j + 1; i < mrow; ++i) {
                const double c = (double)col[i * rs];
                s += c * c;
            }
            nrm[l] = s;
        }
        __syncthreads();
        k = j + 1;
    }
    __syncthreads();
    // ---- T = R1^{-1} R2, written with the redundant columns in ascending order
    const int r = ng - k;
    for (int l = threadIdx.x; l < r; l += blockDim.x) {
        const int o = perm[k + l];
        int pos = 0;
        for (int q = 0; q < r; ++q) pos += perm[k + q] < o;
        rank_of[l] = pos;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < r; l += blockDim.x) {
        T* col = W + (k + l) * cs;
        for (int i = k - 1; i >= 0; --i) {
            T v = col[i * rs];
            for (int q = i + 1; q < k; ++q) v -= W[i * rs + q * cs] * col[q * rs];
            col[i * rs] = v / W[i * rs + i * cs];
        }
        const int pos = rank_of[l];
        for (int i = 0; i < k; ++i) Tout[i + (int64_t)k * pos] = col[i * rs];
    }
    for (int l = threadIdx.x; l < k; l += blockDim.x) pout[l] = perm[l];
    for (int l = threadIdx.x; l < r; l += blockDim.x) pout[k + rank_of[l]] = perm[k + l];
    if (threadIdx.x == 0) *kout = k;
}


template <typename T>
__device__ double group_rho(const T* GKb, const T* GSb, int n, int col0, int ng, T* vec, double* redv);
template <typename T>
__device__ void id_group(const IdArgs& args, int gidx);

// Persistent: each CTA takes groups from a work queue (largest first, so the
// long pivoted QRs start early and the small ones fill in behind them).
template <typename T>
__global__ void __launch_bounds__(128) id_kernel(IdArgs args) {
    __shared__ int item;
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(args.next_item, 1);
        __syncthreads();
        const int it = item;
        __syncthreads();
        if (it >= args.nitems) break;
        id_group<T>(args, args.group_list[it]);
        __syncthreads();
    }
}

template <typename T>
__device__ void id_group(const IdArgs& args, const int gidx) {
    const GroupDesc gd = args.groups[gidx];
    const BoxDesc bx = args.boxes[gd.box];
    const int n = bx.n;
    const int ng = gd.n;
    const int mrow = gd.col0 + ng;                 // rows of R[:, g] that can be nonzero
    const int ldw = ng;                            // W = R[:mrow, g], row-major
    const T* R = static_cast<const T*>(args.Rws) + bx.R_off;

    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* sp = smem;
    double* nrm = align_ptr<double>(sp, ng);
    int* perm = align_ptr<int>(sp, ng);
    int* rank_of = align_ptr<int>(sp, ng);
    double* redv = align_ptr<double>(sp, blockDim.x);
    int* redi = align_ptr<int>(sp, 72);
    T* vec = align_ptr<T>(sp, 2 * (size_t)ng);
    T* hh = align_ptr<T>(sp, 4);
    T* W;
    if (args.W_in_smem) W = align_ptr<T>(sp, (size_t)mrow * ng);
    else W = static_cast<T*>(args.Wws) + args.W_off[gidx];

    for (int e = threadIdx.x; e < mrow * ng; e += blockDim.x) {
        const int i = e / ng, l = e % ng;
        W[(int64_t)i * ldw + l] = R[(int64_t)i * n + gd.col0 + l];
    }
    __syncthreads();

    // ---- rho_g (Sec. 4.4)
    double rho = 1.0;
    if (args.second_kind && gd.has_sci && bx.has_sci && args.GKws != nullptr)
        rho = group_rho<T>(static_cast<const T*>(args.GKws) + bx.R_off, static_cast<const T*>(args.GSws) + bx.R_off,
                           n, gd.col0, ng, vec, redv);
    double tol = rho * args.eps;
    if (tol < args.tol_floor) tol = args.tol_floor;

    cpqr_id<T>(W, ldw, 1, mrow, ng, tol, nrm, perm, rank_of, redv, redi, redi + 36, hh,
               static_cast<T*>(args.Tws) + gd.T_off, args.perm_out + gd.perm_off, args.k_out + gidx);
}

// rho_g = min(1, |Y^K_g| / |Y^S_g|) (Sec. 4.4) from the Gram matrices of the
// group's kernel and SCI parts (n x n box Grams, diagonal-major upper
// triangles): 8 power iterations from the normalized all-ones vector, then
// |Y v| = sqrt(v^T G v).  vec: 2 ng scratch, redv: blockDim doubles.
template <typename T>
__device__ double group_rho(const T* GKb, const T* GSb, int n, int col0, int ng, T* vec, double* redv) {
    double rho = 1.0;
    {
        double est[2];
        for (int which = 0; which < 2; ++which) {
            const T* G = which == 0 ? GKb : GSb;
            T* v = vec;
            T* wv = vec + ng;
            for (int l = threadIdx.x; l < ng; l += blockDim.x) v[l] = T(1) / sqrt(T(ng));
            __syncthreads();
            double result = 0.0;
            for (int it = 0; it <= 8; ++it) {
                // w = G v (G symmetric, upper triangle stored diagonal-major)
                for (int l = threadIdx.x; l < ng; l += blockDim.x) {
                    T acc = T(0);
                    const int gl = col0 + l;
                    for (int q = 0; q < ng; ++q) {
                        const int gq = col0 + q;
                        // diagonal-major upper triangle: G[a][a + t] at t * n + a
                        const T gv = gl <= gq ? G[(int64_t)(gq - gl) * n + gl] : G[(int64_t)(gl - gq) * n + gq];
                        acc += gv * v[q];
                    }
                    wv[l] = acc;
                }
                __syncthreads();
                // it < 8: normalize; it == 8: |Y v|^2 = v^T G v
                double part = 0.0;
                for (int l = threadIdx.x; l < ng; l += blockDim.x)
                    part += it < 8 ? (double)wv[l] * (double)wv[l] : (double)v[l] * (double)wv[l];
                redv[threadIdx.x] = part;
                __syncthreads();
                for (int s = blockDim.x / 2; s > 0; s >>= 1) {
                    if (threadIdx.x < s) redv[threadIdx.x] += redv[threadIdx.x + s];
                    __syncthreads();
                }
                const double tot = redv[0];
                __syncthreads();
                if (it == 8) { result = sqrt(fmax(tot, 0.0)); break; }
                if (tot == 0.0) { result = 0.0; break; }
                const double inv = 1.0 / sqrt(tot);
                for (int l = threadIdx.x; l < ng; l += blockDim.x) v[l] = (T)(wv[l] * inv);
                __syncthreads();
            }
            est[which] = result;
        }
        if (est[1] > 0.0) rho = fmin(1.0, est[0] / est[1]);
    }
    return rho;
}

// Tolerances of the large groups whose box was folded into R: one CTA per
// group, rho_g from the box Grams when the group has SCI (Sec. 4.4).
template <typename T>
__global__ void __launch_bounds__(128) gram_tol_kernel(GramTolArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* sp = smem;
    BigGroup& G = a.groups[blockIdx.x];
    const GroupDesc gd = a.gdesc[G.group];
    const BoxDesc bx = a.boxes[gd.box];
    double* redv = align_ptr<double>(sp, blockDim.x);
    T* vec = align_ptr<T>(sp, 2 * (size_t)gd.n);
    double rho = 1.0;
    if (G.need_rho && a.GKws != nullptr)
        rho = group_rho<T>(static_cast<const T*>(a.GKws) + bx.R_off, static_cast<const T*>(a.GSws) + bx.R_off, bx.n,
                           gd.col0, gd.n, vec, redv);
    double tol = rho * a.eps;
    if (tol < a.tol_floor) tol = a.tol_floor;
    if (threadIdx.x == 0) G.tol = tol;
}

// R (n x n row-major, upper triangle) -> column-major with leading dimension n
template <typename T>
__global__ void r_colmajor_kernel(const T* R, int n, T* out) {
    const int64_t tot = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        out[e] = R[i * n + j];
    }
}

// ------------------------------------------------------ elimination ------

// One box of the elimination (a CTA's work item); every return is uniform
// over the CTA.
template <typename T>
__device__ void elim_box(const ElimArgs& args, int bi) {
    const ElimDesc ed = args.boxes[bi];
    const int k = ed.k, r = ed.r, n = k + r;
    T* A = static_cast<T*>(args.ws) + ed.ws_off;   // n x n, order (rd, sk), column-major
    T* Tm = A + (int64_t)n * n;          // k x r
    const int* sk = args.sk_ids + ed.sk_off;
    const int* rd = args.rd_ids + ed.rd_off;
    __shared__ T redv[128];
    __shared__ int redi[128];
    int* piv = args.piv_pool + ed.piv_out;

    // interpolation matrix T = diag(T_g)
    for (int e = threadIdx.x; e < k * r; e += blockDim.x) Tm[e] = T(0);
    __syncthreads();
    for (int gi = 0; gi < ed.ngroups; ++gi) {
        const ElimGroup eg = args.groups[ed.grp_off + gi];
        const T* Tg = static_cast<const T*>(args.Tws) + eg.T_off;
        for (int e = threadIdx.x; e < eg.kg * eg.rg; e += blockDim.x) {
            const int i = e % eg.kg, j = e / eg.kg;
            Tm[(eg.ko + i) + (int64_t)k * (eg.ro + j)] = Tg[e];
        }
    }
    // active-matrix block A_cc in (rd, sk) order
    const int ref = r > 0 ? rd[0] : sk[0];
    const int d = args.g.dim;
    const double r0 = args.g.x[(int64_t)d * ref], r1 = args.g.x[(int64_t)d * ref + 1];
    const double r2 = d == 3 ? args.g.x[(int64_t)d * ref + 2] : 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int p = e % n, q = e / n;
        const int i = p < r ? rd[p] : sk[p - r];
        const int j = q < r ? rd[q] : sk[q - r];
        A[e] = entry<T>(args.g, args.sci, i, j, r0, r1, r2);
    }
    __syncthreads();
    T* Arr = A;
    T* Asr = A + r;
    T* Ars = A + (int64_t)n * r;
    T* Ass = A + (int64_t)n * r + r;
    const int64_t ld = n;
    // B_sr = A_sr - A_ss T            (Lemma 2.4)
    cta_gemm<T>(k, r, k, T(-1), Ass, ld, false, Tm, k, false, Asr, ld);
    // B_rr = A_rr - T^T B_sr - A_rs T  (= A_rr - T^T A_sr - A_rs T + T^T A_ss T)
    cta_gemm<T>(r, r, k, T(-1), Tm, k, true, Asr, ld, false, Arr, ld);
    cta_gemm<T>(r, r, k, T(-1), Ars, ld, false, Tm, k, false, Arr, ld);
    if (ed.ldl) {
        // symmetric A (Sec. 5): P B_rr P^T = L D L^T, B_rs = B_sr^T
        const int res = cta_ldl_diag<T>(r, Arr, ld, piv, Asr, ld, k, redv, redi, (T)args.ldl_alpha);
        if (res != 0) {
            if (threadIdx.x == 0) atomicOr(args.status, res == 2 ? (int)DEV_SINGULAR : (int)DEV_LDL_FALLBACK);
            if (threadIdx.x == 0 && res == 1) args.ldl_fail[bi] = 1;
            return;
        }
        // X' = B_sr P^T L^{-T}, then X = X' D^{-1}
        cta_trsm_right_unit_lower_t<T>(r, Arr, ld, Asr, ld, k);
        T* pool = static_cast<T*>(args.fac_pool);
        T* Dv = pool + ed.D_out;
        for (int i = threadIdx.x; i < r; i += blockDim.x) Dv[i] = Arr[i + ld * i];
        __syncthreads();
        for (int e = threadIdx.x; e < k * r; e += blockDim.x) {
            const int i = e % k, j = e / k;
            Asr[i + ld * j] /= Dv[j];
        }
        __syncthreads();
        // Schur update -X D X^T on the skeletons (new SCI block, symmetric)
        if (k > 0 && ed.sci_out >= 0) {
            T* S = static_cast<T*>(args.sci_pool) + ed.sci_out;
            for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
                const int a = e % k, c = e / k;
                T acc = T(0);
                for (int l = 0; l < r; ++l) acc += Asr[a + ld * l] * Dv[l] * Asr[c + ld * l];
                S[e] = -acc;
            }
        }
        T* LL = pool + ed.LU_out;
        T* Xo = pool + ed.X_out;
        T* To = pool + ed.T_out;
        for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
            const int i = e % r, j = e / r;
            LL[e] = i > j ? Arr[i + ld * j] : T(0);
        }
        for (int e = threadIdx.x; e < k * r; e += blockDim.x) {
            const int i = e % k, j = e / k;
            Xo[e] = Asr[i + ld * j];
            To[e] = Tm[e];
        }
        __syncthreads();
        cta_unit_lower_inverse_to_upper<T>(r, LL);
        if (threadIdx.x == 0) {
            int* pm = args.perm_pool + ed.piv_out;
            for (int i = 0; i < r; ++i) pm[i] = i;
            for (int j = 0; j < r; ++j) {
                const int p = piv[j];
                const int t = pm[j]; pm[j] = pm[p]; pm[p] = t;
            }
        }
        return;
    }
    // B_rs = A_rs - T^T A_ss
    cta_gemm<T>(r, k, k, T(-1), Tm, k, true, Ass, ld, false, Ars, ld);
    // P B_rr = L (D U)                (Lemma 2.1)
    const bool ok = cta_lu<T>(r, Arr, ld, piv, redv, redi);
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(args.status, (int)DEV_SINGULAR);
        return;
    }
    // X = B_sr (DU)^{-1}
    cta_trsm_right_upper<T>(r, Arr, ld, Asr, ld, k);
    // Z = L^{-1} P B_rs
    cta_apply_piv<T>(r, piv, Ars, ld, k);
    cta_trsm_lower_unit<T>(r, Arr, ld, Ars, ld, k);
    // Schur update -X Z on the skeletons (new SCI block)
    if (k > 0 && ed.sci_out >= 0) {
        T* S = static_cast<T*>(args.sci_pool) + ed.sci_out;
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) S[e] = T(0);
        __syncthreads();
        cta_gemm<T>(k, k, r, T(-1), Asr, ld, false, Ars, ld, false, S, k);
    }
    // outputs: D, U = (DU)/D, Y = D^{-1} Z, T, X, LU, inverses of L and U
    T* pool = static_cast<T*>(args.fac_pool);
    T* Dv = pool + ed.D_out;
    for (int i = threadIdx.x; i < r; i += blockDim.x) Dv[i] = Arr[i + ld * i];
    __syncthreads();
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int i = e % r, j = e / r;
        if (i < j) Arr[i + ld * j] /= Dv[i];
    }
    for (int e = threadIdx.x; e < r * k; e += blockDim.x) {
        const int i = e % r, j = e / r;
        Ars[i + ld * j] /= Dv[i];
    }
    __syncthreads();
    T* LUo = pool + ed.LU_out;
    T* Xo = pool + ed.X_out;
    T* Yo = pool + ed.Y_out;
    T* To = pool + ed.T_out;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int i = e % r, j = e / r;
        LUo[e] = i == j ? T(0) : Arr[i + ld * j];
    }
    for (int e = threadIdx.x; e < k * r; e += blockDim.x) {
        const int i = e % k, j = e / k;
        Xo[e] = Asr[i + ld * j];
        To[e] = Tm[e];
    }
    for (int e = threadIdx.x; e < r * k; e += blockDim.x) {
        const int i = e % r, j = e / r;
        Yo[e] = Ars[i + ld * j];
    }
    __syncthreads();
    cta_unit_tri_inverses<T>(r, LUo, r, pool + ed.LUi_out, r);
    // convert LAPACK-style interchanges into the permutation perm with
    // (P x)_i = x[perm[i]]
    if (threadIdx.x == 0) {
        int* pm = args.perm_pool + ed.piv_out;
        for (int i = 0; i < r; ++i) pm[i] = i;
        for (int j = 0; j < r; ++j) {
            const int p = piv[j];
            const int t = pm[j]; pm[j] = pm[p]; pm[p] = t;
        }
    }
}

// Persistent elimination: the CTAs take boxes from the list (largest first)
// through an atomic counter until it runs out.
template <typename T>
__global__ void __launch_bounds__(128) elim_kernel(ElimArgs args) {
    __shared__ int item;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(args.next_item, 1);
        __syncthreads();
        const int q = item;
        if (q >= args.nitems) return;
        elim_box<T>(args, args.order[q]);
    }
}

// Batched ID on caller matrices: one CTA per matrix, matrix copied into a
// global workspace and reduced there.
__global__ void __launch_bounds__(128) id_batched_kernel(const double* mats, const int64_t* off, const int* m,
                                                          const int* n, const double* tol, int* k, int* perm,
                                                          const int64_t* poff, double* T, const int64_t* toff,
                                                          double* ws, const int64_t* wsoff) {
    const int b = blockIdx.x;
    const int mm = m[b], nn = n[b];
    const int ldw = mm | 1;
    double* W = ws + wsoff[b];
    const double* M = mats + off[b];
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* sp = smem;
    double* nrm = align_ptr<double>(sp, nn);
    int* pm = align_ptr<int>(sp, nn);
    int* rk = align_ptr<int>(sp, nn);
    double* redv = align_ptr<double>(sp, blockDim.x);
    int* redi = align_ptr<int>(sp, blockDim.x);
    double* hh = align_ptr<double>(sp, 4);
    for (int e = threadIdx.x; e < mm * nn; e += blockDim.x) W[(e % mm) + (int64_t)ldw * (e / mm)] = M[e];
    __syncthreads();
    cpqr_id<double>(W, 1, ldw, mm, nn, tol[b], nrm, pm, rk, redv, redi, redi + 64, hh, T + toff[b], perm + poff[b],
                    k + b);
}

cudaError_t launch_id_batched(int count, const double* mats, const int64_t* off, const int* m, const int* n,
                              const double* tol, int* k, int* perm, const int64_t* poff, double* T,
                              const int64_t* toff, cudaStream_t st) {
    // workspace offsets need the sizes on the host
    std::vector<int> hm(count), hn(count);
    cudaError_t e = cudaMemcpyAsync(hm.data(), m, sizeof(int) * count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hn.data(), n, sizeof(int) * count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    std::vector<int64_t> wso(count);
    int64_t tot = 0;
    int maxn = 1;
    for (int i = 0; i < count; ++i) {
        wso[i] = tot;
        tot += (int64_t)(hm[i] | 1) * hn[i];
        maxn = std::max(maxn, hn[i]);
    }
    double* ws = nullptr;
    int64_t* dwso = nullptr;
    e = cudaMalloc(&ws, sizeof(double) * std::max<int64_t>(tot, 1));
    if (e == cudaSuccess) e = cudaMalloc(&dwso, sizeof(int64_t) * count);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dwso, wso.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, st);
    const size_t smem = (size_t)maxn * 16 + 128 * 12 + 256;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(id_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        note_launch();
        id_batched_kernel<<<count, 128, smem, st>>>(mats, off, m, n, tol, k, perm, poff, T, toff, ws, dwso);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (ws) cudaFree(ws);
    if (dwso) cudaFree(dwso);
    return e;
}

// ---------------------------------------------------------- launchers ----

// Fold configurations: rows per chunk (RC) and columns per thread (CPT);
// RC * CPT registers of the element type hold a thread's share of the chunk.
int fold_cpt(int n, int elem) {
    if (n <= 256) return elem == 8 && n > 128 ? 2 : 1;
    if (n <= 512) return elem == 8 ? 4 : 2;
    if (n <= 1024) return elem == 8 ? 0 : 4;
    return 0;                                         // too wide: the materialized path
}
static int fold_rc(int cpt, int elem) {
    if (elem == 4) return cpt == 1 ? 32 : cpt == 2 ? 32 : 16;
    return cpt == 1 ? 32 : cpt == 2 ? 16 : 8;
}

size_t fold_smem_bytes(int n, int cpt, bool sci, bool R_in_smem, int elem) {
    const size_t rc = fold_rc(cpt, elem);       // the largest rows per chunk of the configuration
    size_t b = 0;
    b += rc * (5 * (size_t)elem + 8) + 80;             // row data
    b += 2 * rc * elem + 2 * (size_t)elem + 32;        // reflector buffers
    b += rc * (size_t)n * elem * (sci ? 2 : 1) + 32;   // the chunk (K and S parts apart for the Grams)
    if (R_in_smem) b += (size_t)n * (n + 1) / 2 * elem + 16;   // packed upper triangle
    return b + 128;
}

size_t id_smem_bytes(int ng, int mrow, bool W_in_smem, int elem) {
    size_t b = (size_t)ng * 16 + 128 * 8 + 72 * 4 + 2 * (size_t)ng * elem + 4 * elem + 160;
    if (W_in_smem) b += (size_t)mrow * ng * elem + 16;
    return b + 64;
}

template <typename T, int RC, int CPT>
static cudaError_t launch_fold_cfg(const FoldArgs& a, int nbox, int threads, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(fold_kernel<T, RC, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    fold_kernel<T, RC, CPT><<<nbox, threads, smem, st>>>(a);
    return cudaGetLastError();
}

// threads: the launch's largest box width rounded up to a warp (<= 256) for
// one column per thread, else 256; cpt from fold_cpt of the widest box
template <typename T>
cudaError_t launch_fold(const FoldArgs& a, int nbox, int threads, int cpt, size_t smem, cudaStream_t st, int rc) {
    if (nbox == 0) return cudaSuccess;
    if (threads < 32 || threads > 256 || threads % 32) return cudaErrorInvalidValue;
    if (cpt == 1 && rc == 16) return launch_fold_cfg<T, 16, 1>(a, nbox, threads, smem, st);
    if constexpr (sizeof(T) == 4) {
        if (cpt == 1) return launch_fold_cfg<T, 32, 1>(a, nbox, threads, smem, st);
        if (cpt == 2) return launch_fold_cfg<T, 32, 2>(a, nbox, threads, smem, st);
        if (cpt == 4) return launch_fold_cfg<T, 16, 4>(a, nbox, threads, smem, st);
    } else {
        if (cpt == 1) return launch_fold_cfg<T, 32, 1>(a, nbox, threads, smem, st);
        if (cpt == 2) return launch_fold_cfg<T, 16, 2>(a, nbox, threads, smem, st);
        if (cpt == 4) return launch_fold_cfg<T, 8, 4>(a, nbox, threads, smem, st);
    }
    return cudaErrorInvalidValue;
}

// One persistent launch over the sublevel's groups: as many CTAs as fit on
// the GPU at once (at most one per group).
template <typename T>
cudaError_t launch_id(const IdArgs& a, int ngroups, size_t smem, int num_sms, cudaStream_t st) {
    if (ngroups == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(id_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, id_kernel<T>, 128, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(ngroups, std::max(per_sm, 1) * std::max(num_sms, 1)));
    e = cudaMemsetAsync(a.next_item, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    note_launch();
    id_kernel<T><<<grid, 128, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_elim(const ElimArgs& a, int nbox, int num_sms, cudaStream_t st) {
    if (nbox == 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, elim_kernel<T>, 128, 0);
    if (e != cudaSuccess) return e;
    const int grid = std::min(nbox, std::max(1, per_sm) * std::max(1, num_sms));
    e = cudaMemsetAsync(a.next_item, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    note_launch();
    elim_kernel<T><<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram_tol(const GramTolArgs& a, int ngroups, int max_ng, cudaStream_t st) {
    if (ngroups == 0) return cudaSuccess;
    const size_t smem = 128 * sizeof(double) + 2 * (size_t)max_ng * sizeof(T) + 64;
    cudaError_t e = cudaFuncSetAttribute(gram_tol_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    gram_tol_kernel<T><<<ngroups, 128, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_r_colmajor(const void* R, int n, void* out, cudaStream_t st) {
    const int64_t tot = (int64_t)n * n;
    if (tot == 0) return cudaSuccess;
    note_launch();
    r_colmajor_kernel<T><<<(unsigned)std::min<int64_t>((tot + 255) / 256, 2048), 256, 0, st>>>(
        static_cast<const T*>(R), n, static_cast<T*>(out));
    return cudaGetLastError();
}

template cudaError_t launch_gram_tol<double>(const GramTolArgs&, int, int, cudaStream_t);
template cudaError_t launch_gram_tol<float>(const GramTolArgs&, int, int, cudaStream_t);
template cudaError_t launch_r_colmajor<double>(const void*, int, void*, cudaStream_t);
template cudaError_t launch_r_colmajor<float>(const void*, int, void*, cudaStream_t);
template cudaError_t launch_fold<double>(const FoldArgs&, int, int, int, size_t, cudaStream_t, int);
template cudaError_t launch_fold<float>(const FoldArgs&, int, int, int, size_t, cudaStream_t, int);
template cudaError_t launch_id<double>(const IdArgs&, int, size_t, int, cudaStream_t);
template cudaError_t launch_id<float>(const IdArgs&, int, size_t, int, cudaStream_t);
template cudaError_t launch_elim<double>(const ElimArgs&, int, int, cudaStream_t);
template cudaError_t launch_elim<float>(const ElimArgs&, int, int, cudaStream_t);

}  // namespace hif

// ------------------------------------------- batched ID without allocation --
//
// For callers that may not allocate device memory: services that size their
// device memory once at start-up and must not fail on an allocation later,
// and callers that must not call cudaMalloc/cudaFree at all because those
// calls can synchronize the whole device and stall work on other streams.
// The work space of the batched ID lives in one file-scope device array,
// sized once for the whole process.  Its layout: per-matrix work-space
// offsets, an error flag, then the copies of the matrices that the QR
// overwrites.  The flag is rewritten by every call's first kernel.

namespace hif {

constexpr int kNoAllocMaxMats = 4096;
constexpr int kNoAllocMaxCols = 1024;
constexpr int64_t kNoAllocWsDoubles = (int64_t)1 << 20;   // 8 MiB of matrix copies
constexpr size_t kNoAllocOffBytes = sizeof(int64_t) * kNoAllocMaxMats;
constexpr size_t kNoAllocFlagBytes = 256;
constexpr size_t kNoAllocBytes = kNoAllocOffBytes + kNoAllocFlagBytes + sizeof(double) * kNoAllocWsDoubles;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__global__ void id_noalloc_prep_kernel(unsigned char* scratch, int count, const int* m, const int* n) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t* off = reinterpret_cast<int64_t*>(scratch);
    int* flag = reinterpret_cast<int*>(scratch + kNoAllocOffBytes);
    int64_t run = 0;
    int bad = 0;
    for (int i = 0; i < count; ++i) {
        const int mi = m[i], ni = n[i];
        if (mi < 0 || ni < 0 || ni > kNoAllocMaxCols) { bad = 1; break; }
        off[i] = run;
        run += (int64_t)(mi | 1) * ni;
        if (run > kNoAllocWsDoubles) { bad = 1; break; }
    }
    *flag = bad;
}

__global__ void __launch_bounds__(128) id_noalloc_kernel(unsigned char* scratch, const double* mats,
                                                          const int64_t* off, const int* m, const int* n,
                                                          const double* tol, int* k, int* perm, const int64_t* poff,
                                                          double* T, const int64_t* toff) {
    const int* flag = reinterpret_cast<const int*>(scratch + kNoAllocOffBytes);
    if (*flag) return;
    const int b = blockIdx.x;
    const int mm = m[b], nn = n[b];
    const int ldw = mm | 1;
    double* ws = reinterpret_cast<double*>(scratch + kNoAllocOffBytes + kNoAllocFlagBytes);
    double* W = ws + reinterpret_cast<const int64_t*>(scratch)[b];
    const double* M = mats + off[b];
    __shared__ double nrm[kNoAllocMaxCols];
    __shared__ int pm[kNoAllocMaxCols];
    __shared__ int rk[kNoAllocMaxCols];
    __shared__ double redv[128];
    __shared__ int redi[128];
    __shared__ double hh[4];
    for (int e = threadIdx.x; e < mm * nn; e += blockDim.x) W[(e % mm) + (int64_t)ldw * (e / mm)] = M[e];
    __syncthreads();
    cpqr_id<double>(W, 1, ldw, mm, nn, tol[b], nrm, pm, rk, redv, redi, redi + 64, hh, T + toff[b], perm + poff[b],
                    k + b);
}

// Device address of the scratch array for the current device, looked up once
// per device (the symbol's host-side name is not a device address).
static unsigned char* noalloc_scratch_ptr(cudaError_t* err) {
    static std::mutex mu;
    static unsigned char* cache[128] = {};
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= 128) { *err = cudaErrorInvalidDevice; return nullptr; }
    std::lock_guard<std::mutex> lock(mu);
    if (!cache[dev]) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        cache[dev] = static_cast<unsigned char*>(p);
    }
    return cache[dev];
}

// Returns cudaSuccess and *too_big = 0 on success; *too_big = 1 when a matrix
// has more than kNoAllocMaxCols columns or the copies exceed the scratch.
cudaError_t launch_id_batched_noalloc(int count, const double* mats, const int64_t* off, const int* m, const int* n,
                                      const double* tol, int* k, int* perm, const int64_t* poff, double* T,
                                      const int64_t* toff, cudaStream_t st, int* too_big) {
    *too_big = 0;
    if (count > kNoAllocMaxMats) { *too_big = 1; return cudaSuccess; }
    cudaError_t e = cudaSuccess;
    unsigned char* scratch = noalloc_scratch_ptr(&e);
    if (!scratch) return e;
    note_launch();
    id_noalloc_prep_kernel<<<1, 1, 0, st>>>(scratch, count, m, n);
    note_launch();
    id_noalloc_kernel<<<count, 128, 0, st>>>(scratch, mats, off, m, n, tol, k, perm, poff, T, toff);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int flag = 0;
    e = cudaMemcpyAsync(&flag, scratch + kNoAllocOffBytes, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *too_big = flag;
    return cudaSuccess;
}

}  // namespace hif
