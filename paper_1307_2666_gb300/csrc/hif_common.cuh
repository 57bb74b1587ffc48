// Shared device/host definitions of the HIF-IE CUDA library (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hif_types.h"

namespace hif {

// ---------------------------------------------------------------- kernels --

__host__ __device__ inline double green_d(int kernel_id, double r2) {
    // G of Eq. (1.4) from the squared distance: -log(r)/(2 pi) = -log(r^2)/(4 pi)
    return kernel_id == 0 ? -log(r2) * (0.25 / kPi) : (0.25 / kPi) / sqrt(r2);
}

__device__ inline float green_f(int kernel_id, float r2) {
    return kernel_id == 0 ? -__logf(r2) * (float)(0.25 / kPi) : (float)(0.25 / kPi) * rsqrtf(r2);
}

// Helmholtz kernel (kernel 2, Sec. 5 Example 3): G(r) = (i/4) H_0^(1)(k r)
// = -Y_0(k r)/4 + i J_0(k r)/4, from the CUDA math library's Bessel functions.
__device__ inline void green_helmholtz(double k, double r2, double& gr, double& gi) {
    const double x = k * sqrt(r2);
    gr = -0.25 * y0(x);
    gi = 0.25 * j0(x);
}
__device__ inline void green_helmholtz(float k, float r2, float& gr, float& gi) {
    const float x = k * sqrtf(r2);
    gr = -0.25f * y0f(x);
    gi = 0.25f * j0f(x);
}

// Entry (a, b) of the real 2 x 2 embedding [[Re z, -Im z], [Im z, Re z]]
template <typename T>
__device__ inline T cblk(T zr, T zi, int a, int b) {
    return a == b ? zr : (a == 1 ? zi : -zi);
}

template <typename T> struct Green;
template <> struct Green<double> {
    __device__ static double eval(int kid, double r2) { return green_d(kid, r2); }
};
template <> struct Green<float> {
    __device__ static float eval(int kid, float r2) {
        return kid == 0 ? -logf(r2) * (float)(0.25 / kPi) : (float)(0.25 / kPi) * rsqrtf(r2);
    }
};

// SCI value S_ij of the current active matrix.
template <typename T>
__device__ inline T sci_value(const SciDev& s, int i, int j) {
    T v = T(0);
    for (int q = 0; q < s.nsub; ++q) {
        const int bi = s.blk[(int64_t)q * s.N + i];
        if (bi >= 0 && bi == s.blk[(int64_t)q * s.N + j]) {
            const int k = s.kb[bi];
            const T* p = static_cast<const T*>(s.ptr[bi]);
            v += p[s.loc[(int64_t)q * s.N + i] + (int64_t)k * s.loc[(int64_t)q * s.N + j]];
        }
    }
    return v;
}

template <typename T>
__device__ inline T entry(const GeomDev& g, const SciDev& s, int i, int j, double r0, double r1, double r2) {
    // A_ij of the active matrix: a_i delta_ij + b_i K_ij c_j + SCI_ij
    T v;
    if (g.kernel_id == 2) {
        // real embedding of the complex entry of points i/2, j/2 (components i&1, j&1)
        const int pi = i >> 1, pj = j >> 1, ca = i & 1, cb = j & 1;
        T zr, zi;
        if (pi == pj) {
            zr = (T)(g.b[i] * g.kself[i] * g.c[i]);
            zi = (T)(g.b[i] * g.kself_im[i] * g.c[i]);
            v = (i == j ? (T)g.a[i] : T(0)) + cblk<T>(zr, zi, ca, cb);
        } else {
            const T d0 = (T)(g.x[2 * (int64_t)i] - r0) - (T)(g.x[2 * (int64_t)j] - r0);
            const T d1 = (T)(g.x[2 * (int64_t)i + 1] - r1) - (T)(g.x[2 * (int64_t)j + 1] - r1);
            T gr, gi;
            green_helmholtz((T)g.wavenumber, d0 * d0 + d1 * d1, gr, gi);
            const T s0 = (T)g.b[i] * (T)(g.w[j] * g.c[j]);
            v = cblk<T>(s0 * gr, s0 * gi, ca, cb);
        }
        return v + sci_value<T>(s, i, j);
    }
    if (i == j) {
        v = (T)(g.a[i] + g.b[i] * g.kself[i] * g.c[i]);
    } else {
        const int d = g.dim;
        const T d0 = (T)(g.x[(int64_t)d * i] - r0) - (T)(g.x[(int64_t)d * j] - r0);
        const T d1 = (T)(g.x[(int64_t)d * i + 1] - r1) - (T)(g.x[(int64_t)d * j + 1] - r1);
        const T d2 = d == 3 ? (T)(g.x[(int64_t)d * i + 2] - r2) - (T)(g.x[(int64_t)d * j + 2] - r2) : T(0);
        const T gk = Green<T>::eval(g.kernel_id, d0 * d0 + d1 * d1 + d2 * d2);
        v = (T)g.b[i] * gk * (T)(g.w[j] * g.c[j]);
    }
    return v + sci_value<T>(s, i, j);
}

// Entries of one row pair of Y_c (Eq. (3.3)) in column j: row 2p holds the
// outgoing entry, row 2p+1 the incoming one (Lemma 3.3 with quadrature
// weights).  Coordinates are relative to the box centre.  rid >= 0: near-field
// DOF i (kernel part k1 = b_i G w_j c_j, k2 = b_j G w_i c_i, SCI parts s1 =
// S_ij, s2 = S_ji); rid == -1: proxy point (k1 = G w_j c_j, k2 = b_j G w_j).
// Kernel 2 (real embedding): rcomp and the column's component j & 1 pick the
// entries of the 2 x 2 blocks, k1 from the block of the outgoing entry,
// k2 from the transposed block of the incoming one.
template <typename T>
__device__ inline void y_pair(int kid, int rid, T rx0, T rx1, T rx2, T rb, T rwc, int j, T cx0, T cx1, T cx2,
                              T cwc, T cb, T cbw, bool scival, const SciDev& sci, T& k1, T& k2, T& s1, T& s2,
                              int rcomp = 0, T wavenumber = T(0)) {
    k1 = k2 = s1 = s2 = T(0);
    if (rid == -2) return;
    const T d0 = rx0 - cx0, d1 = rx1 - cx1, d2 = rx2 - cx2;
    if (kid == 2) {
        T gr, gi;
        green_helmholtz(wavenumber, d0 * d0 + d1 * d1, gr, gi);
        const int cc = j & 1;
        const T s_out = rid >= 0 ? rb * cwc : cwc;        // b_i w_j c_j (near) or w_j c_j (proxy)
        const T s_in = rid >= 0 ? cb * rwc : cbw;         // b_j w_i c_i (near) or b_j w_j (proxy)
        k1 = cblk<T>(s_out * gr, s_out * gi, rcomp, cc);
        k2 = cblk<T>(s_in * gr, s_in * gi, cc, rcomp);
    }
    const T gk = kid == 2 ? T(0) : Green<T>::eval(kid, d0 * d0 + d1 * d1 + d2 * d2);
    if (rid >= 0) {
        if (kid != 2) {
            k1 = rb * gk * cwc;
            k2 = cb * gk * rwc;
        }
        if (scival) {
            for (int s = 0; s < sci.nsub; ++s) {
                const int bi = sci.blk[(int64_t)s * sci.N + rid];
                if (bi >= 0 && bi == sci.blk[(int64_t)s * sci.N + j]) {
                    const int kb = sci.kb[bi];
                    const T* P = static_cast<const T*>(sci.ptr[bi]);
                    const int li = sci.loc[(int64_t)s * sci.N + rid];
                    const int lj = sci.loc[(int64_t)s * sci.N + j];
                    s1 += P[li + (int64_t)kb * lj];
                    s2 += P[lj + (int64_t)kb * li];
                }
            }
        }
    } else if (kid != 2) {
        k1 = gk * cwc;
        k2 = cbw * gk;
    }
}

__device__ inline double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace hif
