// Shared device/host definitions of the HIF-IE CUDA library (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hif_types.h"

namespace hif {

// ---------------------------------------------------------------- kernels --

__host__ __device__ inline double green_d(int kernel_id, double r2) {
    // G of Eq. (1.3) from the squared distance: -log(r)/(2 pi) = -log(r^2)/(4 pi)
    return kernel_id == 0 ? -log(r2) * (0.25 / kPi) : (0.25 / kPi) / sqrt(r2);
}

__device__ inline float green_f(int kernel_id, float r2) {
    return kernel_id == 0 ? -__logf(r2) * (float)(0.25 / kPi) : (float)(0.25 / kPi) * rsqrtf(r2);
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

__device__ inline double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace hif
