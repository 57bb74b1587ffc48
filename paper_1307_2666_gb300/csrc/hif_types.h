// Plain data shared by the host orchestration and the kernels (no device code).
#pragma once

#include <cstdint>

namespace hif {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxSub = 64;   // max skeletonization sublevels a factorization may run

// Problem geometry and coefficients on the device (Eq. (1.1), Eq. (3.1)).
struct GeomDev {
    const double* x;      // N x dim row-major
    const double* w;      // cell volumes (one-point quadrature weights)
    const double* a;
    const double* b;
    const double* c;
    const double* kself;  // self-cell integral K_ii (its real part for kernel 2)
    const double* kself_im; // kernel 2: imaginary part of K_ii
    double wavenumber;    // kernel 2: k
    int64_t N;
    int dim;
    int kernel_id;        // 0: -log(r)/(2 pi), 1: 1/(4 pi r), 2: (i/4) H_0^(1)(k r)
    int ncomp;            // real DOFs per point: 2 for kernel 2 (real 2 x 2 embedding), else 1
};

// Schur-complement interaction (SCI) history.  Every box that eliminated
// DOFs left a dense k x k update on its skeletons (Lemma 2.4, B_ss); DOF i
// belongs to at most one such block per sublevel s: blk[s*N+i] (or -1) at
// local position loc[s*N+i].  The SCI between i and j is the sum over past
// sublevels of the shared blocks' entries.
struct SciDev {
    const int* blk;
    const int* loc;
    void* const* ptr;     // per block: column-major k x k values (factor precision)
    const int* kb;        // per block: k
    int nsub;             // number of past sublevels to scan
    int64_t N;
};

// ID phase, one entry per box of the current sublevel.
struct BoxDesc {
    int n;                // |c| columns, ordered group by group
    int m_near;           // |c^N|
    int ngroups;
    int has_sci;          // any SCI touches the box (Grams for rho are needed)
    int sym;              // A symmetric: one row per near-field DOF / proxy point (Y'_c, Sec. 5)
    int pad0;
    int64_t col_off;      // into cols[]
    int64_t near_off;     // into near[]
    int64_t grp_off;      // first group index
    int64_t R_off;        // into the R scratch (n x n, row-major), same offset for the Grams
    double ctr[3];
    double radius;        // proxy radius (absolute)
};

struct GroupDesc {
    int box;
    int col0;             // first column of the group inside the box
    int n;                // columns in the group
    int has_sci;
    int64_t T_off;        // scratch for T_g (k x r, column-major), n*n reserved
    int64_t perm_off;     // n ints: skeletons (pivot order) then redundants (ascending)
};

// Elimination phase, one entry per box that eliminated something (r > 0).
struct ElimDesc {
    int k, r;
    int ngroups;
    int ldl;              // 1: P B_rr P^T = L D L^T (symmetric A, Sec. 5); 0: LU
    int64_t sk_off;       // into the sk ids array (global DOF ids, skeleton order)
    int64_t rd_off;       // into the rd ids array
    int64_t grp_off;      // into the per-group (k_g, r_g, T_off, ko, ro) table
    int64_t ws_off;       // workspace: (k+r)^2 + k*r scalars
    int64_t T_out, LU_out, LUi_out, D_out, X_out, Y_out;  // factor pool offsets
    int64_t piv_out;      // int pool offset (r)
    int64_t sci_out;      // SCI pool offset (k*k), -1 if no skeleton
};

struct ElimGroup {
    int kg, rg;
    int ko, ro;
    int64_t T_off;
};

// Factor record of one box, read by the sweeps (Eqs. (3.4), (4.1)).
struct BoxFac {
    int k, r;
    int ldl;              // LDL box: U = L^T P, Y = X^T; LU_off holds L (strict lower)
                          // and L^{-1} transposed (strict upper); LUi_off == LU_off
    int pad;
    int64_t sk_off, rd_off;                       // into the sublevel's id arrays
    int64_t T_off, LU_off, LUi_off, D_off, X_off, Y_off;
    int64_t piv_off;
};

// Status word written by kernels that detect trouble (checked by the host).
enum DevStatus : int {
    DEV_OK = 0, DEV_SINGULAR = 1, DEV_NONFINITE = 2, DEV_BADSIZE = 4, DEV_LDL_FALLBACK = 8, DEV_TIMEOUT = 16
};

// Counts kernel launches made by the library (diagnostic, see hif_kernel_launches).
void note_launch();

}  // namespace hif
