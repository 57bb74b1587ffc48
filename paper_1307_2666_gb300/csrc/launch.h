// Kernel argument blocks and host-side launchers (internal to the library).
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "hif_types.h"

namespace hif {

struct FoldArgs {
    GeomDev g;
    SciDev sci;
    const BoxDesc* boxes;
    const int* box_list;      // boxes handled by this launch (blockIdx.x -> box)
    const int* cols;
    const int* near;
    const GroupDesc* groups;
    const double* proxy;      // P x dim unit directions
    int P;
    int bpairs;
    int second_kind;
    int R_in_smem;
    void* Rws;
    void* GKws;
    void* GSws;
};

struct IdArgs {
    const GroupDesc* groups;
    const int* group_list;    // work items of this launch, largest first
    int nitems;               // entries of group_list
    int* next_item;           // work-queue counter (zero at launch)
    const BoxDesc* boxes;
    const void* Rws;
    const void* GKws;
    const void* GSws;
    void* Wws;
    const int64_t* W_off;
    int W_in_smem;
    int second_kind;
    void* Tws;
    int* perm_out;
    int* k_out;
    double eps;
    double tol_floor;
};

struct ElimArgs {
    GeomDev g;
    SciDev sci;
    const ElimDesc* boxes;
    const ElimGroup* groups;
    const int* sk_ids;
    const int* rd_ids;
    const void* Tws;
    void* ws;
    void* fac_pool;
    int* piv_pool;
    int* perm_pool;
    void* sci_pool;
    int* status;
    int* ldl_fail;          // per box of the launch: 1 when its LDL pivot failed the test
    double ldl_alpha;       // 1 x 1 pivot acceptance constant ((1 + sqrt 17) / 8)
    const int* order;       // work list: box indices, largest first
    int nitems;
    int* next_item;         // atomic counter of the persistent CTAs
};

struct SweepArgs {
    const BoxFac* boxes;
    const int* sk_ids;
    const int* rd_ids;
    const void* pool;
    const int* perm;
    void* x;                // working vectors, N x nrhs column-major (factor precision)
    int64_t ldx;
    int nrhs;
    int mode;               // see k_sweep.cu
    void* gws;              // non-null: per-box vectors in global memory at gws_off[box] * nrhs
    const int64_t* gws_off; // (boxes too large for shared memory); offsets per right-hand side
};

// ---- large boxes: unpivoted blocked QR to the n x n factor R (k_bigqr.cu)
struct BigQRArgs {
    void* Y;                // proxy matrices, column-major, ld = m, at y_off per box
    const int64_t* y_off;
    const int* m;
    const int* n;
    void* tau;              // per box 16 (the current panel's reflectors)
    void* G;                // per box 16 x 16 FP64 (Gram of the panel's reflectors)
    void* Tf;               // per box 16 x 16 (compact-WY factor)
    void* W;                // per box 16 x wld
    int64_t wld;            // >= the largest n
    double* Gp;             // partial Grams, per box at gp_off (see big_geqrf_partials)
    const int64_t* gp_off;
    double* Wp;             // partial V^T C, per box at wp_off
    const int64_t* wp_off;
};
// offsets of the partial-sum slots; returns the Gram slots' total (doubles)
size_t big_geqrf_partials(const int* m, const int* n, int nbox, std::vector<int64_t>& gp_off,
                          std::vector<int64_t>& wp_off, int64_t* wp_total);
template <typename T> cudaError_t big_geqrf(const BigQRArgs&, int nbox, int max_m, int max_n, cudaStream_t);

// ---- large boxes (k_large.cu)
struct BigBox {
    int box;                // index into the sublevel's BoxDesc array
    int m;                  // rows of Y_c
    int64_t y_off;          // Y_c (m x n, column-major) in the large-box workspace
};

struct BigGroup {
    int group;              // index into the sublevel's GroupDesc array
    int n;                  // columns
    int m;                  // rows (the box's m, or its n once the box is reduced to R)
    int ld;                 // leading dimension (the box's m)
    int need_rho;           // second-kind tolerance needed
    int64_t y_off;          // first column of the group in the workspace
    int64_t vec_off;        // prefix sum of n over groups
    int64_t row_off;        // prefix sum of m over groups
    double tol;             // relative ID tolerance (filled on the device)
};

struct BigState {
    int k;
    int stop;
    double nu0;
    double tau;
    // blocked pivoted QR (big_qp): first pivot of the current panel, panel
    // ended early (a norm lost too much to downdating), launch step of the
    // last pivot taken
    int j0;
    int pend;
    int last_step;
    int pad;
};

struct BigArgs {
    GeomDev g;
    SciDev sci;
    const BoxDesc* boxes;
    const BigBox* bigboxes;
    const int* cols;
    const int* near;
    const double* proxy;
    int P;
    int second_kind;
    void* YK;
    void* YS;
    BigGroup* groups;
    BigState* state;
    const GroupDesc* gdesc;
    double* vec_v;
    double* vec_w;
    double* vec_t;
    double* est;
    double* nrm;
    int* perm;
    void* Tws;
    int* perm_out;
    int* k_out;
    double eps;
    double tol_floor;
    // blocked pivoted QR: F (n x nb per group at vec_off * nb), the panel's
    // V^T v (32 per group), the norms at the last exact computation, panel width
    void* F;
    void* gv;
    double* nrm0;
    int nb;
};

template <typename T> cudaError_t big_ygen(const BigArgs&, int nbig, int64_t max_entries, cudaStream_t);
template <typename T> cudaError_t big_rho(const BigArgs&, int ngroups, int max_m, int max_n, cudaStream_t);
template <typename T> cudaError_t big_add(void* YK, const void* YS, int64_t n, cudaStream_t);
template <typename T> cudaError_t big_qr_init(const BigArgs&, int ngroups, int max_n, cudaStream_t);
template <typename T> cudaError_t big_qr_step(const BigArgs&, int ngroups, int max_n, int j, cudaStream_t);
// Blocked column-pivoted QR of all large groups: one panel of up to a.nb
// pivots per call, its trailing update one product; step counts the pivot
// launches (the state's last_step) across calls.
template <typename T> cudaError_t big_qp_panel(const BigArgs&, int ngroups, int max_n, int max_m, int& step, cudaStream_t);
template <typename T> cudaError_t big_finish(const BigArgs&, int ngroups, int max_n, cudaStream_t);
struct BatchElimArgs {
    GeomDev g;
    SciDev sci;
    const ElimDesc* ed;       // the large boxes
    int nbox;
    const ElimGroup* groups;
    const int* sk;
    const int* rd;
    const void* Tws;
    void* ws;
    void* pool;
    int* piv;
    int* perm;
    void* sci_pool;
    int* status;
    void* gemm_probs;         // FP32: 5 nbox TcGemmProb of work space for the tensor-core products
};
template <typename T> cudaError_t big_elim_batch(const BatchElimArgs&, int max_n, int max_k, int max_r, cudaStream_t);

size_t fold_smem_bytes(int n, int cpt, bool sci, bool R_in_smem, int elem);
size_t id_smem_bytes(int ng, int mrow, bool W_in_smem, int elem);

// tolerances of large groups from the box Grams (boxes folded into R)
struct GramTolArgs {
    BigGroup* groups;
    const GroupDesc* gdesc;
    const BoxDesc* boxes;
    const void* GKws;
    const void* GSws;
    double eps;
    double tol_floor;
};
template <typename T> cudaError_t launch_gram_tol(const GramTolArgs&, int ngroups, int max_ng, cudaStream_t);
template <typename T> cudaError_t launch_r_colmajor(const void* R, int n, void* out, cudaStream_t);

// columns per thread of the fold kernel for a box of n columns (0: too wide)
int fold_cpt(int n, int elem);
template <typename T>
cudaError_t launch_fold(const FoldArgs&, int nbox, int threads, int cpt, size_t smem, cudaStream_t, int rc = 0);
template <typename T> cudaError_t launch_id(const IdArgs&, int ngroups, size_t smem, int num_sms, cudaStream_t);
template <typename T> cudaError_t launch_elim(const ElimArgs&, int nbox, int num_sms, cudaStream_t);

// sweeps
// threads: CTA size, a multiple of 32 up to 512 (the sweep's arithmetic does
// not depend on it)
template <typename T> cudaError_t launch_sweep(const SweepArgs&, int nbox, int threads, cudaStream_t);

// Wide boxes of a sublevel: the pass as stage launches over (box, row tile).
// ws holds per box (k + 2 r) x nr values from ws_off[box] * nr; nr <= 16.
struct WideArgs {
    const BoxFac* boxes;
    const int* sk_ids;
    const int* rd_ids;
    const void* pool;
    const int* perm;
    void* x;
    int64_t ldx;
    int nr;
    void* ws;
    const int64_t* ws_off;
};
template <typename T>
cudaError_t launch_wide_sweep(const WideArgs&, int nwide, int max_k, int max_r, int mode, cudaStream_t);

// vectors and direct sums (FP64 inputs)
template <typename T> cudaError_t launch_to_work(const double* src, int64_t lds, T* dst, int64_t ldd,
                                                 int64_t N, int nrhs, cudaStream_t);
template <typename T> cudaError_t launch_from_work(const T* src, int64_t lds, double* dst, int64_t ldd,
                                                   int64_t N, int nrhs, cudaStream_t);

struct DirectArgs {
    GeomDev g;
    const double* x;        // N x nrhs
    int64_t ldx;
    double* y;
    int64_t ldy;
    int nrhs;
    int trans;
    int64_t seg_off;        // the problem's DOF range [seg_off, seg_off + seg_n)
    int64_t seg_n;
};
cudaError_t launch_direct_general(const DirectArgs&, cudaStream_t);
cudaError_t launch_direct_helmholtz(const DirectArgs&, cudaStream_t);

// Batched FP32 products on the tensor cores (k_tcgemm.cu):
// C = beta C + alpha op(A) op(B), column-major; op(A)[i, l] = tA ? A[l + lda i]
// : A[i + lda l], op(B)[l, j] = tB ? B[j + ldb l] : B[l + ldb j]; beta 0 or 1.
struct TcGemmProb {
    const float* A;
    const float* B;
    float* C;
    int64_t lda, ldb, ldc;
    int m, n, k;
    int tA, tB;
    float alpha;
    int beta;
};
// dprobs: device array of nprob problems; max_m / max_n bound their m / n.
// `flag` is ORed into *status when a bounded wait of the kernel runs out.
cudaError_t launch_tc_gemm(const TcGemmProb* dprobs, int nprob, int max_m, int max_n, int* status, int flag,
                           cudaStream_t st);
size_t tc_gemm_smem_bytes();

struct GridDirectArgs {     // uniform tensor grid: K depends on the index offset only
    const double* table;    // n^dim entries: G(h |delta|) for delta != 0, K_self / w at 0
    const int* dof_of;      // grid position -> DOF id
    int n;                  // points per side
    int dim;
    const double* a;
    const double* b;
    const double* c;
    const double* w;
    const double* x;
    int64_t ldx;
    double* y;
    int64_t ldy;
    int nrhs;
    int trans;
    double* vbuf;           // N x nrhs scratch (grid order)
    double* ybuf;           // N x nrhs scratch (grid order)
};
cudaError_t launch_direct_grid(const GridDirectArgs&, cudaStream_t);
// same sum in paired-FP32 arithmetic; tdf: the table split into (hi, lo)
// floats, vdf: N x nrhs float2 scratch
cudaError_t launch_direct_grid_df(const GridDirectArgs&, const float2* tdf, float2* vdf, cudaStream_t);
cudaError_t launch_split_df(const double* src, float2* dst, int64_t n, cudaStream_t);
// grid-order staging v = (source weight) x and the final y = a x + (target
// weight) ybuf, shared by the grid sums (eb blocks of 256 threads)
void grid_scatter_kernel_launch(const GridDirectArgs&, int64_t N, int eb, cudaStream_t);
void grid_finish_kernel_launch(const GridDirectArgs&, int64_t N, int eb, cudaStream_t);
// same sum on the tensor cores in exact 8-bit digits (k_tcconv.cu):
// R = mirrored table digit rows (tc_table_rows_bytes), built once per grid by
// launch_tc_table with tmax its max |entry|; XB = tc_source_digits_bytes of
// scratch, xmax 8 entries, status one int (set to 1 if a wait expired)
size_t tc_table_rows_bytes(int n, int dim);
size_t tc_source_digits_bytes(int n, int dim);
cudaError_t launch_tc_table(const double* table, int n, int dim, unsigned long long* tmax, void* R,
                            cudaStream_t);
// CUDA-event timing of tc_conv_kernel launches (see hif_kernel_timing)
void tc_timing_set(bool enable);
cudaError_t tc_timing_collect(double* ms, int64_t* launches);
// classes: digit classes kept (8: the full sum; 6, 5 or 4: the shorter sums
// of the refinement's intermediate residuals)
cudaError_t launch_direct_grid_tc(const GridDirectArgs&, const void* R, const unsigned long long* tmax,
                                  void* XB, unsigned long long* xmax, int* status, int num_sms, int classes,
                                  cudaStream_t);
cudaError_t launch_grid_table(double* table, int n, int dim, double h, int kernel_id, double kself_over_w,
                              cudaStream_t);

cudaError_t launch_kernel_block(const GeomDev& g, const int* rows, int64_t nr, const int* cols, int64_t nc,
                                double* out, int64_t ldo, cudaStream_t);
cudaError_t launch_kself(const GeomDev& g, double* kself, cudaStream_t);

// BLAS-1 helpers for the refinement loops (FP64)
cudaError_t launch_adjoint_coef(int64_t N, int nrhs, const double* a, const double* b, const double* c,
                                const double* u, const double* lam, const double* Fu, const double* Ftl, double* ga,
                                double* gb, double* gc, int* bad, cudaStream_t st);
cudaError_t launch_kpart(int64_t N, int nrhs, const double* f, const double* r, const double* a, const double* u,
                         double* out, cudaStream_t);
cudaError_t launch_axpby(int64_t N, int nrhs, double alpha, const double* x, int64_t ldx, double beta,
                         double* y, int64_t ldy, cudaStream_t);
cudaError_t launch_seg_dots(int nseg, const int64_t* off, const int64_t* cnt, int nrhs, const double* x, int64_t ldx,
                            const double* y, int64_t ldy, double* out, cudaStream_t);
cudaError_t launch_col_dots(int64_t N, int nrhs, const double* x, int64_t ldx, const double* y, int64_t ldy,
                            double* out, cudaStream_t);

// Batched ID with its work space in a file-scope device array (hif_id_batched_noalloc)
cudaError_t launch_id_batched_noalloc(int count, const double* mats, const int64_t* off, const int* m, const int* n,
                                      const double* tol, int* k, int* perm, const int64_t* poff, double* T,
                                      const int64_t* toff, cudaStream_t st, int* too_big);

// Batched ID on caller-provided matrices (hif_id_batched)
cudaError_t launch_id_batched(int count, const double* mats, const int64_t* off, const int* m, const int* n,
                              const double* tol, int* k, int* perm, const int64_t* poff, double* T,
                              const int64_t* toff, cudaStream_t);

}  // namespace hif
