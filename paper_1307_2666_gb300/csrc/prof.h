// Per-kernel-family device timing for measurement (hif_kernel_profile).
//
// While enabled, every launch (or launch group) of the factorization, the
// sweeps and the direct sum is bracketed by a pair of CUDA events on the
// stream it is issued on, together with the algorithmic work the host knows
// for it (flops or bytes, counted from the actual sizes of the run).  When
// disabled a ProfRange is two branches and nothing else.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hif {

enum ProfKind {
    PROF_FOLD = 0,      // fold_kernel: proxy matrix + Householder fold into R
    PROF_ID,            // id_kernel: rho_g + pivoted QR of R[:, g] + T
    PROF_ELIM,          // elim_kernel: one CTA per box
    PROF_BIG_YGEN,      // big_ygen_kernel: proxy matrices of large boxes in HBM
    PROF_BIG_RHO,       // rho_g power iterations on large groups
    PROF_BIG_QR,        // big_step + big_update: one pivot step of all large groups
    PROF_BIG_T,         // T = R1^{-1} R2 of large groups
    PROF_BIG_ELIM,      // batched multi-CTA elimination of large boxes
    PROF_SWEEP,         // one full solve/apply sweep (all sublevels, both passes)
    PROF_DIRECT,        // direct sum (one launch per block of right-hand sides)
    PROF_DIRECT_SHORT,  // tensor-core direct sum with a short digit set (intermediate residuals)
    PROF_COUNT
};

bool prof_enabled();

// Adds work to a kind without a timed range (work known only after a launch).
void prof_add_work(int kind, double flops, double bytes);

class ProfRange {
public:
    ProfRange(int kind, cudaStream_t st, double flops, double bytes);
    ~ProfRange();
    ProfRange(const ProfRange&) = delete;
    ProfRange& operator=(const ProfRange&) = delete;

private:
    int kind_;
    cudaStream_t st_;
    cudaEvent_t e0_ = nullptr;
};

// Sums per kind since the previous collect: ranges, event milliseconds,
// flops, bytes.  Synchronizes on the recorded events and frees them.
cudaError_t prof_collect(int64_t* ranges, double* ms, double* flops, double* bytes);
void prof_set(bool enable);
const char* prof_name(int kind);

}  // namespace hif
