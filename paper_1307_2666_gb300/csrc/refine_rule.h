// Which digit set of the tensor-core direct sum each residual of the
// iterative refinement takes (Sec. 5 refinement; the short sums are the
// tensor-core sum with digit classes 0..KD-1, KD = 4, 5, 6; 8 is the full
// sum).  Host-only arithmetic on residual norms.
#pragma once

namespace hif {

// C_KD (KD = 4, 5, 6): the bound on a short sum's relative error per unit of
// the grid table's spread S (table_spread).
extern const double kShortErr[3];

// Digit classes for residual k.  hist[0..k-1]: the relative residuals found
// so far; SY: S times |b K c u| / |f| from the last residual; fp32_factor:
// the factorization was FP32.
int short_residual_classes(int k, bool fp32_factor, const double* hist, double SY, double tol);

// Whether a residual computed with `classes` (< 8) that came out at relative
// size `worst` may drive the correction; otherwise it is recomputed in full.
bool short_residual_usable(int classes, double worst, double SY, double tol, bool last_step);

}  // namespace hif
