// Short digit sets for the residuals of the refinement.  A residual computed
// with an error d enters the next one in full (r' = (I - A F^{-1}) r - d), so
// only the residual that decides convergence has to be the full sum; another
// may take KD < 8 digit classes while its error stays below both 0.05 tol and
// 1e-4 of the residual itself (an FP32 factor reduces the residual by at most
// ~10^3 per step, so the next residual stays >= 10x above that error).  The
// error of a short sum is estimated as C_KD S Y.  The dropped digits sit at a
// fixed level below max|T| whatever the entry, so the relative error of
// y = K v grows with the table's spread S = max|T| sqrt(#T) / |T|_2; C_KD
// bounds the ratio of the two measured for Gaussian sources (exact integer
// convolutions of the digits, self term included: 2D log kernel n = 64..1024,
// S = 8..13, ratios up to 3.2e-9, 1.4e-11, 6.2e-14; 3D 1/r kernel n = 16..64,
// S = 23..104, up to 1.9e-9, 8.6e-12, 3.8e-14; the spread of the ratios comes
// from where max|T| and max|v| fall against their power-of-two scales), and
// Y = |b K c u| / |f|, the size of the kernel part of A u, is measured after
// every residual.
#include "refine_rule.h"

#include <algorithm>
#include <cmath>

namespace hif {

const double kShortErr[3] = {4e-9, 1.6e-11, 7e-14};      // C_KD, KD = 4, 5, 6

// Step 0 has no Y yet and takes 5 classes after an FP32 factorization (its
// first residual is of the order of the 2^-17 tolerance floor or above), 6
// after an FP64 one; step k >= 1 takes the fewest classes whose estimated
// error C_KD S Y meets the bound above for its predicted residual, the last
// one times the last contraction (sqrt of the first residual for the first
// contraction), if that prediction is above 10 tol, and the full sum
// otherwise.
int short_residual_classes(int k, bool fp32_factor, const double* hist, double SY, double tol) {
    if (k == 0) return fp32_factor ? 5 : 6;
    const double last = hist[k - 1];
    const double rho = k == 1 ? std::sqrt(hist[0]) : (hist[k - 2] > 0 ? last / hist[k - 2] : 0.0);
    const double pred = last * rho;
    if (!(pred > 10.0 * tol)) return 8;
    for (int kd = 4; kd <= 6; ++kd)
        if (kShortErr[kd - 4] * SY <= std::max(0.05 * tol, 1e-4 * pred)) return kd;
    return 8;
}

bool short_residual_usable(int classes, double worst, double SY, double tol, bool last_step) {
    if (classes < 4 || classes > 6) return false;
    return worst > tol && !last_step && kShortErr[classes - 4] * SY <= std::max(0.05 * tol, 1e-4 * worst);
}

}  // namespace hif
