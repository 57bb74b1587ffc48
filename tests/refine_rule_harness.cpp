// Evaluates the refinement's digit-set rule (csrc/refine_rule.cpp) on query
// lines from stdin and prints one integer per query.  Test infrastructure;
// built by tests/test_short_sum_model.py.
//   "C k fp32 SY tol nh h0 h1 ..."   -> short_residual_classes
//   "U classes worst SY tol last"     -> short_residual_usable (0 or 1)
#include <cstdio>
#include <vector>

#include "../paper_1307_2666_gb300/csrc/refine_rule.h"

int main() {
    char op;
    while (std::scanf(" %c", &op) == 1) {
        if (op == 'C') {
            int k, fp32, nh;
            double SY, tol;
            if (std::scanf("%d %d %lf %lf %d", &k, &fp32, &SY, &tol, &nh) != 5) return 2;
            std::vector<double> h(nh > 0 ? nh : 1);
            for (int q = 0; q < nh; ++q)
                if (std::scanf("%lf", &h[q]) != 1) return 2;
            std::printf("%d\n", hif::short_residual_classes(k, fp32 != 0, h.data(), SY, tol));
        } else if (op == 'U') {
            int classes, last;
            double worst, SY, tol;
            if (std::scanf("%d %lf %lf %lf %d", &classes, &worst, &SY, &tol, &last) != 5) return 2;
            std::printf("%d\n", hif::short_residual_usable(classes, worst, SY, tol, last != 0) ? 1 : 0);
        } else {
            return 2;
        }
    }
    return 0;
}
