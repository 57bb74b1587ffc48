// Prints the library's grid-table spread (table_spread in csrc/geometry.cpp)
// for each "n dim k0" triple read from stdin: the kernel is the 2D log kernel
// for dim 2 and the 3D 1/r kernel for dim 3, with h = 1/n.  Test
// infrastructure; built by tests/test_short_sum_model.py.
#include <cstdio>

#include "../paper_1307_2666_gb300/csrc/geometry.h"

int main() {
    int n, dim;
    double k0;
    while (std::scanf("%d %d %lf", &n, &dim, &k0) == 3)
        std::printf("%.17g\n", hif::table_spread(n, dim, 1.0 / n, dim == 2 ? 0 : 1, k0));
    return 0;
}
