// Runs the library's uniform-grid detection (grid_layout in csrc/geometry.cpp)
// on the points read from stdin ("N d off", N*d coordinates, N weights) and
// prints "1 n h" and the DOF of every grid position, or "0".  Test
// infrastructure; built by tests/test_plan_replay.py.
#include <cstdio>
#include <vector>

#include "../paper_1307_2666_gb300/csrc/geometry.h"

int main() {
    long long N, off;
    int d;
    if (std::scanf("%lld %d %lld", &N, &d, &off) != 3) return 2;
    std::vector<double> x((size_t)N * d), w((size_t)N);
    for (auto& v : x)
        if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : w)
        if (std::scanf("%lf", &v) != 1) return 2;
    std::vector<int> dof_of;
    int n = 0;
    double h = 0.0;
    if (!hif::grid_layout(x.data(), w.data(), N, d, off, &n, &h, dof_of)) {
        std::printf("0\n");
        return 0;
    }
    std::printf("1 %d %.17g\n", n, h);
    for (int v : dof_of) std::printf("%d ", v);
    std::printf("\n");
    return 0;
}
