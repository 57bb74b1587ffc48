// Replays the oracle's skeletonization decisions through the library's host
// planner (csrc/geometry.cpp) and prints every sublevel's plan, so that a CPU
// test can compare it with the oracle's index sets box by box: the tree
// (root box, depth), the sublevel sequence, and per box its DOFs, its near
// field (proxy interior plus SCI-coupled DOFs, Sec. 3.3 / 4.3) and its column
// groups (Sec. 4.4).  Test infrastructure; built by tests/test_plan_replay.py.
//
// stdin:  N dim occupancy proxy_radius second_kind, then N*dim coordinates and
//         N weights, then the number of sublevels and, per sublevel, its box
//         count and per box (in centre order) "nsk sk... nrd rd..." -- the
//         oracle's skeletons (in pivot order) and redundant DOFs.
// stdout: "TREE lo0 lo1 lo2 W L", "PLAN kind level ...", then per sublevel
//         "SUB kind level nbox" and per box "BOX", "MEM n ...", "NEAR n ...",
//         "GROUPS ng", and per group "G n sci cols...".
#include <cstdio>
#include <vector>

#include "../paper_1307_2666_gb300/csrc/geometry.h"

int main() {
    long long N;
    int dim, occ, second_kind;
    double radius;
    if (std::scanf("%lld %d %d %lf %d", &N, &dim, &occ, &radius, &second_kind) != 5) return 2;
    std::vector<double> x((size_t)N * dim), w((size_t)N);
    for (auto& v : x)
        if (std::scanf("%lf", &v) != 1) return 2;
    for (auto& v : w)
        if (std::scanf("%lf", &v) != 1) return 2;
    hif::Tree t{dim, {0.0, 0.0, 0.0}, 0.0, 0};
    hif::root_box(x.data(), w.data(), N, dim, t.lo, &t.W);
    t.L = hif::num_levels(x.data(), N, dim, t.lo, t.W, occ);
    std::printf("TREE %.17g %.17g %.17g %.17g %d\n", t.lo[0], t.lo[1], t.lo[2], t.W, t.L);
    std::vector<int> kinds, levels;
    hif::plan_sublevels(dim, t.L, true, 0, kinds, levels);
    std::printf("PLAN");
    for (size_t q = 0; q < kinds.size(); ++q) std::printf(" %d %d", kinds[q], levels[q]);
    std::printf("\n");

    int nsub;
    if (std::scanf("%d", &nsub) != 1) return 2;
    std::vector<char> active((size_t)N, 1);
    std::vector<int> box_of((size_t)N, -1);
    hif::SciHost sci;
    hif::NearCache cache;
    for (int tau = 0; tau < nsub && tau < (int)kinds.size(); ++tau) {
        const int s = 1 << (t.L - levels[tau]);
        std::vector<int> ids;
        for (long long i = 0; i < N; ++i)
            if (active[i]) ids.push_back((int)i);
        for (int i : ids) box_of[i] = -1;
        hif::SublevelPlan p;
        hif::partition(t, x.data(), kinds[tau], s, ids, p, box_of);
        hif::build_near_groups(t, x.data(), s, radius, second_kind, ids, active, box_of, sci, p, &cache);
        std::printf("SUB %d %d %d\n", kinds[tau], levels[tau], p.nbox);
        for (int b = 0; b < p.nbox; ++b) {
            std::printf("BOX\nMEM %lld", (long long)(p.box_off[b + 1] - p.box_off[b]));
            for (long long e = p.box_off[b]; e < p.box_off[b + 1]; ++e) std::printf(" %d", p.members[e]);
            std::printf("\nNEAR %lld", (long long)(p.near_off[b + 1] - p.near_off[b]));
            for (long long e = p.near_off[b]; e < p.near_off[b + 1]; ++e) std::printf(" %d", p.near[e]);
            const long long g0 = p.grp_off[b], g1 = p.grp_off[b + 1];
            std::printf("\nGROUPS %lld\n", g1 - g0);
            for (long long g = g0; g < g1; ++g) {
                std::printf("G %d %d", p.grp_n[g], p.grp_sci[g]);
                const long long c0 = p.box_off[b] + p.grp_col0[g];
                for (long long e = c0; e < c0 + p.grp_n[g]; ++e) std::printf(" %d", p.cols[e]);
                std::printf("\n");
            }
        }
        // the oracle's decisions: redundant DOFs leave the active set; the
        // skeletons of a box that eliminated something form an SCI block
        int nb;
        if (std::scanf("%d", &nb) != 1) return 2;
        sci.blk.emplace_back((size_t)N, -1);
        sci.loc.emplace_back((size_t)N, 0);
        for (int b = 0; b < nb; ++b) {
            int nsk, nrd;
            if (std::scanf("%d", &nsk) != 1) return 2;
            std::vector<int> sk(nsk);
            for (auto& v : sk)
                if (std::scanf("%d", &v) != 1) return 2;
            if (std::scanf("%d", &nrd) != 1) return 2;
            std::vector<int> rd(nrd);
            for (auto& v : rd)
                if (std::scanf("%d", &v) != 1) return 2;
            for (int i : rd) active[i] = 0;
            if (nsk > 0 && nrd > 0) {
                const int id = (int)sci.members.size();
                for (int l = 0; l < nsk; ++l) {
                    sci.blk.back()[sk[l]] = id;
                    sci.loc.back()[sk[l]] = l;
                }
                sci.members.push_back(sk);
            }
        }
    }
    return 0;
}
