// Appends the sublevel plans read from stdin into one combined plan with the
// library's append_plan (the plan of a batched handle, one problem after the
// other) and prints it.  Test infrastructure; built by
// tests/test_plan_replay.py.
//   stdin:  nplans, then per plan: nbox, then per box "nm members... nn near...
//           ng (col0 n sci)..." followed by one box_sci flag and 3 centre coordinates
//   stdout: the combined plan's arrays, one per line, each "name count values..."
#include <cstdio>
#include <utility>
#include <vector>

#include "../paper_1307_2666_gb300/csrc/geometry.h"

template <class T>
static void put(const char* name, const std::vector<T>& v) {
    std::printf("%s %zu", name, v.size());
    for (const T& e : v) std::printf(" %.17g", (double)e);
    std::printf("\n");
}

int main() {
    int np;
    if (std::scanf("%d", &np) != 1) return 2;
    hif::SublevelPlan p;
    p.nbox = 0;
    p.box_off.assign(1, 0);
    p.near_off.assign(1, 0);
    p.grp_off.assign(1, 0);
    for (int k = 0; k < np; ++k) {
        hif::SublevelPlan q;
        if (std::scanf("%d", &q.nbox) != 1) return 2;
        q.box_off.assign(1, 0);
        q.near_off.assign(1, 0);
        q.grp_off.assign(1, 0);
        for (int b = 0; b < q.nbox; ++b) {
            int nm, nn, ng, v, sci;
            if (std::scanf("%d", &nm) != 1) return 2;
            for (int e = 0; e < nm; ++e) {
                if (std::scanf("%d", &v) != 1) return 2;
                q.members.push_back(v);
                q.cols.push_back(v);
            }
            if (std::scanf("%d", &nn) != 1) return 2;
            for (int e = 0; e < nn; ++e) {
                if (std::scanf("%d", &v) != 1) return 2;
                q.near.push_back(v);
            }
            if (std::scanf("%d", &ng) != 1) return 2;
            for (int e = 0; e < ng; ++e) {
                int c0, n, s;
                if (std::scanf("%d %d %d", &c0, &n, &s) != 3) return 2;
                q.grp_col0.push_back(c0);
                q.grp_n.push_back(n);
                q.grp_sci.push_back(s);
            }
            if (std::scanf("%d", &sci) != 1) return 2;
            q.box_sci.push_back(sci);
            for (int e = 0; e < 3; ++e) {
                double c;
                if (std::scanf("%lf", &c) != 1) return 2;
                q.centers.push_back(c);
            }
            q.box_off.push_back((int64_t)q.members.size());
            q.near_off.push_back((int64_t)q.near.size());
            q.grp_off.push_back((int64_t)q.grp_col0.size());
        }
        hif::append_plan(p, std::move(q));
    }
    std::printf("nbox %d\n", p.nbox);
    put("box_off", p.box_off);
    put("members", p.members);
    put("cols", p.cols);
    put("near_off", p.near_off);
    put("near", p.near);
    put("grp_off", p.grp_off);
    put("grp_col0", p.grp_col0);
    put("grp_n", p.grp_n);
    put("grp_sci", p.grp_sci);
    put("box_sci", p.box_sci);
    put("centers", p.centers);
    return 0;
}
