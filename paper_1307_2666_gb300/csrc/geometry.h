// Host-side integer bookkeeping of one skeletonization sublevel: the index
// sets C_l (cells by floor index, edges/faces by nearest interior centre --
// Sec. 4.1 / 4.2), their near fields (Sec. 3.3 proxy interior plus the
// SCI-coupled DOFs of Sec. 4.3) and the column groups of Sec. 4.4.
#pragma once

#include <cstdint>
#include <vector>

namespace hif {

enum BoxKind { KIND_CELL = 0, KIND_FACE = 1, KIND_EDGE = 2 };

struct Tree {
    int dim;
    double lo[3];
    double W;
    int L;
};

// Past SCI blocks: DOF i belongs to block blk[s][i] (or -1) at loc[s][i].
struct SciHost {
    std::vector<std::vector<int>> blk;      // per past sublevel, size N
    std::vector<std::vector<int>> loc;
    std::vector<std::vector<int>> members;  // per block id: skeleton DOFs in order
};

struct SublevelPlan {
    int nbox;
    std::vector<int64_t> box_off;           // members CSR
    std::vector<int> members;               // ascending within a box
    std::vector<double> centers;            // nbox x 3
    // filled by build_near_groups
    std::vector<int64_t> near_off;
    std::vector<int> near;
    std::vector<int> cols;                  // group-ordered columns (CSR = box_off)
    std::vector<int64_t> grp_off;           // per box: first group
    std::vector<int> grp_col0, grp_n, grp_sci;
    std::vector<int> box_sci;
};

void root_box(const double* x, const double* w, int64_t N, int dim, double lo[3], double* W);
int num_levels(const double* x, int64_t N, int dim, const double lo[3], double W, int occupancy);
void plan_sublevels(int dim, int L, bool fractional, int skip_levels, std::vector<int>& kinds,
                    std::vector<int>& levels);

// Partition the active DOFs (ascending ids) into the boxes of (kind, s).
void partition(const Tree& t, const double* x, int kind, int s, const std::vector<int>& active_ids,
               SublevelPlan& out, std::vector<int>& box_of);

// Per-thread mark arrays (epoch stamps over all DOFs) kept by the caller from
// one sublevel to the next, so that build_near_groups does not allocate and
// clear N entries per thread per sublevel.
struct NearCache {
    std::vector<std::vector<uint32_t>> mark;
    std::vector<uint32_t> epoch;
};

// Near fields and groups; `active` flags DOFs active at the start of the
// sublevel.  `cache` (may be null) keeps the mark arrays between calls; it is
// used by one call at a time.
void build_near_groups(const Tree& t, const double* x, int s, double proxy_radius, int second_kind,
                       const std::vector<int>& active_ids, const std::vector<char>& active,
                       const std::vector<int>& box_of, const SciHost& sci, SublevelPlan& p,
                       NearCache* cache = nullptr);

// Whether the N points (row-major, dim d) with weights Wt fill a full uniform
// n^d grid of spacing h with cell volumes h^d (in any order); if so sets n, h
// and dof_of[grid position] = off + point index (grid position: the first
// coordinate slowest), the layout of the grid convolution (Sec. 3.1: K_ij
// depends only on the offset).
bool grid_layout(const double* X, const double* Wt, int64_t N, int d, int64_t off, int* n_out, double* h_out,
                 std::vector<int>& dof_of);

// Appends the plan q of the next problem of a batched handle to the combined
// plan p (boxes, members, near fields and groups concatenated, offsets
// shifted); the first problem's plan is moved in.
void append_plan(SublevelPlan& p, SublevelPlan&& q);

// Spread S = max|T| sqrt(#T) / |T|_2 of the uniform-grid table T(o) =
// G(h |o|) (o != 0; kernel 0: -log(r)/(2 pi), kernel 1: 1/(4 pi r)), T(0) =
// k0, over the offsets o in [0, n)^dim: the scale of the short tensor-core
// sums' relative error (the refinement's error estimate).
double table_spread(int n, int dim, double h, int kernel_id, double k0);

// Trace of build_near_groups: returns the per-phase times summed since the
// previous call into ms[6] (bins, gather: wall ms; proxy scan, SCI patterns,
// near list, groups: thread ms) and sets the collection on or off.
void geometry_trace(bool on, double* ms);

}  // namespace hif
