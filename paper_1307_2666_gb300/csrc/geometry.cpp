// Host-side index bookkeeping of HIF-IE sublevels (see geometry.h).
//
// The arithmetic that decides memberships (cell floor indices, squared
// distances to edge/face centres and to the proxy centre) is written as plain
// IEEE double operations in a fixed order and compiled without FMA
// contraction, so that the same inputs always give the same index sets.  A
// DOF joins the nearest edge/face centre; centres whose squared distance is
// within a relative kTie of the nearest one count as tied, and the lowest
// centre id wins.  On a grid, tied centres are exactly equidistant, but the
// computed distances can differ in the last bits (three squares summed in
// different orders; a cube root for the root box's cell side that is not
// correctly rounded in every math library moves all centres by an ulp).
#include "geometry.h"
#include "hif_types.h"

#include <algorithm>
#include <cmath>
#include <memory>
#include <numeric>
#include <chrono>
#include <unordered_map>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace hif {

// relative distance difference within which two centres count as tied
constexpr double kTie = 0x1p-40;

// Stable counting sort of the indices 0..n-1 by key[a] in [0, nkeys): on
// return order[off[k] .. off[k+1]) lists the a with key k, ascending.  With
// several threads every thread counts and places one contiguous range of a,
// the ranges of one key following one another in order, so the result is the
// serial one.
// Work array whose entries are left uninitialized (every use writes them
// before reading): large per-sublevel buffers skip the serial zero fill.
template <class T>
struct RawBuf {
    std::unique_ptr<T[]> p;
    explicit RawBuf(size_t n) : p(new T[n > 0 ? n : 1]) {}
    T& operator[](size_t i) { return p[i]; }
    const T& operator[](size_t i) const { return p[i]; }
    T* data() { return p.get(); }
};

static void stable_bucket(const int64_t* key, int64_t n, int64_t nkeys, std::vector<int64_t>& off, int64_t* order) {
    off.assign(nkeys + 1, 0);
    int nch = 1;
#ifdef _OPENMP
    nch = omp_get_max_threads();
#endif
    if (n < 65536 || (int64_t)nch * nkeys > ((int64_t)1 << 22)) nch = 1;
    if (nch == 1) {
        for (int64_t a = 0; a < n; ++a) off[key[a] + 1]++;
        for (int64_t k = 0; k < nkeys; ++k) off[k + 1] += off[k];
        std::vector<int64_t> pos(off.begin(), off.end() - 1);
        for (int64_t a = 0; a < n; ++a) order[pos[key[a]]++] = a;
        return;
    }
    std::vector<int64_t> cnt((size_t)nch * nkeys, 0);
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nch; ++c) {
        int64_t* h = &cnt[(size_t)c * nkeys];
        for (int64_t a = n * c / nch; a < n * (c + 1) / nch; ++a) h[key[a]]++;
    }
    int64_t run = 0;
    for (int64_t k = 0; k < nkeys; ++k) {
        off[k] = run;
        for (int c = 0; c < nch; ++c) {
            const int64_t v = cnt[(size_t)c * nkeys + k];
            cnt[(size_t)c * nkeys + k] = run;
            run += v;
        }
    }
    off[nkeys] = run;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nch; ++c) {
        int64_t* pos = &cnt[(size_t)c * nkeys];
        for (int64_t a = n * c / nch; a < n * (c + 1) / nch; ++a) order[pos[key[a]]++] = a;
    }
}

void root_box(const double* x, const double* w, int64_t N, int dim, double lo[3], double* W) {
    double hi[3];
    for (int k = 0; k < 3; ++k) { lo[k] = 0.0; hi[k] = 0.0; }
    for (int64_t i = 0; i < N; ++i) {
        const double side = dim == 2 ? std::sqrt(w[i]) : std::cbrt(w[i]);
        const double half = 0.5 * side;
        for (int k = 0; k < dim; ++k) {
            const double a = x[dim * i + k] - half, b = x[dim * i + k] + half;
            if (i == 0 || a < lo[k]) lo[k] = a;
            if (i == 0 || b > hi[k]) hi[k] = b;
        }
    }
    double Wm = 0.0;
    for (int k = 0; k < dim; ++k) Wm = std::max(Wm, hi[k] - lo[k]);
    *W = Wm;
}

static inline int cell_coord(double xk, double lo, double w, int s) {
    const double t = std::floor((xk - lo) / w);
    int c = t < 0.0 ? 0 : (t > (double)(s - 1) ? s - 1 : (int)t);
    return c;
}

int num_levels(const double* x, int64_t N, int dim, const double lo[3], double W, int occupancy) {
    for (int L = 0; L <= 24; ++L) {
        const int s = 1 << L;
        const double w = W / s;
        std::unordered_map<int64_t, int> cnt;
        cnt.reserve((size_t)std::min<int64_t>(N, (int64_t)1 << 22));
        int mx = 0;
        for (int64_t i = 0; i < N; ++i) {
            int64_t flat = 0;
            for (int k = 0; k < dim; ++k) flat = flat * s + cell_coord(x[dim * i + k], lo[k], w, s);
            mx = std::max(mx, ++cnt[flat]);
            if (mx > occupancy) break;
        }
        if (mx <= occupancy) return L;
    }
    return 24;
}

void plan_sublevels(int dim, int L, bool fractional, int skip_levels, std::vector<int>& kinds,
                    std::vector<int>& levels) {
    kinds.clear();
    levels.clear();
    for (int l = 0; l < L; ++l) {
        kinds.push_back(KIND_CELL);
        levels.push_back(l);
        if (fractional && l >= skip_levels) {
            if (dim == 3) {
                kinds.push_back(KIND_FACE);
                levels.push_back(l);
            }
            kinds.push_back(KIND_EDGE);
            levels.push_back(l);
        }
    }
}

// Families of centres (Sec. 4.1, 4.2): per axis 'I' = on a cell boundary
// (index 1..s-1, offset 0), 'H' = mid-cell (index 0..s-1, offset 1/2).
struct Family {
    int nf;
    bool I[3][3];
};

static Family families(int dim, int kind) {
    Family f{};
    auto set = [&](int q, bool a, bool b, bool c) { f.I[q][0] = a; f.I[q][1] = b; f.I[q][2] = c; };
    if (kind == KIND_CELL) { f.nf = 1; set(0, false, false, false); }
    else if (dim == 2) { f.nf = 2; set(0, true, false, false); set(1, false, true, false); }
    else if (kind == KIND_FACE) { f.nf = 3; set(0, true, false, false); set(1, false, true, false); set(2, false, false, true); }
    else { f.nf = 3; set(0, true, true, false); set(1, true, false, true); set(2, false, true, true); }
    return f;
}

void partition(const Tree& t, const double* x, int kind, int s, const std::vector<int>& active_ids,
               SublevelPlan& out, std::vector<int>& box_of) {
    const int dim = t.dim;
    const double w = t.W / s;
    const Family fam = families(dim, kind);
    // family sizes and offsets (ids follow the paper's listing order)
    int64_t fam_off[4] = {0, 0, 0, 0};
    int64_t ext[3][3];
    for (int q = 0; q < fam.nf; ++q) {
        int64_t sz = 1;
        for (int k = 0; k < dim; ++k) {
            ext[q][k] = fam.I[q][k] ? s - 1 : s;
            sz *= ext[q][k];
        }
        fam_off[q + 1] = fam_off[q] + sz;
    }
    const int64_t ncent = fam_off[fam.nf];
    const int64_t na = (int64_t)active_ids.size();
    RawBuf<int64_t> owner((size_t)na);

#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < na; ++a) {
        const int i = active_ids[a];
        const double* p = x + (int64_t)dim * i;
        int c[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) c[k] = cell_coord(p[k], t.lo[k], w, s);
        if (kind == KIND_CELL) {
            int64_t flat = 0;
            for (int k = 0; k < dim; ++k) flat = flat * s + c[k];
            owner[a] = flat;
            continue;
        }
        // the candidate centres around the DOF's cell: the smallest distance,
        // then the lowest id within kTie of it
        auto visit = [&](auto&& f) {
            for (int q = 0; q < fam.nf; ++q) {
                int jlo[3], jhi[3];
                for (int k = 0; k < 3; ++k) { jlo[k] = 0; jhi[k] = 0; }
                for (int k = 0; k < dim; ++k) {
                    if (fam.I[q][k]) { jlo[k] = std::max(1, c[k] - 1); jhi[k] = std::min(s - 1, c[k] + 2); }
                    else { jlo[k] = std::max(0, c[k] - 1); jhi[k] = std::min(s - 1, c[k] + 1); }
                }
                for (int j0 = jlo[0]; j0 <= jhi[0]; ++j0)
                    for (int j1 = jlo[1]; j1 <= jhi[1]; ++j1)
                        for (int j2 = jlo[2]; j2 <= jhi[2]; ++j2) {
                            const int js[3] = {j0, j1, j2};
                            int64_t id = 0;
                            double d2 = 0.0;
                            for (int k = 0; k < dim; ++k) {
                                const double ck = t.lo[k] + ((double)js[k] + (fam.I[q][k] ? 0.0 : 0.5)) * w;
                                const double dd = p[k] - ck;
                                d2 = d2 + dd * dd;
                                id = id * ext[q][k] + (fam.I[q][k] ? js[k] - 1 : js[k]);
                            }
                            f(id + fam_off[q], d2);
                        }
            }
        };
        // at most 3 families x (4 x 4 x 3) candidates (3D edges)
        constexpr int MAXC = 160;
        int64_t cid[MAXC];
        double cd2[MAXC];
        int ncand = 0;
        double best = -1.0;
        visit([&](int64_t id, double d2) {
            if (ncand < MAXC) {
                cid[ncand] = id;
                cd2[ncand] = d2;
                ++ncand;
            }
            if (best < 0.0 || d2 < best) best = d2;
        });
        const double lim = best * (1.0 + kTie);
        int64_t best_id = -1;
        for (int e = 0; e < ncand; ++e)
            if (cd2[e] <= lim && (best_id < 0 || cid[e] < best_id)) best_id = cid[e];
        owner[a] = best_id;
    }
    // bucket by owner (stable: ascending DOF ids inside a box); the members
    // of the non-empty centres, in centre order, are the bucketed ids
    std::vector<int64_t> count;
    RawBuf<int64_t> order((size_t)na);
    stable_bucket(owner.data(), na, ncent, count, order.data());
    out.members.resize(na);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < na; ++e) out.members[e] = active_ids[order[e]];
    std::vector<int64_t> used;                       // the non-empty centres
    for (int64_t b = 0; b < ncent; ++b)
        if (count[b + 1] > count[b]) used.push_back(b);
    const int nbox = (int)used.size();
    out.box_off.resize(nbox + 1);
    out.centers.resize(3 * (size_t)nbox);
    out.box_off[0] = 0;
#pragma omp parallel for schedule(static)
    for (int bi = 0; bi < nbox; ++bi) {
        const int64_t b = used[bi];
        out.box_off[bi + 1] = count[b + 1];
        // centre of box b
        int q = 0;
        while (b >= fam_off[q + 1]) ++q;
        int64_t rem = b - fam_off[q];
        int js[3] = {0, 0, 0};
        for (int k = dim - 1; k >= 0; --k) {
            js[k] = (int)(rem % ext[q][k]);
            rem /= ext[q][k];
            if (fam.I[q][k]) js[k] += 1;
        }
        for (int k = 0; k < 3; ++k)
            out.centers[3 * (size_t)bi + k] = k < dim ? t.lo[k] + ((double)js[k] + (fam.I[q][k] ? 0.0 : 0.5)) * w : 0.0;
        for (int64_t e = count[b]; e < count[b + 1]; ++e) box_of[out.members[e]] = bi;
    }
    out.nbox = nbox;
}

namespace {

// per-phase time of build_near_groups (trace only)
bool g_geo_trace = false;
double g_geo_ms[6] = {0, 0, 0, 0, 0, 0};

inline double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Work arrays of one thread of build_near_groups, reused box after box, and
// the thread's share of the output (boxes in the order the thread took them).
struct NearScratch {
    std::vector<int> nl, blocks;
    std::vector<int> order, col_pat, pat_data, canon, gid, gfirst;
    std::vector<int64_t> pat_off;
    std::vector<uint64_t> pat_hash;
    std::vector<uint32_t> mark;   // epoch stamps over all DOFs
    uint32_t epoch = 0;
    // output arena
    std::vector<int> near, cols, gcol0, gn, gsci;
    double ms[4] = {0, 0, 0, 0};   // trace: proxy scan, patterns, near list, groups
};

struct BoxOut {
    int thread;
    int64_t near0, near1, cols0, grp0, grp1;
    int sci;
};

// a 64-bit mixing function (the splitmix64 finalizer), summed over a set
// for an order-independent hash
inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

// S of the grid table T(o) = G(h |o|) (o != 0), T(0) = k0, over the offsets
// o in [0, n)^dim, in fixed chunks so that the sum is the same on every run.
double table_spread(int n, int dim, double h, int kernel_id, double k0) {
    const int64_t tot = dim == 2 ? (int64_t)n * n : (int64_t)n * n * n;
    constexpr int64_t NCH = 256;
    std::vector<double> ss(NCH, 0.0), mx(NCH, 0.0);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < NCH; ++c) {
        const int64_t e0 = tot * c / NCH, e1 = tot * (c + 1) / NCH;
        for (int64_t e = e0; e < e1; ++e) {
            int64_t t = e;
            double r2 = 0.0;
            for (int q = 0; q < dim; ++q) {
                const double dd = (double)(t % n) * h;
                r2 += dd * dd;
                t /= n;
            }
            const double v = e == 0 ? k0
                             : kernel_id == 0 ? -std::log(r2) * (0.25 / kPi)
                                              : (0.25 / kPi) / std::sqrt(r2);
            ss[c] += v * v;
            mx[c] = std::max(mx[c], std::fabs(v));
        }
    }
    double s = 0.0, m = 0.0;
    for (int64_t c = 0; c < NCH; ++c) {
        s += ss[c];
        m = std::max(m, mx[c]);
    }
    return s > 0.0 ? m * std::sqrt((double)tot / s) : 1.0;
}

void append_plan(SublevelPlan& p, SublevelPlan&& q) {
    // the first problem's plan is taken over whole (the offsets of an empty
    // plan are all 0), which saves copying its near-field lists
    if (p.nbox == 0 && p.members.empty() && p.near.empty() && p.cols.empty() && p.centers.empty() &&
        p.grp_col0.empty() && p.box_sci.empty() && p.box_off.size() == 1 && p.near_off.size() == 1 &&
        p.grp_off.size() == 1 && q.box_off.size() == (size_t)q.nbox + 1) {
        p = std::move(q);
        return;
    }
    const int64_t mo = (int64_t)p.members.size(), no = (int64_t)p.near.size(), go = p.grp_off.back();
    for (int b = 1; b <= q.nbox; ++b) {
        p.box_off.push_back(q.box_off[b] + mo);
        p.near_off.push_back(q.near_off[b] + no);
        p.grp_off.push_back(q.grp_off[b] + go);
    }
    p.members.insert(p.members.end(), q.members.begin(), q.members.end());
    p.cols.insert(p.cols.end(), q.cols.begin(), q.cols.end());
    p.near.insert(p.near.end(), q.near.begin(), q.near.end());
    p.centers.insert(p.centers.end(), q.centers.begin(), q.centers.end());
    p.grp_col0.insert(p.grp_col0.end(), q.grp_col0.begin(), q.grp_col0.end());
    p.grp_n.insert(p.grp_n.end(), q.grp_n.begin(), q.grp_n.end());
    p.grp_sci.insert(p.grp_sci.end(), q.grp_sci.begin(), q.grp_sci.end());
    p.box_sci.insert(p.box_sci.end(), q.box_sci.begin(), q.box_sci.end());
    p.nbox += q.nbox;
}

bool grid_layout(const double* X, const double* Wt, int64_t N, int d, int64_t off, int* n_out, double* h_out,
                 std::vector<int>& dof_of) {
    const int n = (int)std::llround(std::pow((double)N, 1.0 / d));
    int64_t nn = 1;
    for (int k = 0; k < d; ++k) nn *= n;
    if (n < 2 || nn != N) return false;
    double lo[3], hx = 0;
    for (int k = 0; k < d; ++k) {
        double mn = X[k], mx = X[k];
        for (int64_t i = 0; i < N; ++i) {
            mn = std::min(mn, X[d * i + k]);
            mx = std::max(mx, X[d * i + k]);
        }
        const double hk = (mx - mn) / (n - 1);
        if (k == 0) hx = hk;
        if (std::fabs(hk - hx) > 1e-12 * hx) return false;
        lo[k] = mn;
    }
    const double wv = Wt[0];
    for (int64_t i = 0; i < N; ++i)
        if (Wt[i] != wv) return false;
    if (std::fabs(std::pow(wv, 1.0 / d) - hx) > 1e-9 * hx) return false;
    dof_of.assign((size_t)N, -1);
    for (int64_t i = 0; i < N; ++i) {
        int64_t gpos = 0;
        for (int k = 0; k < d; ++k) {
            const double t = (X[d * i + k] - lo[k]) / hx;
            const int64_t id = std::llround(t);
            if (id < 0 || id >= n || std::fabs(t - id) > 1e-6) return false;
            gpos = gpos * n + id;
        }
        if (dof_of[gpos] != -1) return false;
        dof_of[gpos] = (int)(off + i);
    }
    *n_out = n;
    *h_out = hx;
    return true;
}

void geometry_trace(bool on, double* ms) {
    if (ms)
        for (int q = 0; q < 6; ++q) ms[q] = g_geo_ms[q];
    for (double& v : g_geo_ms) v = 0.0;
    g_geo_trace = on;
}

void build_near_groups(const Tree& t, const double* x, int s, double proxy_radius, int second_kind,
                       const std::vector<int>& active_ids, const std::vector<char>& active,
                       const std::vector<int>& box_of, const SciHost& sci, SublevelPlan& p,
                       NearCache* cache) {
    const bool tr = g_geo_trace;
    const double tb0 = tr ? now_ms() : 0.0;
    const int dim = t.dim;
    const double w = t.W / s;
    const double R = proxy_radius * w;
    // strictly inside the proxy sphere: a DOF within a relative kTie of the
    // radius counts as on it (grids put DOFs exactly there, e.g. the 3D
    // faces of a 3 x 3 x 3 cell; rounding must not decide)
    const double R2 = R * R * (1.0 - kTie);
    const int nsub = (int)sci.blk.size();
    // bins of the active DOFs: cells of width w at this level
    int64_t nbins = 1;
    for (int k = 0; k < dim; ++k) nbins *= s;
    const int64_t nact = (int64_t)active_ids.size();
    RawBuf<int64_t> bin_of((size_t)nact);
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < nact; ++a) {
        const double* q = x + (int64_t)dim * active_ids[a];
        int64_t flat = 0;
        for (int k = 0; k < dim; ++k) flat = flat * s + cell_coord(q[k], t.lo[k], w, s);
        bin_of[a] = flat;
    }
    std::vector<int64_t> boff;
    RawBuf<int64_t> border((size_t)nact);
    stable_bucket(bin_of.data(), nact, nbins, boff, border.data());
    // binned copies of the ids, coordinates and boxes, so that the proxy
    // scans below read contiguous memory
    RawBuf<int> bins((size_t)nact), bins_box((size_t)nact);
    RawBuf<double> bins_x((size_t)nact * dim);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nact; ++e) {
        const int i = active_ids[border[e]];
        bins[e] = i;
        bins_box[e] = box_of[i];
        for (int k = 0; k < dim; ++k) bins_x[(size_t)dim * e + k] = x[(int64_t)dim * i + k];
    }

    const int nb = p.nbox;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    std::vector<NearScratch> scr(nthr);
    if (cache) {
        // the stamps left in a reused array are all at most its epoch, so the
        // epochs that follow never match them
        cache->mark.resize(nthr);
        cache->epoch.resize(nthr, 0u);
        for (int q = 0; q < nthr; ++q) {
            scr[q].mark.swap(cache->mark[q]);
            scr[q].epoch = cache->epoch[q];
        }
    }
    std::vector<BoxOut> bo(nb);
    const double tb1 = tr ? now_ms() : 0.0;

    // chunks of up to 16 boxes, but at least ~8 chunks per thread, so that the
    // few-box sublevels near the top spread over all threads
    const int chunk = std::max(1, std::min(16, nb / (8 * nthr)));
#pragma omp parallel for schedule(dynamic, chunk)
    for (int b = 0; b < nb; ++b) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        NearScratch& S = scr[tid];
        double c0 = tr ? now_ms() : 0.0;
        const double* ctr = &p.centers[3 * (size_t)b];
        std::vector<int>& nl = S.nl;
        nl.clear();
        // proxy interior
        int lo_b[3] = {0, 0, 0}, hi_b[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) {
            lo_b[k] = cell_coord(ctr[k] - R, t.lo[k], w, s);
            hi_b[k] = cell_coord(ctr[k] + R, t.lo[k], w, s);
        }
        for (int b0 = lo_b[0]; b0 <= hi_b[0]; ++b0)
            for (int b1 = lo_b[1]; b1 <= hi_b[1]; ++b1)
                for (int b2 = lo_b[2]; b2 <= hi_b[2]; ++b2) {
                    int64_t flat = (int64_t)b0 * s + b1;
                    if (dim == 3) flat = flat * s + b2;
                    for (int64_t e = boff[flat]; e < boff[flat + 1]; ++e) {
                        if (bins_box[e] == b) continue;
                        const double* q = &bins_x[(size_t)dim * e];
                        double d2 = 0.0;
                        for (int k = 0; k < dim; ++k) {
                            const double dd = q[k] - ctr[k];
                            d2 = d2 + dd * dd;
                        }
                        if (d2 < R2) nl.push_back(bins[e]);
                    }
                    if (dim == 2) break;
                }

        double c1 = tr ? now_ms() : 0.0;
        // SCI patterns (Sec. 4.3/4.4): the pattern of column j is the set of
        // active DOFs outside the box in the past SCI blocks holding j.  It
        // depends only on j's block ids, so columns are sorted by that tuple
        // and each distinct tuple's pattern is formed once.
        const int64_t n0 = p.box_off[b], n1 = p.box_off[b + 1];
        const int nc = (int)(n1 - n0);
        auto blk = [&](int l, int q) { return sci.blk[q][p.members[n0 + l]]; };
        std::vector<int>& order = S.order;
        order.resize(nc);
        for (int l = 0; l < nc; ++l) order[l] = l;
        if (nsub > 0)
            std::sort(order.begin(), order.end(), [&](int u, int v) {
                for (int q = 0; q < nsub; ++q) {
                    const int bu = blk(u, q), bv = blk(v, q);
                    if (bu != bv) return bu < bv;
                }
                return u < v;
            });
        // Distinct tuples' patterns are formed with an epoch-stamped mark
        // array over the DOFs (deduplicated, unsorted) together with an
        // order-independent hash; equal patterns are found by sorting on
        // (hash, size) and confirmed element by element with the marks.
        std::vector<uint32_t>& mark = S.mark;
        if (mark.size() < box_of.size()) mark.assign(box_of.size(), 0u);
        auto next_epoch = [&]() {
            if (++S.epoch == 0) {
                std::fill(mark.begin(), mark.end(), 0u);
                S.epoch = 1;
            }
            return S.epoch;
        };
        S.col_pat.assign(nc, 0);
        S.pat_data.clear();
        S.pat_off.assign(1, 0);
        S.pat_hash.clear();
        int npat = 0;
        for (int e = 0; e < nc; ++e) {
            const int l = order[e];
            bool same = e > 0;
            if (same)
                for (int q = 0; q < nsub && same; ++q) same = blk(l, q) == blk(order[e - 1], q);
            if (!same) {
                const uint32_t ep = next_epoch();
                uint64_t h = 0;
                for (int q = 0; q < nsub; ++q) {
                    const int bid = blk(l, q);
                    if (bid < 0) continue;
                    for (int i : sci.members[bid])
                        if (active[i] && box_of[i] != b && mark[i] != ep) {
                            mark[i] = ep;
                            S.pat_data.push_back(i);
                            h += mix64((uint64_t)(uint32_t)i);
                        }
                }
                S.pat_off.push_back((int64_t)S.pat_data.size());
                S.pat_hash.push_back(h);
                ++npat;
            }
            S.col_pat[l] = npat - 1;
        }
        double c2 = tr ? now_ms() : 0.0;
        // the SCI-coupled DOFs of the near field: the union of all patterns
        {
            const uint32_t ep = next_epoch();
            for (int i : nl) mark[i] = ep;
            for (int i : S.pat_data)
                if (mark[i] != ep) {
                    mark[i] = ep;
                    nl.push_back(i);
                }
        }
        std::sort(nl.begin(), nl.end());

        double c3 = tr ? now_ms() : 0.0;
        bool any = false;
        for (int q = 0; q < npat; ++q) any = any || S.pat_off[q + 1] > S.pat_off[q];
        // patterns with equal content share a canonical id
        auto plen = [&](int q) { return S.pat_off[q + 1] - S.pat_off[q]; };
        std::vector<int>& byh = S.gid;               // scratch: pattern ids by (hash, size)
        byh.resize(npat);
        for (int q = 0; q < npat; ++q) byh[q] = q;
        std::sort(byh.begin(), byh.end(), [&](int u, int v) {
            if (S.pat_hash[u] != S.pat_hash[v]) return S.pat_hash[u] < S.pat_hash[v];
            if (plen(u) != plen(v)) return plen(u) < plen(v);
            return u < v;
        });
        S.canon.assign(npat, -1);
        for (int e0 = 0; e0 < npat;) {
            int e1 = e0 + 1;
            while (e1 < npat && S.pat_hash[byh[e1]] == S.pat_hash[byh[e0]] && plen(byh[e1]) == plen(byh[e0])) ++e1;
            for (int u = e0; u < e1; ++u) {
                const int q = byh[u];
                if (S.canon[q] >= 0) continue;
                S.canon[q] = q;
                if (u + 1 == e1) break;
                const uint32_t ep = next_epoch();
                for (int64_t z = S.pat_off[q]; z < S.pat_off[q + 1]; ++z) mark[S.pat_data[z]] = ep;
                for (int v = u + 1; v < e1; ++v) {
                    const int r = byh[v];
                    if (S.canon[r] >= 0) continue;
                    bool eq = true;
                    for (int64_t z = S.pat_off[r]; z < S.pat_off[r + 1] && eq; ++z) eq = mark[S.pat_data[z]] == ep;
                    if (eq) S.canon[r] = q;
                }
            }
            e0 = e1;
        }
        // groups by pattern, numbered in order of first appearance
        S.gid.assign(nc, 0);
        int ng = 1;
        if (second_kind) {
            S.gfirst.assign(npat, -1);
            ng = 0;
            for (int l = 0; l < nc; ++l) {
                const int c = S.canon[S.col_pat[l]];
                if (S.gfirst[c] < 0) S.gfirst[c] = ng++;
                S.gid[l] = S.gfirst[c];
            }
        }
        BoxOut& o = bo[b];
        o.thread = tid;
        o.sci = any ? 1 : 0;
        o.near0 = (int64_t)S.near.size();
        S.near.insert(S.near.end(), nl.begin(), nl.end());
        o.near1 = (int64_t)S.near.size();
        o.cols0 = (int64_t)S.cols.size();
        o.grp0 = (int64_t)S.gn.size();
        if (ng == 1) {
            S.gcol0.push_back(0);
            S.cols.insert(S.cols.end(), p.members.begin() + n0, p.members.begin() + n1);
            S.gn.push_back(nc);
            S.gsci.push_back(any ? 1 : 0);
        } else {
            // counting sort of the columns by group, ascending inside a group
            std::vector<int>& gcnt = S.gfirst;
            gcnt.assign(ng + 1, 0);
            for (int l = 0; l < nc; ++l) gcnt[S.gid[l] + 1]++;
            for (int g = 0; g < ng; ++g) gcnt[g + 1] += gcnt[g];
            const int64_t base = (int64_t)S.cols.size();
            S.cols.resize(base + nc);
            for (int g = 0; g < ng; ++g) {
                S.gcol0.push_back(gcnt[g]);
                S.gn.push_back(gcnt[g + 1] - gcnt[g]);
                S.gsci.push_back(0);
            }
            for (int l = 0; l < nc; ++l) {
                const int g = S.gid[l];
                S.cols[base + gcnt[g]++] = p.members[n0 + l];
                if (S.pat_off[S.col_pat[l] + 1] > S.pat_off[S.col_pat[l]]) S.gsci[o.grp0 + g] = 1;
            }
        }
        o.grp1 = (int64_t)S.gn.size();
        if (tr) {
            const double c4 = now_ms();
            S.ms[0] += c1 - c0;
            S.ms[1] += c2 - c1;
            S.ms[2] += c3 - c2;
            S.ms[3] += c4 - c3;
        }
    }
    const double tb2 = tr ? now_ms() : 0.0;
    p.near_off.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) p.near_off[b + 1] = p.near_off[b] + (bo[b].near1 - bo[b].near0);
    p.near.resize(p.near_off[nb]);
    p.cols.resize(p.members.size());
    p.grp_off.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) p.grp_off[b + 1] = p.grp_off[b] + (bo[b].grp1 - bo[b].grp0);
    p.grp_col0.resize(p.grp_off[nb]);
    p.grp_n.resize(p.grp_off[nb]);
    p.grp_sci.resize(p.grp_off[nb]);
    p.box_sci.assign(nb, 0);
#pragma omp parallel for schedule(static)
    for (int b = 0; b < nb; ++b) {
        const BoxOut& o = bo[b];
        const NearScratch& S = scr[o.thread];
        std::copy(S.near.begin() + o.near0, S.near.begin() + o.near1, p.near.begin() + p.near_off[b]);
        std::copy(S.cols.begin() + o.cols0, S.cols.begin() + o.cols0 + (p.box_off[b + 1] - p.box_off[b]),
                  p.cols.begin() + p.box_off[b]);
        for (int64_t g = 0; g < o.grp1 - o.grp0; ++g) {
            p.grp_col0[p.grp_off[b] + g] = S.gcol0[o.grp0 + g];
            p.grp_n[p.grp_off[b] + g] = S.gn[o.grp0 + g];
            p.grp_sci[p.grp_off[b] + g] = S.gsci[o.grp0 + g];
        }
        p.box_sci[b] = o.sci;
    }
    if (cache)
        for (int q = 0; q < nthr; ++q) {
            scr[q].mark.swap(cache->mark[q]);
            cache->epoch[q] = scr[q].epoch;
        }
    if (tr) {
        g_geo_ms[0] += tb1 - tb0;                      // bins and set-up (wall)
        g_geo_ms[1] += now_ms() - tb2;                 // gather (wall)
        for (const NearScratch& S : scr)               // per-box phases (thread time)
            for (int q = 0; q < 4; ++q) g_geo_ms[2 + q] += S.ms[q];
    }
}

}  // namespace hif
