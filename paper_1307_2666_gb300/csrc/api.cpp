// C ABI of the HIF-IE library: host orchestration of the factorization (Algorithms 4.1 / 4.2),
// apply / solve sweeps, FP64 direct-sum operator and refinement loops.
//
// The host runs the integer bookkeeping of each sublevel (geometry.cpp) and
// launches the floating-point work: per sublevel one fold launch (proxy
// matrices folded into R factors), one ID launch over all column groups and
// one elimination launch; the host reads back only the ranks and skeleton
// permutations it needs to form the next sublevel.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hif.h"
#include "geometry.h"
#include "launch.h"
#include "prof.h"
#include "refine_rule.h"

namespace hif {

// ------------------------------------------------------------ plumbing --

struct Err {
    hif_status s;
};

#define HIF_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            std::snprintf(g_last_error, sizeof(g_last_error), "%s:%d %s: %s", __FILE__, \
                          __LINE__, #call, cudaGetErrorString(e_));                     \
            throw Err{e_ == cudaErrorMemoryAllocation ? HIF_ENOMEM : HIF_ECUDA};        \
        }                                                                               \
    } while (0)

static thread_local char g_last_error[512];
// rows per fold chunk chosen by the autotuner, per (box width, element size)
static std::mutex g_fold_rc_mu;
static std::map<int, int> g_fold_rc;
static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static void fail(hif_status s, const char* msg) {
    std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
    throw Err{s};
}

// Device allocation that frees itself.
struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
    ~DevMem() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    void* ensure(size_t b) {
        if (b <= bytes && p) return p;
        release();
        const size_t want = std::max<size_t>(b, 256);
        HIF_CUDA(cudaMalloc(&p, want));
        bytes = want;
        return p;
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

template <typename T>
static void upload(DevMem& d, const std::vector<T>& h, cudaStream_t st) {
    d.ensure(h.size() * sizeof(T));
    if (!h.empty()) HIF_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

static bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Input array: device pointer used in place, host array copied.
struct InArr {
    const double* d = nullptr;
    DevMem own;
    void set(const double* p, size_t count, cudaStream_t st) {
        if (is_device_ptr(p)) {
            d = p;
        } else {
            own.ensure(count * sizeof(double));
            HIF_CUDA(cudaMemcpyAsync(own.p, p, count * sizeof(double), cudaMemcpyHostToDevice, st));
            d = own.as<double>();
        }
    }
};

// One independent problem of a handle: DOFs [off, off + N) of the
// concatenated arrays, with its own tree and direct-sum structure.
struct Segment {
    int64_t off = 0, N = 0;
    Tree tree{};
    std::vector<int> kinds, levels;
    bool grid = false;
    bool sym = false;             // b == c and equal weights: A symmetric, Y'_c compressed (Sec. 5)
    int gn = 0;
    double gh = 0;
    DevMem dof_of, table, table_df;
    DevMem tc_rows, tc_tmax;      // digit rows of the table for the tensor-core sum (built on first use)
    double spread = 1.0;          // max|T| sqrt(#T) / |T|_2 of the table (scale of the short sums' error)
};

struct FactorScratch {
    DevMem d_ed, d_ed_big, d_eg, ews, piv, ldl_fail, gemm_probs, elim_order, elim_next;
};

constexpr int KIND_TOP = 3;   // the top blocks, eliminated as boxes without skeletons

struct SubFactor {
    int kind = 0, level = 0;
    int nbox = 0;                  // boxes with r > 0
    std::vector<BoxFac> hbox;
    DevMem boxes, sk, rd, pool, perm;
    int max_kr2 = 0;               // max over boxes of k + 2 r
    // sweep plan: boxes whose vectors exceed shared memory use a global work
    // space (offsets per right-hand side); the CTA size is tuned per sublevel
    bool global = false;
    DevMem gws_off;
    int64_t gws_units = 0;
    int threads = 256;
    // boxes of the one-CTA sweep kernel (sboxes) and the wide boxes whose
    // passes run as stage launches over the whole GPU (wboxes, work space at
    // wws_off per box in units of k + 2 r, per right-hand side)
    DevMem sboxes, wboxes, wws_off;
    int nsmall = 0, nwide = 0, wmax_k = 0, wmax_r = 0, max_kr2_small = 0;
    int64_t wws_units = 0;
    // algorithmic elements the two passes of one sweep read from the factors
    // (T twice, X or Y once each, one triangle of L^{-1}/U^{-1} or L/U per
    // pass, D) and the box vectors they gather and scatter (sum of k + r)
    double sweep_factor_elems = 0, sweep_perm_ints = 0, sweep_vec_elems = 0;
};

// A captured sequence of sweeps (one operation, one right-hand-side count, one
// work buffer) and the number of kernels in it.
struct SweepGraph {
    int op = 0, nrhs = 0;
    void* xw = nullptr;            // the buffers baked into the graph
    void* ws = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;
};

}  // namespace hif

struct hif_handle_s {
    int dim = 2, kernel_id = 0, precision = 0, second_kind = 1;
    int64_t N = 0;
    double eps = 0;
    hif_options opt{};
    cudaStream_t st = nullptr;
    int elem = 8;
    hif::DevMem x, w, a, b, c, kself, kself_im, proxy;
    double wavenumber = 0.0;   // kernel 2
    int ncomp = 1;             // real DOFs per point (2: real embedding of the complex operator)
    std::vector<double> hx, hw;
    std::vector<std::unique_ptr<hif::Segment>> segs;
    hif::DevMem seg_off, seg_n;
    int P = 0;
    // SCI store
    hif::DevMem sci_blk, sci_loc, blk_ptr, blk_k;
    std::vector<void*> blk_ptr_h;
    std::vector<int> blk_k_h;
    std::vector<std::unique_ptr<hif::DevMem>> sci_pools;
    // factors
    std::vector<std::unique_ptr<hif::SubFactor>> subs;
    // direct-sum scratch
    hif::DevMem vbuf, ybuf, vdf, tc_xb, tc_xmax, tc_status;
    int num_sms = 0;
    // work buffers
    hif::DevMem work, work2, tmp, status, sweep_ws, sweep_off;
    hif_stats_t stats{};
    // CUDA graphs of the sweeps, captured on a stream of the handle's own
    std::vector<hif::SweepGraph> graphs;
    cudaStream_t cap_st = nullptr;
    // streams forked from st for concurrent launches of one sublevel, and
    // the fork / join events (created on first use)
    cudaStream_t aux[8] = {};
    cudaEvent_t fork = nullptr, join[8] = {};
    cudaStream_t aux_stream(size_t i) {
        i %= 8;
        if (!aux[i] && cudaStreamCreateWithFlags(&aux[i], cudaStreamNonBlocking) != cudaSuccess) aux[i] = nullptr;
        return aux[i] ? aux[i] : st;
    }
    cudaEvent_t fork_ev() {
        if (!fork) cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        return fork;
    }
    cudaEvent_t join_ev(size_t i) {
        i %= 8;
        if (!join[i]) cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
        return join[i];
    }
    ~hif_handle_s() {
        for (auto& g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (cap_st) cudaStreamDestroy(cap_st);
        for (auto& s2 : aux)
            if (s2) cudaStreamDestroy(s2);
        if (fork) cudaEventDestroy(fork);
        for (auto& e : join)
            if (e) cudaEventDestroy(e);
    }
};

namespace hif {

static GeomDev geom(hif_handle h) {
    GeomDev g;
    g.x = h->x.as<double>();
    g.w = h->w.as<double>();
    g.a = h->a.as<double>();
    g.b = h->b.as<double>();
    g.c = h->c.as<double>();
    g.kself = h->kself.as<double>();
    g.kself_im = h->ncomp == 2 ? h->kself_im.as<double>() : nullptr;
    g.wavenumber = h->wavenumber;
    g.N = h->N;
    g.dim = h->dim;
    g.kernel_id = h->kernel_id;
    g.ncomp = h->ncomp;
    return g;
}

static SciDev scidev(hif_handle h, int nsub) {
    SciDev s;
    s.blk = h->sci_blk.as<int>();
    s.loc = h->sci_loc.as<int>();
    s.ptr = h->blk_ptr.as<void*>();
    s.kb = h->blk_k.as<int>();
    s.nsub = nsub;
    s.N = h->N;
    return s;
}

static void check_status(hif_handle h) {
    int st = 0;
    HIF_CUDA(cudaMemcpyAsync(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    HIF_CUDA(cudaStreamSynchronize(h->st));
    if (st & DEV_SINGULAR) fail(HIF_ESINGULAR, "zero pivot in an elimination block");
    if (st & DEV_NONFINITE) fail(HIF_ENUMERIC, "non-finite value in the factorization");
    if (st & DEV_TIMEOUT) fail(HIF_ETIMEOUT, "a bounded wait of a tensor-core kernel ran out");
}

// Detect whether a problem is a full uniform tensor grid: x = lo + h (idx + 1/2)
// with equal weights h^d.  Then K_ij = G(h |idx_i - idx_j|) w exactly and the
// direct sum is a convolution.
static void detect_grid(hif_handle h, Segment& sg) {
    sg.grid = false;
    std::vector<int> dof_of;
    int n = 0;
    double hx = 0.0;
    if (!grid_layout(h->hx.data() + (size_t)h->dim * sg.off, h->hw.data() + sg.off, sg.N, h->dim, sg.off, &n, &hx,
                     dof_of))
        return;
    sg.grid = true;
    sg.gn = n;
    sg.gh = hx;
    upload(sg.dof_of, dof_of, h->st);
}

static int env_int(const char* name, int dflt) {
    const char* v = std::getenv(name);
    if (!v || !*v) return dflt;
    return std::atoi(v);
}

struct BigBuffers {
    DevMem bb, bg, state, YK, YS, vv, vw, vt, est, nrm, perm, F, gv, nrm0;
    DevMem q_yoff, q_m, q_n, q_tau, q_G, q_T, q_W, q_Gp, q_Wp, q_gpoff, q_wpoff;
};

// The column-pivoted QR of all large groups of a sublevel: by panels of
// HIF_BIG_QP_NB pivots (blocked, one trailing product per panel) or, at 1,
// one launch pair per pivot.  Default: panels of 32 in FP32; one pivot per
// step in FP64, whose exact norms at every step keep the rank decisions of
// the symmetric and full proxy matrices identical at eps = 1e-9 (the blocked
// update's rounding moved one decision at the threshold by one).
template <typename T>
static void run_big_pivoted_qr(BigArgs& a, BigBuffers& B, const std::vector<BigGroup>& bgv, int max_n, int maxk,
                               int64_t voff, cudaStream_t st) {
    const int ng = (int)bgv.size();
    int max_m = 0;
    for (const BigGroup& x : bgv) max_m = std::max(max_m, x.m);
    const int nbq = std::min(32, std::max(1, env_int("HIF_BIG_QP_NB", sizeof(T) == 4 ? 32 : 1)));
    std::vector<BigState> hs(ng);
    if (nbq > 1) {
        B.F.ensure(sizeof(T) * std::max<int64_t>(voff, 1) * nbq);
        B.gv.ensure(sizeof(T) * 32 * std::max(ng, 1));
        B.nrm0.ensure(sizeof(double) * std::max<int64_t>(voff, 1));
        a.F = B.F.p;
        a.gv = B.gv.p;
        a.nrm0 = B.nrm0.as<double>();
        a.nb = nbq;
    } else {
        a.nrm0 = nullptr;
    }
    HIF_CUDA((big_qr_init<T>(a, ng, max_n, st)));
    if (nbq > 1) {
        int step = 0;
        for (int panel = 0; panel <= maxk; ++panel) {
            {
                ProfRange pr(PROF_BIG_QR, st, 0.0, 0.0);   // bytes added once the ranks are known
                HIF_CUDA((big_qp_panel<T>(a, ng, max_n, max_m, step, st)));
            }
            HIF_CUDA(cudaMemcpyAsync(hs.data(), a.state, sizeof(BigState) * ng, cudaMemcpyDeviceToHost, st));
            HIF_CUDA(cudaStreamSynchronize(st));
            bool all = true;
            for (const BigState& x : hs) all = all && x.stop;
            if (all) break;
        }
        return;
    }
    for (int j = 0; j < maxk; ++j) {
        {
            ProfRange pr(PROF_BIG_QR, st, 0.0, 0.0);   // bytes added once the ranks are known
            HIF_CUDA((big_qr_step<T>(a, ng, max_n, j, st)));
        }
        if ((j + 1) % 16 == 0) {
            HIF_CUDA(cudaMemcpyAsync(hs.data(), a.state, sizeof(BigState) * ng, cudaMemcpyDeviceToHost, st));
            HIF_CUDA(cudaStreamSynchronize(st));
            bool all = true;
            for (const BigState& x : hs) all = all && x.stop;
            if (all) break;
        }
    }
}

// ID of the large boxes of one sublevel: Y_c materialized in HBM and, when it
// has more rows than columns, reduced to its n x n factor R by a blocked
// unpivoted QR (same ID); then pivoted QR by per-step launches shared by all
// large column groups.
template <typename T>
static void run_big_id(hif_handle h, size_t tau, const std::vector<BoxDesc>& bd, const std::vector<GroupDesc>& gd,
                       const SublevelPlan& p, const std::vector<int>& big_boxes, DevMem& d_boxes, DevMem& d_groups,
                       DevMem& d_cols, DevMem& d_near, DevMem& Tws, DevMem& perm_out, DevMem& k_out,
                       double tol_floor, BigBuffers& B) {
    (void)p;
    const cudaStream_t st = h->st;
    std::vector<BigBox> bbv;
    std::vector<BigGroup> bgv;
    int64_t yoff = 0, voff = 0, roff = 0, max_entries = 0;
    int max_m = 0, max_n = 0, maxk = 0;
    bool split = false;
    for (int bI : big_boxes) {
        const BoxDesc& b = bd[bI];
        BigBox x{};
        x.box = bI;
        x.m = (b.sym ? 1 : 2) * (b.m_near + h->P);
        x.y_off = yoff;
        yoff += (int64_t)x.m * b.n;
        max_entries = std::max(max_entries, (int64_t)(b.m_near + h->P) * b.n);
        if (b.has_sci && h->second_kind && tau > 0) split = true;
        for (int q = 0; q < b.ngroups; ++q) {
            const int64_t gi = b.grp_off + q;
            const GroupDesc& G = gd[gi];
            BigGroup y{};
            y.group = (int)gi;
            y.n = G.n;
            y.m = x.m;
            y.ld = x.m;
            y.need_rho = (h->second_kind && G.has_sci && b.has_sci && tau > 0) ? 1 : 0;
            y.y_off = x.y_off + (int64_t)x.m * G.col0;
            y.vec_off = voff;
            y.row_off = roff;
            voff += G.n;
            roff += x.m;
            max_m = std::max(max_m, x.m);
            max_n = std::max(max_n, G.n);
            maxk = std::max(maxk, std::min(x.m, G.n));
            bgv.push_back(y);
        }
        bbv.push_back(x);
    }
    const int ng = (int)bgv.size();
    upload(B.bb, bbv, st);
    upload(B.bg, bgv, st);
    B.state.ensure(sizeof(BigState) * ng);
    B.YK.ensure(sizeof(T) * std::max<int64_t>(yoff, 1));
    if (split) B.YS.ensure(sizeof(T) * yoff);
    B.vv.ensure(sizeof(double) * 2 * std::max<int64_t>(voff, 1));
    B.vw.ensure(sizeof(double) * 2 * std::max<int64_t>(voff, 1));
    B.vt.ensure(sizeof(double) * 2 * std::max<int64_t>(roff, 1));
    B.est.ensure(sizeof(double) * 2 * ng);
    B.nrm.ensure(sizeof(double) * std::max<int64_t>(voff, 1));
    B.perm.ensure(sizeof(int) * std::max<int64_t>(voff, 1));
    BigArgs a{};
    a.g = geom(h);
    a.sci = scidev(h, (int)tau);
    a.boxes = d_boxes.as<BoxDesc>();
    a.bigboxes = B.bb.as<BigBox>();
    a.cols = d_cols.as<int>();
    a.near = d_near.as<int>();
    a.proxy = h->proxy.as<double>();
    a.P = h->P;
    a.second_kind = h->second_kind;
    a.YK = B.YK.p;
    a.YS = split ? B.YS.p : nullptr;
    a.groups = B.bg.as<BigGroup>();
    a.state = B.state.as<BigState>();
    a.gdesc = d_groups.as<GroupDesc>();
    a.vec_v = B.vv.as<double>();
    a.vec_w = B.vw.as<double>();
    a.vec_t = B.vt.as<double>();
    a.est = B.est.as<double>();
    a.nrm = B.nrm.as<double>();
    a.perm = B.perm.as<int>();
    a.Tws = Tws.p;
    a.perm_out = perm_out.as<int>();
    a.k_out = k_out.as<int>();
    a.eps = h->eps;
    a.tol_floor = tol_floor;
    {
        ProfRange pr(PROF_BIG_YGEN, st, 0.0, (split ? 2.0 : 1.0) * sizeof(T) * (double)yoff);
        HIF_CUDA((big_ygen<T>(a, (int)bbv.size(), max_entries, st)));
    }
    {
        ProfRange pr(PROF_BIG_RHO, st, 0.0, 0.0);
        HIF_CUDA((big_rho<T>(a, ng, max_m, max_n, st)));
        if (split) HIF_CUDA((big_add<T>(B.YK.p, B.YS.p, yoff, st)));
    }
    // Opt-in (HIF_BIG_RFIRST=1): measured slower at present, see k_bigqr.cu.
    if (env_int("HIF_BIG_RFIRST", 0)) {
        // Y_c = Q R for the tall boxes; the groups then work on R's rows
        std::vector<int64_t> qy;
        std::vector<int> qm, qn;
        int qmax_m = 0, qmax_n = 0;
        for (const BigBox& x : bbv) {
            qy.push_back(x.y_off);
            qm.push_back(x.m);
            qn.push_back(bd[x.box].n);
            if (x.m > bd[x.box].n) {
                qmax_m = std::max(qmax_m, x.m);
                qmax_n = std::max(qmax_n, bd[x.box].n);
            }
        }
        if (qmax_n > 0) {
            const int nbx = (int)bbv.size();
            upload(B.q_yoff, qy, st);
            upload(B.q_m, qm, st);
            upload(B.q_n, qn, st);
            B.q_tau.ensure(sizeof(T) * 16 * nbx);
            B.q_G.ensure(sizeof(double) * 16 * 16 * nbx);
            B.q_T.ensure(sizeof(T) * 16 * 16 * nbx);
            B.q_W.ensure(sizeof(T) * 16 * (size_t)qmax_n * nbx);
            BigQRArgs q{};
            q.Y = B.YK.p;
            q.y_off = B.q_yoff.as<int64_t>();
            q.m = B.q_m.as<int>();
            q.n = B.q_n.as<int>();
            q.tau = B.q_tau.p;
            q.G = B.q_G.p;
            q.Tf = B.q_T.p;
            q.W = B.q_W.p;
            q.wld = qmax_n;
            std::vector<int64_t> gpo, wpo;
            int64_t wp_total = 0;
            const size_t gp_total = big_geqrf_partials(qm.data(), qn.data(), nbx, gpo, wpo, &wp_total);
            upload(B.q_gpoff, gpo, st);
            upload(B.q_wpoff, wpo, st);
            B.q_Gp.ensure(sizeof(double) * std::max<size_t>(gp_total, 1));
            B.q_Wp.ensure(sizeof(double) * (size_t)std::max<int64_t>(wp_total, 1));
            q.Gp = B.q_Gp.as<double>();
            q.gp_off = B.q_gpoff.as<int64_t>();
            q.Wp = B.q_Wp.as<double>();
            q.wp_off = B.q_wpoff.as<int64_t>();
            HIF_CUDA((big_geqrf<T>(q, nbx, qmax_m, qmax_n, st)));
            // the tolerances were filled on the device: read the groups back
            // before changing their row counts
            HIF_CUDA(cudaMemcpyAsync(bgv.data(), B.bg.p, sizeof(BigGroup) * bgv.size(), cudaMemcpyDeviceToHost, st));
            HIF_CUDA(cudaStreamSynchronize(st));
            size_t gi = 0;
            maxk = 0;
            for (const BigBox& x : bbv) {
                const int nbox = bd[x.box].n;
                for (int q2 = 0; q2 < bd[x.box].ngroups; ++q2, ++gi) {
                    if (x.m > nbox) bgv[gi].m = nbox;
                    maxk = std::max(maxk, std::min(bgv[gi].m, bgv[gi].n));
                }
            }
            upload(B.bg, bgv, st);
        }
    }
    run_big_pivoted_qr<T>(a, B, bgv, max_n, maxk, voff, st);
    ProfRange pr(PROF_BIG_T, st, 0.0, 0.0);
    HIF_CUDA((big_finish<T>(a, ng, max_n, st)));
}

template <typename T>
static void launch_elims(hif_handle h, SubFactor& sf, const std::vector<ElimDesc>& ed,
                         const std::vector<ElimDesc>& ed_big, const std::vector<ElimGroup>& eg,
                         const std::vector<int>& skv, const std::vector<int>& rdv, int64_t fac_off, int64_t piv_off,
                         int64_t ws_off, void* sci_pool, int nsub_sci, DevMem& Tws, FactorScratch& S,
                         const double* work) {
    const cudaStream_t st = h->st;
    upload(S.d_ed, ed, st);
    upload(S.d_eg, eg, st);
    upload(sf.sk, skv, st);
    upload(sf.rd, rdv, st);
    S.ews.ensure(sizeof(T) * std::max<int64_t>(ws_off, 1));
    sf.pool.ensure(sizeof(T) * std::max<int64_t>(fac_off, 1));
    sf.perm.ensure(sizeof(int) * std::max<int64_t>(piv_off, 1));
    S.piv.ensure(sizeof(int) * std::max<int64_t>(piv_off, 1));
    upload(sf.boxes, sf.hbox, st);
    Tws.ensure(sizeof(T));
    ElimArgs ea{};
    ea.g = geom(h);
    ea.sci = scidev(h, nsub_sci);
    ea.boxes = S.d_ed.as<ElimDesc>();
    ea.groups = S.d_eg.as<ElimGroup>();
    ea.sk_ids = sf.sk.as<int>();
    ea.rd_ids = sf.rd.as<int>();
    ea.Tws = Tws.p;
    ea.ws = S.ews.p;
    ea.fac_pool = sf.pool.p;
    ea.piv_pool = S.piv.as<int>();
    ea.perm_pool = sf.perm.as<int>();
    ea.sci_pool = sci_pool;
    ea.status = h->status.as<int>();
    S.ldl_fail.ensure(sizeof(int) * std::max<size_t>(ed.size(), 1));
    HIF_CUDA(cudaMemsetAsync(S.ldl_fail.p, 0, sizeof(int) * std::max<size_t>(ed.size(), 1), st));
    ea.ldl_fail = S.ldl_fail.as<int>();
    // HIF_LDL_TEST_ALPHA (tests only): a larger acceptance constant, so that
    // the LU fallback of LDL boxes can be exercised on any problem
    ea.ldl_alpha = (1.0 + std::sqrt(17.0)) / 8.0;
    if (const char* v = std::getenv("HIF_LDL_TEST_ALPHA")) ea.ldl_alpha = std::atof(v);
    // work list of the persistent launch: boxes by (k + r)^3 descending
    {
        std::vector<int> order(ed.size());
        for (size_t q = 0; q < ed.size(); ++q) order[q] = (int)q;
        std::stable_sort(order.begin(), order.end(), [&](int u, int v) {
            return ed[u].k + ed[u].r > ed[v].k + ed[v].r;
        });
        upload(S.elim_order, order, st);
        S.elim_next.ensure(sizeof(int));
        ea.order = S.elim_order.as<int>();
        ea.nitems = (int)ed.size();
        ea.next_item = S.elim_next.as<int>();
    }
    {
        ProfRange pr(PROF_ELIM, st, work[0], 0.0);
        HIF_CUDA((launch_elim<T>(ea, (int)ed.size(), h->num_sms, st)));
    }
    if (!ed_big.empty()) {
        upload(S.d_ed_big, ed_big, st);
        int mxn = 0, mxk = 0, mxr = 0;
        for (const ElimDesc& eb : ed_big) {
            mxn = std::max(mxn, eb.k + eb.r);
            mxk = std::max(mxk, eb.k);
            mxr = std::max(mxr, eb.r);
        }
        BatchElimArgs ba{};
        ba.g = ea.g;
        ba.sci = ea.sci;
        ba.ed = S.d_ed_big.as<ElimDesc>();
        ba.nbox = (int)ed_big.size();
        ba.groups = S.d_eg.as<ElimGroup>();
        ba.sk = sf.sk.as<int>();
        ba.rd = sf.rd.as<int>();
        ba.Tws = Tws.p;
        ba.ws = S.ews.p;
        ba.pool = sf.pool.p;
        ba.piv = S.piv.as<int>();
        ba.perm = sf.perm.as<int>();
        ba.sci_pool = sci_pool;
        ba.status = h->status.as<int>();
        // HIF_TC_GEMM=1: the products on the tensor cores (hif_gemm_batched_f32).
        // Off by default: the tensor core's FP32 accumulation of the long
        // products (K = k or r) is less accurate than the SIMT FMA chains, and
        // at N = 1M the FP32 factor's refinement contraction went from ~1e-3
        // to ~4e-3 per step (one refinement step more), for no gain in time.
        if (env_int("HIF_TC_GEMM", 0)) {
            S.gemm_probs.ensure(sizeof(TcGemmProb) * 5 * ed_big.size());
            ba.gemm_probs = S.gemm_probs.p;
        }
        ProfRange pr(PROF_BIG_ELIM, st, work[1], 0.0);
        HIF_CUDA((big_elim_batch<T>(ba, mxn, mxk, mxr, st)));
    }
}

// Factor offsets of one eliminated box inside its sublevel's pools.  An LDL
// box (symmetric A, Sec. 5) keeps T, L (with L^{-1} packed in the same r x r
// array), D and X; Y = X^T and U = L^T P are not stored.
static void place_box(ElimDesc& e, BoxFac& bf, int k, int r, bool ldl, int64_t& fac_off, int64_t& piv_off,
                      int64_t& ws_off) {
    const int n = k + r;
    e.k = k;
    e.r = r;
    e.ldl = ldl ? 1 : 0;
    e.ws_off = ws_off;
    ws_off += (int64_t)n * n + (int64_t)k * r;
    e.T_out = fac_off; fac_off += (int64_t)k * r;
    e.LU_out = fac_off; fac_off += (int64_t)r * r;
    if (ldl) e.LUi_out = e.LU_out;
    else { e.LUi_out = fac_off; fac_off += (int64_t)r * r; }
    e.D_out = fac_off; fac_off += r;
    e.X_out = fac_off; fac_off += (int64_t)k * r;
    if (ldl) e.Y_out = e.X_out;
    else { e.Y_out = fac_off; fac_off += (int64_t)r * k; }
    e.piv_out = piv_off; piv_off += r;
    bf.k = k;
    bf.r = r;
    bf.ldl = e.ldl;
    bf.sk_off = e.sk_off;
    bf.rd_off = e.rd_off;
    bf.T_off = e.T_out;
    bf.LU_off = e.LU_out;
    bf.LUi_off = e.LUi_out;
    bf.D_off = e.D_out;
    bf.X_off = e.X_out;
    bf.Y_off = e.Y_out;
    bf.piv_off = e.piv_out;
}

// ID of the large boxes that the fold kernel reduced to their n x n factor R
// (the ID of R[:, g] is that of Y_c[:, g]): R in column-major order, rho_g
// from the box Grams, then the pivoted QR by per-step launches shared by all
// such groups, on the col0 + n_g rows of R[:, g] that can be nonzero.
template <typename T>
static void run_big_id_R(hif_handle h, const std::vector<BoxDesc>& bd, const std::vector<GroupDesc>& gd,
                         const std::vector<int>& boxes, DevMem& d_boxes, DevMem& d_groups, DevMem& Rws, void* GK,
                         void* GS, DevMem& Tws, DevMem& perm_out, DevMem& k_out, double tol_floor, BigBuffers& B) {
    const cudaStream_t st = h->st;
    std::vector<BigGroup> bgv;
    std::vector<int64_t> roff;
    int64_t yoff = 0, voff = 0;
    int max_n = 0, maxk = 0, max_ng = 0;
    for (int bI : boxes) {
        const BoxDesc& b = bd[bI];
        roff.push_back(yoff);
        for (int q = 0; q < b.ngroups; ++q) {
            const int64_t gi = b.grp_off + q;
            const GroupDesc& G = gd[gi];
            BigGroup y{};
            y.group = (int)gi;
            y.n = G.n;
            y.m = G.col0 + G.n;
            y.ld = b.n;
            y.need_rho = (h->second_kind && G.has_sci && b.has_sci && GK) ? 1 : 0;
            y.y_off = yoff + (int64_t)b.n * G.col0;
            y.vec_off = voff;
            y.row_off = 0;
            voff += G.n;
            max_n = std::max(max_n, G.n);
            max_ng = std::max(max_ng, G.n);
            maxk = std::max(maxk, std::min(y.m, G.n));
            bgv.push_back(y);
        }
        yoff += (int64_t)b.n * b.n;
    }
    const int ng = (int)bgv.size();
    upload(B.bg, bgv, st);
    B.state.ensure(sizeof(BigState) * ng);
    B.YK.ensure(sizeof(T) * std::max<int64_t>(yoff, 1));
    B.nrm.ensure(sizeof(double) * std::max<int64_t>(voff, 1));
    B.perm.ensure(sizeof(int) * std::max<int64_t>(voff, 1));
    for (size_t q = 0; q < boxes.size(); ++q) {
        const BoxDesc& b = bd[boxes[q]];
        HIF_CUDA((launch_r_colmajor<T>(Rws.as<T>() + b.R_off, b.n, B.YK.as<T>() + roff[q], st)));
    }
    GramTolArgs ga{};
    ga.groups = B.bg.as<BigGroup>();
    ga.gdesc = d_groups.as<GroupDesc>();
    ga.boxes = d_boxes.as<BoxDesc>();
    ga.GKws = GK;
    ga.GSws = GS;
    ga.eps = h->eps;
    ga.tol_floor = tol_floor;
    HIF_CUDA((launch_gram_tol<T>(ga, ng, max_ng, st)));
    BigArgs a{};
    a.groups = B.bg.as<BigGroup>();
    a.state = B.state.as<BigState>();
    a.gdesc = d_groups.as<GroupDesc>();
    a.YK = B.YK.p;
    a.nrm = B.nrm.as<double>();
    a.perm = B.perm.as<int>();
    a.Tws = Tws.p;
    a.perm_out = perm_out.as<int>();
    a.k_out = k_out.as<int>();
    run_big_pivoted_qr<T>(a, B, bgv, max_n, maxk, voff, st);
    ProfRange pr(PROF_BIG_T, st, 0.0, 0.0);
    HIF_CUDA((big_finish<T>(a, ng, max_n, st)));
}

// The eliminations of one sublevel (or of the top blocks): boxes in factor
// order, each in the one-CTA list (ed) or the batched multi-CTA list
// (ed_big).  Places every box in the sublevel's pools, launches, and, if an
// LDL box met a pivot that fails the 1 x 1 test, gives that box the LU form
// and runs the sublevel's eliminations once more (every box recomputes its
// block from the unchanged inputs, so the others are reproduced exactly).
struct ElimPlan {
    std::vector<ElimDesc> ed, ed_big;
    std::vector<std::pair<bool, int>> where;   // per factor box: (in ed_big, index)
    std::vector<ElimGroup> eg;
    std::vector<int> skv, rdv;
    double work[2] = {0.0, 0.0};
    void add(const ElimDesc& e, bool big, double flops) {
        where.push_back({big, (int)(big ? ed_big.size() : ed.size())});
        (big ? ed_big : ed).push_back(e);
        work[big ? 1 : 0] += flops;
    }
};

template <typename T>
static void launch_elims(hif_handle h, SubFactor& sf, const std::vector<ElimDesc>& ed,
                         const std::vector<ElimDesc>& ed_big, const std::vector<ElimGroup>& eg,
                         const std::vector<int>& skv, const std::vector<int>& rdv, int64_t fac_off, int64_t piv_off,
                         int64_t ws_off, void* sci_pool, int nsub_sci, DevMem& Tws, FactorScratch& S,
                         const double* work);

template <typename T>
struct Eliminator {
    hif_handle h;
    SubFactor& sf;
    ElimPlan& ep;
    void* sci_pool;
    int nsub_sci;
    DevMem& Tws;
    FactorScratch& S;
    int64_t fac_off = 0, piv_off = 0;

    void place_and_launch() {
        int64_t ws_off = 0;
        fac_off = piv_off = 0;
        for (size_t q = 0; q < ep.where.size(); ++q) {
            ElimDesc& e = ep.where[q].first ? ep.ed_big[ep.where[q].second] : ep.ed[ep.where[q].second];
            place_box(e, sf.hbox[q], e.k, e.r, e.ldl != 0, fac_off, piv_off, ws_off);
        }
        launch_elims<T>(h, sf, ep.ed, ep.ed_big, ep.eg, ep.skv, ep.rdv, fac_off, piv_off, ws_off, sci_pool, nsub_sci,
                        Tws, S, ep.work);
    }
    // issues the eliminations and returns without waiting for them
    void launch() { place_and_launch(); }
    // waits for them; an LDL box whose pivot failed the 1 x 1 test takes the
    // LU form and the eliminations run once more (every box recomputes its
    // block from the unchanged inputs, so the others are reproduced exactly)
    void finish() {
        for (int attempt = 0; attempt < 2; ++attempt) {
            bool any_ldl = false;
            for (const ElimDesc& e : ep.ed) any_ldl = any_ldl || e.ldl;
            int stw = 0;
            if (any_ldl) HIF_CUDA(cudaMemcpyAsync(&stw, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, h->st));
            HIF_CUDA(cudaStreamSynchronize(h->st));
            if (!(stw & DEV_LDL_FALLBACK)) break;
            if (attempt == 1) fail(HIF_ENUMERIC, "LDL fallback repeated");
            std::vector<int> failed(ep.ed.size());
            HIF_CUDA(cudaMemcpyAsync(failed.data(), S.ldl_fail.p, sizeof(int) * failed.size(),
                                     cudaMemcpyDeviceToHost, h->st));
            stw &= ~(int)DEV_LDL_FALLBACK;
            HIF_CUDA(cudaMemcpyAsync(h->status.p, &stw, sizeof(int), cudaMemcpyHostToDevice, h->st));
            HIF_CUDA(cudaStreamSynchronize(h->st));
            for (size_t q = 0; q < failed.size(); ++q)
                if (failed[q]) ep.ed[q].ldl = 0;
            h->stats.ldl_fallbacks += (int64_t)std::count(failed.begin(), failed.end(), 1);
            place_and_launch();
        }
        h->stats.factor_bytes += (int64_t)(fac_off * sizeof(T) + piv_off * sizeof(int));
        for (const ElimDesc& e : ep.ed) h->stats.ldl_boxes += e.ldl ? 1 : 0;
    }
};


template <typename T>
static void run_factor(hif_handle h) {
    const cudaStream_t st = h->st;
    const int d = h->dim;
    const int64_t N = h->N;
    const GeomDev g = geom(h);
    size_t nsub = 0;
    int maxL = 0;
    for (auto& sp : h->segs) {
        Segment& sg = *sp;
        Tree& t = sg.tree;
        t.dim = d;
        const double* xs = h->hx.data() + (size_t)d * sg.off;
        const double* wsg = h->hw.data() + sg.off;
        if (h->opt.root_width > 0) {
            for (int k = 0; k < 3; ++k) t.lo[k] = h->opt.root_lo[k];
            t.W = h->opt.root_width;
        } else {
            root_box(xs, wsg, sg.N, d, t.lo, &t.W);
        }
        t.L = num_levels(xs, sg.N, d, t.lo, t.W, h->opt.leaf_occupancy);
        plan_sublevels(d, t.L, h->opt.fractional_levels != 0, h->opt.skip_levels, sg.kinds, sg.levels);
        nsub = std::max(nsub, sg.kinds.size());
        maxL = std::max(maxL, t.L);
    }
    if ((int)nsub + 1 > kMaxSub) fail(HIF_EINVAL, "too many sublevels");

    h->sci_blk.ensure(sizeof(int) * (size_t)kMaxSub * N);
    h->sci_loc.ensure(sizeof(int) * (size_t)kMaxSub * N);
    HIF_CUDA(cudaMemsetAsync(h->sci_blk.p, 0xff, sizeof(int) * (size_t)kMaxSub * N, st));
    HIF_CUDA(cudaMemsetAsync(h->sci_loc.p, 0, sizeof(int) * (size_t)kMaxSub * N, st));
    h->status.ensure(sizeof(int));
    HIF_CUDA(cudaMemsetAsync(h->status.p, 0, sizeof(int), st));

    SciHost sci;
    std::vector<char> active(N, 1);
    std::vector<int> box_of(N, -1);
    DevMem d_boxes, d_groups, d_cols, d_near, Rws, GKws, GSws, Tws, Wws, Woff, perm_out, k_out;
    DevMem d_small_boxes, d_small_groups, d_small_sorted, id_counter;
    FactorScratch S;
    BigBuffers big, bigR;
    const int big_id_n = env_int("HIF_BIG_ID", sizeof(T) == 8 ? 128 : 256);
    // HIF_FOLD_BIG=1: large FP32 boxes up to 1024 columns are folded to R by
    // one CTA each and take their pivoted QR on R.  Off by default: with one
    // CTA per box the few-box sublevels near the top of the tree serialize
    // (measured 2.6 s against 1.2 s for the FP32 factorization at n = 1024).
    const bool fold_big = sizeof(T) == 4 && env_int("HIF_FOLD_BIG", 0) != 0;
    // boxes with k + r above this are eliminated by the batched multi-CTA
    // kernels instead of one CTA per box (measured on GB300 for the n = 1024
    // grid: 400 beats 600 by 15% in FP32 and 5% in FP64)
    const int big_elim_n = env_int("HIF_BIG_ELIM", 400);
    const bool trace = env_int("HIF_TRACE", 0) != 0;
    if (trace) geometry_trace(true, nullptr);
    double flops = 0, evals = 0;
    const double tol_floor = sizeof(T) == 4 ? h->opt.fp32_tol_floor : 0.0;

    // ---- index sets of one sublevel, problem by problem, merged (host work;
    // the plan of sublevel tau + 1 is made while the GPU eliminates tau)
    struct Planned {
        SublevelPlan p;
        std::vector<double> radius;
        std::vector<int> symv;
        int kind = -1, ell = -1;
        double ms_partition = 0, ms_near = 0;    // host time (trace)
    };
    NearCache near_cache;                    // mark arrays reused by every sublevel's plan
    auto plan_sublevel = [&](size_t tau, Planned& P) {
        SublevelPlan& p = P.p;
        std::vector<double>& radius = P.radius;
        std::vector<int>& symv = P.symv;
        int& kind = P.kind;
        int& ell = P.ell;
        p.nbox = 0;
        p.box_off.assign(1, 0);
        p.near_off.assign(1, 0);
        p.grp_off.assign(1, 0);
        for (auto& sp : h->segs) {
            Segment& sg = *sp;
            if (tau >= sg.kinds.size()) continue;
            const int kd = sg.kinds[tau], lv = sg.levels[tau];
            if (kind < 0) { kind = kd; ell = lv; }
            const int s = 1 << (sg.tree.L - lv);
            const double wl = sg.tree.W / s;
            std::vector<int> act_ids;
            act_ids.reserve(sg.N);
            for (int64_t i = sg.off; i < sg.off + sg.N; ++i)
                if (active[i]) act_ids.push_back((int)i);
            for (int i : act_ids) box_of[i] = -1;
            SublevelPlan ps;
            const auto q0 = std::chrono::steady_clock::now();
            partition(sg.tree, h->hx.data(), kd, s, act_ids, ps, box_of);
            const auto q1 = std::chrono::steady_clock::now();
            build_near_groups(sg.tree, h->hx.data(), s, h->opt.proxy_radius, h->second_kind, act_ids, active, box_of,
                              sci, ps, &near_cache);
            const auto q2 = std::chrono::steady_clock::now();
            P.ms_partition += std::chrono::duration<double, std::milli>(q1 - q0).count();
            P.ms_near += std::chrono::duration<double, std::milli>(q2 - q1).count();
            const int nb_seg = ps.nbox;
            append_plan(p, std::move(ps));
            radius.insert(radius.end(), nb_seg, h->opt.proxy_radius * wl);
            symv.insert(symv.end(), nb_seg, sg.sym ? 1 : 0);
        }
    };
    Planned next;
    if (nsub > 0) plan_sublevel(0, next);
    for (size_t tau = 0; tau < nsub; ++tau) {
        const auto tr0 = std::chrono::steady_clock::now();
        auto tr_fold = tr0;
        Planned cur = std::move(next);
        next = Planned();
        SublevelPlan& p = cur.p;
        const std::vector<double>& radius = cur.radius;
        const std::vector<int>& symv = cur.symv;
        const int kind = cur.kind, ell = cur.ell;
        const int nb = p.nbox;
        const int64_t ngr = p.grp_off[nb];

        // ---- descriptors for the fold and ID launches
        std::vector<BoxDesc> bd(nb);
        std::vector<GroupDesc> gd(ngr);
        int64_t Roff = 0, Toff = 0, Woffs = 0;
        int maxn = 0, maxng = 0, maxmrow = 0;
        bool any_sci = false;
        std::vector<int64_t> woff(ngr);
        std::vector<int> small_boxes, small_groups, big_boxes, rbig_boxes;
        std::vector<char> box_class(nb, 0);   // 0 small, 1 folded large, 2 materialized large
        double fold_flops = 0.0;
        for (int bI = 0; bI < nb; ++bI) {
            BoxDesc& b = bd[bI];
            const int nbI = (int)(p.box_off[bI + 1] - p.box_off[bI]);
            // large boxes whose proxy matrix the fold kernel can still reduce
            // to R (FP32, up to 1024 columns) take their pivoted QR on R
            const bool folded = nbI > big_id_n && fold_big && fold_cpt(nbI, (int)sizeof(T)) > 0;
            const bool isbig = nbI > big_id_n && !folded;
            box_class[bI] = isbig ? 2 : folded ? 1 : 0;
            b.n = (int)(p.box_off[bI + 1] - p.box_off[bI]);
            b.m_near = (int)(p.near_off[bI + 1] - p.near_off[bI]);
            b.ngroups = (int)(p.grp_off[bI + 1] - p.grp_off[bI]);
            b.has_sci = p.box_sci[bI];
            b.sym = symv[bI];
            b.col_off = p.box_off[bI];
            b.near_off = p.near_off[bI];
            b.grp_off = p.grp_off[bI];
            b.R_off = Roff;
            if (!isbig) Roff += (int64_t)b.n * b.n;
            for (int k = 0; k < 3; ++k) b.ctr[k] = p.centers[3 * bI + k];
            b.radius = radius[bI];
            if (isbig) big_boxes.push_back(bI);
            else {
                small_boxes.push_back(bI);          // every folded box
                if (folded) rbig_boxes.push_back(bI);
                maxn = std::max(maxn, b.n);
                if (b.has_sci) any_sci = true;
            }
            const double m = (b.sym ? 1.0 : 2.0) * (b.m_near + h->P);
            h->stats.proxy_rows += (int64_t)m;
            evals += (double)(b.m_near + h->P) * b.n;
            flops += 2.0 * m * b.n * b.n;
            if (!isbig) fold_flops += 2.0 * m * b.n * b.n;
            for (int q = 0; q < b.ngroups; ++q) {
                const int64_t gi = b.grp_off + q;
                GroupDesc& G = gd[gi];
                G.box = bI;
                G.col0 = p.grp_col0[gi];
                G.n = p.grp_n[gi];
                G.has_sci = p.grp_sci[gi];
                G.T_off = Toff;
                Toff += (int64_t)G.n * G.n;
                G.perm_off = b.col_off + G.col0;
                const int mrow = G.col0 + G.n;
                woff[gi] = Woffs;
                if (!isbig && !folded) {
                    small_groups.push_back((int)gi);
                    Woffs += (int64_t)(mrow | 1) * G.n;
                    maxng = std::max(maxng, G.n);
                    maxmrow = std::max(maxmrow, mrow);
                }
            }
        }
        upload(d_boxes, bd, st);
        upload(d_groups, gd, st);
        upload(d_cols, p.cols, st);
        upload(d_near, p.near, st);
        upload(Woff, woff, st);
        upload(d_small_boxes, small_boxes, st);
        // the small boxes by width, for the fold launches
        std::vector<int> small_sorted(small_boxes);
        std::stable_sort(small_sorted.begin(), small_sorted.end(),
                         [&](int x, int y) { return bd[x].n < bd[y].n; });
        upload(d_small_sorted, small_sorted, st);
        // the ID's work items, largest first (a persistent launch takes them in order)
        std::stable_sort(small_groups.begin(), small_groups.end(), [&](int x, int y) {
            const double wx = (double)(gd[x].col0 + gd[x].n) * gd[x].n * gd[x].n;
            const double wy = (double)(gd[y].col0 + gd[y].n) * gd[y].n * gd[y].n;
            return wx > wy;
        });
        upload(d_small_groups, small_groups, st);
        Rws.ensure(sizeof(T) * std::max<int64_t>(Roff, 1));
        const bool grams = h->second_kind && any_sci;
        if (grams) {
            GKws.ensure(sizeof(T) * Roff);
            GSws.ensure(sizeof(T) * Roff);
        }
        Tws.ensure(sizeof(T) * std::max<int64_t>(Toff, 1));
        perm_out.ensure(sizeof(int) * std::max<size_t>(p.cols.size(), 1));
        k_out.ensure(sizeof(int) * std::max<int64_t>(ngr, 1));

        if (!small_boxes.empty()) {
            FoldArgs fa{};
            fa.g = g;
            fa.sci = scidev(h, (int)tau);
            fa.boxes = d_boxes.as<BoxDesc>();
            fa.box_list = d_small_boxes.as<int>();
            fa.cols = d_cols.as<int>();
            fa.near = d_near.as<int>();
            fa.groups = d_groups.as<GroupDesc>();
            fa.proxy = h->proxy.as<double>();
            fa.P = h->P;
            fa.bpairs = 16;
            fa.second_kind = h->second_kind;
            fa.Rws = Rws.p;
            fa.GKws = grams ? GKws.p : nullptr;
            fa.GSws = grams ? GSws.p : nullptr;
            {
                // one launch per width bucket: a thread per column, so the
                // CTA is the box width rounded up to a warp.  The buckets of
                // a sublevel run concurrently on streams forked from the
                // handle's; the rows per chunk of each one-column-per-thread
                // bucket are autotuned once per process (and precision, width)
                ProfRange pr(PROF_FOLD, st, fold_flops, 0.0);
                struct Bucket { FoldArgs fa; int count, w, cpt, rc; size_t smem; };
                std::vector<Bucket> buckets;
                int64_t at = 0;
                const int widths[] = {32, 64, 96, 128, 160, 192, 224, 256, 512, 1024};
                for (int w : widths) {
                    if (at >= (int64_t)small_boxes.size()) break;
                    const int64_t b0 = at;
                    while (at < (int64_t)small_boxes.size() && bd[small_sorted[at]].n <= w) ++at;
                    if (at == b0) continue;
                    const int cpt = fold_cpt(w, (int)sizeof(T));
                    if (cpt == 0) fail(HIF_EINVAL, "box too wide for the fold kernel");
                    Bucket bk{fa, (int)(at - b0), w, cpt, 0, 0};
                    bk.fa.box_list = d_small_sorted.as<int>() + b0;
                    bk.smem = fold_smem_bytes(w, cpt, grams, true, sizeof(T));
                    bk.fa.R_in_smem = bk.smem <= 220 * 1024;
                    if (!bk.fa.R_in_smem) bk.smem = fold_smem_bytes(w, cpt, grams, false, sizeof(T));
                    if (bk.smem > 220 * 1024) fail(HIF_EINVAL, "box too large for the fold kernel");
                    buckets.push_back(bk);
                }
                if (at != (int64_t)small_boxes.size()) fail(HIF_EINVAL, "box too wide for the fold kernel");
                // autotune (synchronous, first sighting of a bucket only)
                std::vector<char> done(buckets.size(), 0);
                for (size_t q = 0; q < buckets.size(); ++q) {
                    Bucket& bk = buckets[q];
                    if (bk.cpt != 1) continue;
                    const int key = bk.w * 16 + (int)sizeof(T);
                    if (h->opt.autotune && sizeof(T) == 4) {
                        std::lock_guard<std::mutex> lk(g_fold_rc_mu);
                        auto it = g_fold_rc.find(key);
                        if (it != g_fold_rc.end()) { bk.rc = it->second; continue; }
                    }
                    // (FP64 keeps 32 rows so that its rounding never depends on a timing)
                    if (!h->opt.autotune || sizeof(T) == 8) { bk.rc = 32; continue; }
                    cudaEvent_t e0, e1;
                    HIF_CUDA(cudaEventCreate(&e0));
                    HIF_CUDA(cudaEventCreate(&e1));
                    float t16 = 0.f, t32 = 0.f;
                    for (int rc : {16, 32}) {
                        HIF_CUDA(cudaEventRecord(e0, st));
                        HIF_CUDA((launch_fold<T>(bk.fa, bk.count, bk.w, 1, bk.smem, st, rc)));
                        HIF_CUDA(cudaEventRecord(e1, st));
                        HIF_CUDA(cudaEventSynchronize(e1));
                        HIF_CUDA(cudaEventElapsedTime(rc == 16 ? &t16 : &t32, e0, e1));
                    }
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    // 16 rows only on a clear win: the choice changes the FP32
                    // rounding of R, so it should not follow timing noise
                    bk.rc = t16 < 0.85f * t32 ? 16 : 32;
                    if (env_int("HIF_TRACE", 0))
                        std::fprintf(stderr, "[hif] fold autotune width %d: 16 rows %.3f ms, 32 rows %.3f ms -> %d\n",
                                     bk.w, t16, t32, bk.rc);
                    // the bucket's R must come from the kept variant
                    if (bk.rc == 16) HIF_CUDA((launch_fold<T>(bk.fa, bk.count, bk.w, 1, bk.smem, st, 16)));
                    done[q] = 1;
                    std::lock_guard<std::mutex> lk(g_fold_rc_mu);
                    g_fold_rc[key] = bk.rc;
                }
                std::vector<size_t> todo;
                for (size_t q = 0; q < buckets.size(); ++q)
                    if (!done[q]) todo.push_back(q);
                if (todo.size() <= 1) {
                    for (size_t q : todo) {
                        const Bucket& bk = buckets[q];
                        HIF_CUDA((launch_fold<T>(bk.fa, bk.count, bk.cpt == 1 ? bk.w : 256, bk.cpt, bk.smem, st,
                                                 bk.rc)));
                    }
                } else {
                    HIF_CUDA(cudaEventRecord(h->fork_ev(), st));
                    for (size_t i = 0; i < todo.size(); ++i) {
                        const Bucket& bk = buckets[todo[i]];
                        cudaStream_t s2 = h->aux_stream(i);
                        HIF_CUDA(cudaStreamWaitEvent(s2, h->fork_ev(), 0));
                        HIF_CUDA((launch_fold<T>(bk.fa, bk.count, bk.cpt == 1 ? bk.w : 256, bk.cpt, bk.smem, s2,
                                                 bk.rc)));
                        HIF_CUDA(cudaEventRecord(h->join_ev(i), s2));
                    }
                    for (size_t i = 0; i < todo.size(); ++i) HIF_CUDA(cudaStreamWaitEvent(st, h->join_ev(i), 0));
                }
            }
            if (trace) {
                HIF_CUDA(cudaStreamSynchronize(st));
                tr_fold = std::chrono::steady_clock::now();
            }

            IdArgs ia{};
            ia.groups = d_groups.as<GroupDesc>();
            ia.group_list = d_small_groups.as<int>();
            ia.nitems = (int)small_groups.size();
            id_counter.ensure(sizeof(int));
            ia.next_item = id_counter.as<int>();
            ia.boxes = d_boxes.as<BoxDesc>();
            ia.Rws = Rws.p;
            ia.GKws = grams ? GKws.p : nullptr;
            ia.GSws = grams ? GSws.p : nullptr;
            ia.second_kind = h->second_kind;
            ia.Tws = Tws.p;
            ia.perm_out = perm_out.as<int>();
            ia.k_out = k_out.as<int>();
            ia.eps = h->eps;
            ia.tol_floor = tol_floor;
            size_t ismem = id_smem_bytes(maxng, maxmrow, true, sizeof(T));
            ia.W_in_smem = ismem <= 200 * 1024;
            if (!ia.W_in_smem) {
                Wws.ensure(sizeof(T) * std::max<int64_t>(Woffs, 1));
                ismem = id_smem_bytes(maxng, maxmrow, false, sizeof(T));
            }
            ia.Wws = Wws.p;
            ia.W_off = Woff.as<int64_t>();
            {
                ProfRange pr(PROF_ID, st, 0.0, 0.0);     // work added once the ranks are known
                HIF_CUDA((launch_id<T>(ia, (int)small_groups.size(), ismem, h->num_sms, st)));
            }
            if (!rbig_boxes.empty())
                run_big_id_R<T>(h, bd, gd, rbig_boxes, d_boxes, d_groups, Rws, grams ? GKws.p : nullptr,
                                grams ? GSws.p : nullptr, Tws, perm_out, k_out, tol_floor, bigR);
        }
        if (!big_boxes.empty()) run_big_id<T>(h, tau, bd, gd, p, big_boxes, d_boxes, d_groups, d_cols, d_near, Tws,
                                              perm_out, k_out, tol_floor, big);

        const auto tr1 = std::chrono::steady_clock::now();
        std::vector<int> kg(ngr), permh(p.cols.size());
        if (ngr) HIF_CUDA(cudaMemcpyAsync(kg.data(), k_out.p, sizeof(int) * ngr, cudaMemcpyDeviceToHost, st));
        if (!permh.empty())
            HIF_CUDA(cudaMemcpyAsync(permh.data(), perm_out.p, sizeof(int) * permh.size(), cudaMemcpyDeviceToHost, st));
        HIF_CUDA(cudaStreamSynchronize(st));
        const auto tr2 = std::chrono::steady_clock::now();
        if (prof_enabled()) {
            // pivoted QR to rank k of an mrow x ng block plus T = R1^{-1} R2;
            // large groups: one read + write of the remaining columns per step
            double idf = 0.0, qr_bytes = 0.0;
            for (int64_t gi = 0; gi < ngr; ++gi) {
                const GroupDesc& G = gd[gi];
                const BoxDesc& b = bd[G.box];
                const double k = kg[gi], n = G.n, r = n - k;
                const int cls = box_class[G.box];
                if (cls == 0) {
                    const double mr = G.col0 + G.n;
                    idf += 4.0 * mr * n * k - 2.0 * k * k * (mr + n) + 4.0 * k * k * k / 3.0 + k * k * r;
                } else if (cls == 1) {
                    const double mr = G.col0 + G.n;
                    for (int j = 0; j < kg[gi]; ++j) qr_bytes += 2.0 * sizeof(T) * (mr - j) * (n - j);
                } else {
                    const double m = (b.sym ? 1.0 : 2.0) * (b.m_near + h->P);
                    for (int j = 0; j < kg[gi]; ++j) qr_bytes += 2.0 * sizeof(T) * m * (n - j);
                }
            }
            prof_add_work(PROF_ID, idf, 0.0);
            prof_add_work(PROF_BIG_QR, 0.0, qr_bytes);
        }

        // ---- skeleton / redundant sets, elimination descriptors
        auto sf = std::make_unique<SubFactor>();
        sf->kind = kind;
        sf->level = ell;
        ElimPlan ep;
        std::vector<ElimGroup>& eg = ep.eg;
        std::vector<int>& skv = ep.skv;
        std::vector<int>& rdv = ep.rdv;
        int64_t sci_off = 0;
        struct NewBlock { int box; int64_t sk_off; int k; int64_t sci_off; };
        std::vector<NewBlock> nblk;
        int64_t ksum = 0, rsum = 0;
        int maxbox = 0;
        for (int bI = 0; bI < nb; ++bI) {
            const BoxDesc& b = bd[bI];
            maxbox = std::max(maxbox, b.n);
            int k = 0, r = 0;
            for (int q = 0; q < b.ngroups; ++q) {
                k += kg[b.grp_off + q];
                r += gd[b.grp_off + q].n - kg[b.grp_off + q];
            }
            ksum += k;
            rsum += r;
            if (r == 0) continue;
            ElimDesc e{};
            e.ngroups = b.ngroups;
            e.sk_off = (int64_t)skv.size();
            e.rd_off = (int64_t)rdv.size();
            e.grp_off = (int64_t)eg.size();
            int ko = 0, ro = 0;
            for (int q = 0; q < b.ngroups; ++q) {
                const GroupDesc& G = gd[b.grp_off + q];
                const int kq = kg[b.grp_off + q];
                for (int l = 0; l < kq; ++l) skv.push_back(p.cols[b.col_off + G.col0 + permh[G.perm_off + l]]);
                ElimGroup E{};
                E.kg = kq;
                E.rg = G.n - kq;
                E.ko = ko;
                E.ro = ro;
                E.T_off = G.T_off;
                eg.push_back(E);
                ko += kq;
                ro += G.n - kq;
            }
            for (int q = 0; q < b.ngroups; ++q) {
                const GroupDesc& G = gd[b.grp_off + q];
                const int kq = kg[b.grp_off + q];
                for (int l = kq; l < G.n; ++l) rdv.push_back(p.cols[b.col_off + G.col0 + permh[G.perm_off + l]]);
            }
            e.k = k;
            e.r = r;
            const bool big = k + r > big_elim_n;
            // LDL for symmetric problems (Sec. 5) on the one-CTA path
            e.ldl = (h->opt.ldl && b.sym && !big) ? 1 : 0;
            if (k > 0) {
                e.sci_out = sci_off;
                nblk.push_back({bI, e.sk_off, k, sci_off});
                sci_off += (int64_t)k * k;
            } else {
                e.sci_out = -1;
            }
            BoxFac bf{};
            sf->hbox.push_back(bf);
            sf->max_kr2 = std::max(sf->max_kr2, k + 2 * r);
            const double kk = k, rr = r;
            const double ef = 2.0 * (kk * kk * rr + 2 * kk * rr * rr + kk * kk * rr) + 2.0 / 3.0 * rr * rr * rr +
                              2.0 * kk * rr * rr + 2.0 * kk * kk * rr;
            flops += ef;
            ep.add(e, big, ef);
        }
        sf->nbox = (int)sf->hbox.size();
        h->stats.kinds[tau] = kind;
        h->stats.boxes[tau] = nb;
        h->stats.skeletons[tau] = ksum;
        h->stats.redundant[tau] = rsum;
        h->stats.max_box[tau] = maxbox;

        // SCI pool of this sublevel and the block table
        auto pool = std::make_unique<DevMem>();
        pool->ensure(sizeof(T) * std::max<int64_t>(sci_off, 1));
        const int first_block = (int)h->blk_k_h.size();
        for (const NewBlock& nbk : nblk) {
            h->blk_ptr_h.push_back(static_cast<char*>(pool->p) + sizeof(T) * nbk.sci_off);
            h->blk_k_h.push_back(nbk.k);
        }
        Eliminator<T> elim{h, *sf, ep, pool->p, (int)tau, Tws, S};
        if (sf->nbox) elim.launch();
        h->sci_pools.push_back(std::move(pool));

        // ---- state for the next sublevel: active set and SCI membership
        sci.blk.emplace_back(N, -1);
        sci.loc.emplace_back(N, 0);
        std::vector<int>& hb = sci.blk.back();
        std::vector<int>& hl = sci.loc.back();
        for (size_t q = 0; q < nblk.size(); ++q) {
            const NewBlock& nbk = nblk[q];
            std::vector<int> mem(skv.begin() + nbk.sk_off, skv.begin() + nbk.sk_off + nbk.k);
            for (int l = 0; l < nbk.k; ++l) {
                hb[mem[l]] = first_block + (int)q;
                hl[mem[l]] = l;
            }
            sci.members.push_back(std::move(mem));
        }
        for (int i : rdv) active[i] = 0;
        // the next sublevel's plan needs only host state: made while the GPU eliminates
        if (tau + 1 < nsub) plan_sublevel(tau + 1, next);
        const auto tr_plan = std::chrono::steady_clock::now();
        if (sf->nbox) elim.finish();
        HIF_CUDA(cudaStreamSynchronize(st));   // kernels of this sublevel hold the old block table
        HIF_CUDA(cudaMemcpyAsync(h->sci_blk.as<int>() + tau * N, hb.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
        HIF_CUDA(cudaMemcpyAsync(h->sci_loc.as<int>() + tau * N, hl.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
        upload(h->blk_ptr, h->blk_ptr_h, st);
        upload(h->blk_k, h->blk_k_h, st);
        HIF_CUDA(cudaStreamSynchronize(st));
        check_status(h);
        if (trace) {
            const auto tr3 = std::chrono::steady_clock::now();
            auto ms = [](auto a0, auto b0) { return std::chrono::duration<double, std::milli>(b0 - a0).count(); };
            std::fprintf(stderr, "[hif] sub %2zu kind %d level %d boxes %d big %zu maxn %d | launch %.1f ms, id %.1f ms, "
                                 "elim+next plan %.1f ms (plan done at %.1f ms)\n",
                         tau, kind, ell, nb, big_boxes.size(), maxbox, ms(tr0, tr1), ms(tr1, tr2), ms(tr2, tr3),
                         ms(tr2, tr_plan));
            if (!small_boxes.empty())
                std::fprintf(stderr, "[hif]        fold %.1f ms (ends at the sync)\n", ms(tr0, tr_fold));
            if (tau + 1 < nsub) {
                double gm[6];
                geometry_trace(true, gm);
                std::fprintf(stderr, "[hif]        next plan: partition %.1f ms, near fields and groups %.1f ms "
                                     "(bins %.1f, gather %.1f; thread ms: proxy %.1f, patterns %.1f, near list %.1f, "
                                     "groups %.1f)\n",
                             next.ms_partition, next.ms_near, gm[0], gm[1], gm[2], gm[3], gm[4], gm[5]);
            }
        }
        h->subs.push_back(std::move(sf));
    }
    h->stats.sublevels = (int)nsub;
    h->stats.levels = maxL;

    // ---- top blocks D = A_L over s_L (Sec. 3.1, level L), one per problem,
    // eliminated as boxes without skeletons: L, D, U of Lemma 2.1 and the
    // unit-triangular inverses used by the sweeps
    {
        auto sf = std::make_unique<SubFactor>();
        sf->kind = KIND_TOP;
        sf->level = maxL;
        ElimPlan ep;
        std::vector<int>& rdv = ep.rdv;
        int64_t top = 0;
        for (auto& sp : h->segs) {
            const Segment& sg = *sp;
            ElimDesc e{};
            e.ngroups = 0;
            e.sk_off = 0;
            e.rd_off = (int64_t)rdv.size();
            e.grp_off = 0;
            e.sci_out = -1;
            for (int64_t i = sg.off; i < sg.off + sg.N; ++i)
                if (active[i]) rdv.push_back((int)i);
            const int r = (int)((int64_t)rdv.size() - e.rd_off);
            if (r == 0) continue;
            top += r;
            e.k = 0;
            e.r = r;
            const bool big = r > big_elim_n;
            e.ldl = (h->opt.ldl && sg.sym && !big) ? 1 : 0;
            BoxFac bf{};
            sf->hbox.push_back(bf);
            sf->max_kr2 = std::max(sf->max_kr2, 2 * r);
            const double tf = 2.0 / 3.0 * (double)r * r * r + 2.0 * (double)r * r * r / 3.0;
            flops += tf;
            ep.add(e, big, tf);
        }
        sf->nbox = (int)sf->hbox.size();
        h->stats.top_size = top;
        if (sf->nbox) {
            Eliminator<T> elim{h, *sf, ep, nullptr, (int)nsub, Tws, S};
            elim.launch();
            elim.finish();
            HIF_CUDA(cudaStreamSynchronize(st));
            check_status(h);
        }
        h->subs.push_back(std::move(sf));
    }
    h->stats.flops = flops;
    h->stats.kernel_evals = evals;
}

// ---------------------------------------------------------- sweeps ------

enum { SOLVE_UP = 0, SOLVE_DOWN = 1, APPLY_UP = 2, APPLY_DOWN = 3,
       SOLVET_UP = 4, SOLVET_DOWN = 5, APPLYT_UP = 6, APPLYT_DOWN = 7 };

// One sublevel in one direction for all right-hand sides (CTA size: the
// sublevel's tuned value unless threads > 0).
template <typename T>
static void sweep_one(hif_handle h, SubFactor& sf, int mode, T* xw, int64_t ldx, int nrhs, int threads,
                      cudaStream_t st) {
    if (!sf.nbox) return;
    for (int r0 = 0; sf.nwide && r0 < nrhs; r0 += 16) {
        WideArgs w{};
        w.boxes = sf.wboxes.as<BoxFac>();
        w.sk_ids = sf.sk.as<int>();
        w.rd_ids = sf.rd.as<int>();
        w.pool = sf.pool.p;
        w.perm = sf.perm.as<int>();
        w.x = xw + ldx * r0;
        w.ldx = ldx;
        w.nr = std::min(16, nrhs - r0);
        w.ws = h->sweep_ws.p;
        w.ws_off = sf.wws_off.as<int64_t>();
        HIF_CUDA((launch_wide_sweep<T>(w, sf.nwide, sf.wmax_k, sf.wmax_r, mode, st)));
    }
    if (!sf.nsmall) return;
    const size_t per_col = (size_t)sf.max_kr2_small * sizeof(T);
    const int batch = sf.global ? nrhs : (int)std::min<size_t>((size_t)nrhs, std::max<size_t>(1, (200 * 1024) / per_col));
    for (int r0 = 0; r0 < nrhs; r0 += batch) {
        const int nr = std::min(batch, nrhs - r0);
        SweepArgs a{};
        a.boxes = sf.sboxes.as<BoxFac>();
        a.sk_ids = sf.sk.as<int>();
        a.rd_ids = sf.rd.as<int>();
        a.pool = sf.pool.p;
        a.perm = sf.perm.as<int>();
        a.x = xw + ldx * r0;
        a.ldx = ldx;
        a.nrhs = nr;
        const size_t smem = sf.global ? 0 : per_col * nr + 64;
        a.mode = mode | (int)(smem << 8);
        a.gws = sf.global ? h->sweep_ws.p : nullptr;
        a.gws_off = sf.global ? sf.gws_off.as<int64_t>() : nullptr;
        HIF_CUDA((launch_sweep<T>(a, sf.nsmall, threads > 0 ? threads : sf.threads, st)));
    }
}

template <typename T>
static void sweep_seq(hif_handle h, T* xw, int64_t ldx, int nrhs, int op, cudaStream_t st) {
    // op: 0 solve, 1 apply, 2 solve^T, 3 apply^T
    const int up = op == 0 ? SOLVE_UP : op == 1 ? APPLY_UP : op == 2 ? SOLVET_UP : APPLYT_UP;
    for (auto& sf : h->subs) sweep_one<T>(h, *sf, up, xw, ldx, nrhs, 0, st);
    for (auto it = h->subs.rbegin(); it != h->subs.rend(); ++it) sweep_one<T>(h, **it, up + 1, xw, ldx, nrhs, 0, st);
}

static void ensure_sweep_ws(hif_handle h, int nrhs, size_t elem) {
    int64_t need = 1;
    for (auto& sf : h->subs)
        need = std::max({need, sf->gws_units * std::max(nrhs, 1), sf->wws_units * std::min(std::max(nrhs, 1), 16)});
    h->sweep_ws.ensure(elem * (size_t)need);
}

// All sweeps of one operation.  With use_graphs the launch sequence for this
// (operation, nrhs, work buffer) is captured once into a CUDA graph on the
// handle's capture stream and replayed on the handle's stream.
template <typename T>
static void sweep_all(hif_handle h, T* xw, int64_t ldx, int nrhs, int op) {
    ensure_sweep_ws(h, nrhs, sizeof(T));
    double sweep_bytes = 0.0;
    if (prof_enabled())
        for (auto& sf : h->subs)
            sweep_bytes += sizeof(T) * (sf->sweep_factor_elems + 4.0 * sf->sweep_vec_elems * nrhs) +
                           sizeof(int) * sf->sweep_perm_ints;
    ProfRange pr(PROF_SWEEP, h->st, 0.0, sweep_bytes);
    if (!h->opt.use_graphs || ldx != h->N) {
        sweep_seq<T>(h, xw, ldx, nrhs, op, h->st);
        return;
    }
    SweepGraph* g = nullptr;
    for (auto& c : h->graphs)
        if (c.op == op && c.nrhs == nrhs && c.xw == (void*)xw && c.ws == h->sweep_ws.p) g = &c;
    if (!g) {
        if (!h->cap_st) HIF_CUDA(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
        const uint64_t before = g_launches.load();
        HIF_CUDA(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t graph = nullptr;
        try {
            sweep_seq<T>(h, xw, ldx, nrhs, op, h->cap_st);
        } catch (...) {
            cudaStreamEndCapture(h->cap_st, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        HIF_CUDA(cudaStreamEndCapture(h->cap_st, &graph));
        const uint64_t kernels = g_launches.load() - before;
        g_launches.fetch_sub(kernels);                 // counted when the graph runs
        SweepGraph ng;
        ng.op = op;
        ng.nrhs = nrhs;
        ng.xw = xw;
        ng.ws = h->sweep_ws.p;
        ng.kernels = kernels;
        const cudaError_t e = cudaGraphInstantiate(&ng.exec, graph, 0);
        cudaGraphDestroy(graph);
        HIF_CUDA(e);
        h->graphs.push_back(ng);
        g = &h->graphs.back();
    }
    HIF_CUDA(cudaGraphLaunch(g->exec, h->st));
    g_launches.fetch_add(g->kernels);
}

// After the factorization: the global work-space offsets of every sublevel,
// and (with autotune) the CTA size of each sublevel's sweep, picked by timing
// one solve sweep per candidate on the work vector.
template <typename T>
static void prepare_sweeps(hif_handle h) {
    const cudaStream_t st = h->st;
    for (auto& sp : h->subs) {
        SubFactor& sf = *sp;
        sf.sweep_factor_elems = sf.sweep_perm_ints = sf.sweep_vec_elems = 0;
        for (const BoxFac& bf : sf.hbox) {
            const double k = bf.k, r = bf.r;
            sf.sweep_factor_elems += 4.0 * k * r + r * r;
            sf.sweep_perm_ints += r;
            sf.sweep_vec_elems += k + r;
        }
        // wide LU boxes take the stage path (HIF_SWEEP_WIDE: the k + r above
        // which a box is wide)
        const int wide_min = env_int("HIF_SWEEP_WIDE", 768);
        std::vector<BoxFac> sb, wb;
        std::vector<int64_t> woffs;
        sf.wmax_k = sf.wmax_r = sf.max_kr2_small = 0;
        sf.wws_units = 0;
        for (const BoxFac& bf : sf.hbox) {
            if (!bf.ldl && bf.k + bf.r > wide_min) {
                wb.push_back(bf);
                woffs.push_back(sf.wws_units);
                sf.wws_units += (int64_t)bf.k + 2 * (int64_t)bf.r;
                sf.wmax_k = std::max(sf.wmax_k, bf.k);
                sf.wmax_r = std::max(sf.wmax_r, bf.r);
            } else {
                sb.push_back(bf);
                sf.max_kr2_small = std::max(sf.max_kr2_small, bf.k + 2 * bf.r);
            }
        }
        sf.nsmall = (int)sb.size();
        sf.nwide = (int)wb.size();
        upload(sf.sboxes, sb, st);
        upload(sf.wboxes, wb, st);
        upload(sf.wws_off, woffs, st);
        sf.global = (size_t)sf.max_kr2_small * sizeof(T) > 200 * 1024;
        sf.gws_units = 0;
        if (!sf.global || !sf.nsmall) continue;
        std::vector<int64_t> offs(sb.size());
        int64_t tot = 0;
        for (size_t q = 0; q < sb.size(); ++q) {
            offs[q] = tot;
            tot += (int64_t)(sb[q].k + 2 * sb[q].r);
        }
        upload(sf.gws_off, offs, st);
        sf.gws_units = tot;
    }
    if (!h->opt.autotune) return;
    const int64_t N = h->N;
    h->work.ensure(sizeof(T) * N);
    T* xw = h->work.as<T>();
    HIF_CUDA(cudaMemsetAsync(xw, 0, sizeof(T) * N, st));
    ensure_sweep_ws(h, 1, sizeof(T));
    cudaEvent_t e0, e1;
    HIF_CUDA(cudaEventCreate(&e0));
    HIF_CUDA(cudaEventCreate(&e1));
    const int cand[3] = {128, 256, 512};
    for (auto& sp : h->subs) {
        SubFactor& sf = *sp;
        if (!sf.nsmall) continue;
        float best = 1e30f;
        for (int c : cand) {
            float t = 0.f;
            for (int rep = 0; rep < 2; ++rep) {           // the first run warms the factor data
                HIF_CUDA(cudaEventRecord(e0, st));
                sweep_one<T>(h, sf, SOLVE_UP, xw, N, 1, c, st);
                HIF_CUDA(cudaEventRecord(e1, st));
                HIF_CUDA(cudaEventSynchronize(e1));
                HIF_CUDA(cudaEventElapsedTime(&t, e0, e1));
            }
            if (t < best) {
                best = t;
                sf.threads = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

static void apply_op(hif_handle h, const double* in, double* out, int64_t nrhs, int64_t ld, int op) {
    if (!h) fail(HIF_EINVAL, "null handle");
    if (nrhs < 0 || ld < h->N || !in || !out) fail(HIF_EINVAL, "bad vector arguments");
    if (nrhs == 0) return;
    const cudaStream_t st = h->st;
    const int64_t N = h->N;
    // device views of the caller's arrays
    const bool din = is_device_ptr(in), dout = is_device_ptr(out);
    DevMem tin, tout;
    const double* din_p = in;
    double* dout_p = out;
    int64_t ldi = ld, ldo = ld;
    if (!din) {
        tin.ensure(sizeof(double) * N * nrhs);
        HIF_CUDA(cudaMemcpy2DAsync(tin.p, sizeof(double) * N, in, sizeof(double) * ld, sizeof(double) * N, nrhs,
                                   cudaMemcpyHostToDevice, st));
        din_p = tin.as<double>();
        ldi = N;
    }
    if (!dout) {
        tout.ensure(sizeof(double) * N * nrhs);
        dout_p = tout.as<double>();
        ldo = N;
    }
    if (h->precision == 0) {
        h->work.ensure(sizeof(double) * N * nrhs);
        double* xw = h->work.as<double>();
        HIF_CUDA(launch_to_work<double>(din_p, ldi, xw, N, N, (int)nrhs, st));
        sweep_all<double>(h, xw, N, (int)nrhs, op);
        HIF_CUDA(launch_from_work<double>(xw, N, dout_p, ldo, N, (int)nrhs, st));
    } else {
        h->work.ensure(sizeof(float) * N * nrhs);
        float* xw = h->work.as<float>();
        HIF_CUDA(launch_to_work<float>(din_p, ldi, xw, N, N, (int)nrhs, st));
        sweep_all<float>(h, xw, N, (int)nrhs, op);
        HIF_CUDA(launch_from_work<float>(xw, N, dout_p, ldo, N, (int)nrhs, st));
    }
    if (!dout)
        HIF_CUDA(cudaMemcpy2DAsync(out, sizeof(double) * ld, dout_p, sizeof(double) * N, sizeof(double) * N, nrhs,
                                   cudaMemcpyDeviceToHost, st));
    HIF_CUDA(cudaStreamSynchronize(st));
}

// Direct sum on device arrays, problem by problem (the operator of a handle
// is block diagonal over its problems).  classes < 8 selects a short digit set
// of the tensor-core sum (grid problems with direct_precision 2); every other
// path computes its one sum.
static void matvec_dev(hif_handle h, int trans, const double* x, int64_t ldx, double* y, int64_t ldy, int nrhs,
                       int classes = 8) {
    const cudaStream_t st = h->st;
    for (auto& sp : h->segs) {
        Segment& sg = *sp;
        if (sg.grid) {
            const int64_t n = sg.N;
            h->vbuf.ensure(sizeof(double) * n * nrhs);
            h->ybuf.ensure(sizeof(double) * n * nrhs);
            GridDirectArgs ga{};
            ga.table = sg.table.as<double>();
            ga.dof_of = sg.dof_of.as<int>();
            ga.n = sg.gn;
            ga.dim = h->dim;
            ga.a = h->a.as<double>();
            ga.b = h->b.as<double>();
            ga.c = h->c.as<double>();
            ga.w = h->w.as<double>();
            ga.x = x;
            ga.ldx = ldx;
            ga.y = y;
            ga.ldy = ldy;
            ga.nrhs = nrhs;
            ga.trans = trans;
            ga.vbuf = h->vbuf.as<double>();
            ga.ybuf = h->ybuf.as<double>();
            if (h->opt.direct_precision == 0) {
                h->vdf.ensure(sizeof(float2) * n * nrhs);
                ProfRange pr(PROF_DIRECT, st, 2.0 * (double)n * n * nrhs, 0.0);
                HIF_CUDA(launch_direct_grid_df(ga, sg.table_df.as<float2>(), h->vdf.as<float2>(), st));
            } else if (h->opt.direct_precision == 2) {
                if (!sg.tc_rows.p) {
                    sg.tc_tmax.ensure(sizeof(unsigned long long));
                    sg.tc_rows.ensure(tc_table_rows_bytes(sg.gn, h->dim));
                    HIF_CUDA(launch_tc_table(sg.table.as<double>(), sg.gn, h->dim,
                                             sg.tc_tmax.as<unsigned long long>(), sg.tc_rows.p, st));
                }
                h->tc_xb.ensure(tc_source_digits_bytes(sg.gn, h->dim));
                h->tc_xmax.ensure(8 * sizeof(unsigned long long));
                h->tc_status.ensure(sizeof(int));
                HIF_CUDA(cudaMemsetAsync(h->tc_status.p, 0, sizeof(int), st));
                {
                    ProfRange pr(classes == 8 ? PROF_DIRECT : PROF_DIRECT_SHORT, st, 2.0 * (double)n * n * nrhs, 0.0);
                    HIF_CUDA(launch_direct_grid_tc(ga, sg.tc_rows.p, sg.tc_tmax.as<unsigned long long>(), h->tc_xb.p,
                                                   h->tc_xmax.as<unsigned long long>(), h->tc_status.as<int>(),
                                                   h->num_sms, classes, st));
                }
                int flag = 0;
                HIF_CUDA(cudaMemcpyAsync(&flag, h->tc_status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
                HIF_CUDA(cudaStreamSynchronize(st));
                if (flag) fail(HIF_ETIMEOUT, "tensor-core direct sum: a pipeline wait expired");
            } else {
                ProfRange pr(PROF_DIRECT, st, 2.0 * (double)n * n * nrhs, 0.0);
                HIF_CUDA(launch_direct_grid(ga, st));
            }
        } else {
            DirectArgs da{};
            da.g = geom(h);
            da.x = x;
            da.ldx = ldx;
            da.y = y;
            da.ldy = ldy;
            da.nrhs = nrhs;
            da.trans = trans;
            da.seg_off = sg.off;
            da.seg_n = sg.N;
            ProfRange pr(PROF_DIRECT, st, 2.0 * (double)sg.N * sg.N * nrhs, 0.0);
            if (h->ncomp == 2) HIF_CUDA(launch_direct_helmholtz(da, st));
            else HIF_CUDA(launch_direct_general(da, st));
        }
    }
}

// x = F^{-1} b, F b, F^{-T} b or F^T b (op 0, 1, 2, 3) on device arrays with ld = N
static void fac_dev(hif_handle h, int op, const double* b, double* x, int nrhs) {
    const cudaStream_t st = h->st;
    const int64_t N = h->N;
    if (h->precision == 0) {
        h->work.ensure(sizeof(double) * N * nrhs);
        double* xw = h->work.as<double>();
        HIF_CUDA(launch_to_work<double>(b, N, xw, N, N, nrhs, st));
        sweep_all<double>(h, xw, N, nrhs, op);
        HIF_CUDA(launch_from_work<double>(xw, N, x, N, N, nrhs, st));
    } else {
        h->work.ensure(sizeof(float) * N * nrhs);
        float* xw = h->work.as<float>();
        HIF_CUDA(launch_to_work<float>(b, N, xw, N, N, nrhs, st));
        sweep_all<float>(h, xw, N, nrhs, op);
        HIF_CUDA(launch_from_work<float>(xw, N, x, N, N, nrhs, st));
    }
}

static void solve_dev(hif_handle h, int trans, const double* b, double* x, int nrhs) {
    fac_dev(h, trans ? 2 : 0, b, x, nrhs);
}

static std::vector<double> col_norms(hif_handle h, const double* v, int nrhs) {
    h->tmp.ensure(sizeof(double) * std::max(nrhs, 1));
    HIF_CUDA(launch_col_dots(h->N, nrhs, v, h->N, v, h->N, h->tmp.as<double>(), h->st));
    std::vector<double> out(nrhs);
    HIF_CUDA(cudaMemcpyAsync(out.data(), h->tmp.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, h->st));
    HIF_CUDA(cudaStreamSynchronize(h->st));
    for (double& o : out) o = std::sqrt(std::max(o, 0.0));
    return out;
}

// 2-norms of every column restricted to every problem: nseg x nrhs, column-major.
static std::vector<double> seg_norms(hif_handle h, const double* v, int nrhs) {
    const int ns = (int)h->segs.size();
    h->tmp.ensure(sizeof(double) * std::max(ns * nrhs, 1));
    HIF_CUDA(launch_seg_dots(ns, h->seg_off.as<int64_t>(), h->seg_n.as<int64_t>(), nrhs, v, h->N, v, h->N,
                             h->tmp.as<double>(), h->st));
    std::vector<double> out((size_t)ns * nrhs);
    HIF_CUDA(cudaMemcpyAsync(out.data(), h->tmp.p, sizeof(double) * out.size(), cudaMemcpyDeviceToHost, h->st));
    HIF_CUDA(cudaStreamSynchronize(h->st));
    for (double& o : out) o = std::sqrt(std::max(o, 0.0));
    return out;
}

static bool short_residuals_on(hif_handle h, double tol) {
    if (h->opt.direct_precision != 2 || tol < 1e-11 || !env_int("HIF_SHORT_RESIDUAL", 1)) return false;
    for (auto& sp : h->segs)
        if (!sp->grid) return false;
    return true;
}

// Iterative refinement: u = F^{-1} f; r = f - A u; u += F^{-1} r ...  The
// returned residual is always that of the full sum: a short residual at or
// below tol, at the last step, or whose estimated error misses the bound for
// the residual it found is recomputed in full.
static hif_status refine_ir(hif_handle h, int trans, const double* f, double* u, int nrhs, double tol, int maxit,
                            int* iters, double* relres) {
    const int64_t N = h->N;
    DevMem r, du;
    r.ensure(sizeof(double) * N * nrhs);
    du.ensure(sizeof(double) * N * nrhs);
    // relative residuals are judged per problem and per column
    const std::vector<double> fn = seg_norms(h, f, nrhs);
    solve_dev(h, trans, f, u, nrhs);
    const bool shorts = short_residuals_on(h, tol);
    double S = 1.0;
    for (auto& sp : h->segs) S = std::max(S, sp->spread);
    int it = 0;
    double worst = 0, Y = 0;
    std::vector<double> hist;
    for (;; ++it) {
        int classes = shorts ? short_residual_classes(it, h->precision == 1, hist.data(), S * Y, tol) : 8;
        for (;;) {
            matvec_dev(h, trans, u, N, r.as<double>(), N, nrhs, classes);
            HIF_CUDA(launch_axpby(N, nrhs, 1.0, f, N, -1.0, r.as<double>(), N, h->st));
            const std::vector<double> rn = seg_norms(h, r.as<double>(), nrhs);
            worst = 0;
            for (size_t q = 0; q < rn.size(); ++q) worst = std::max(worst, fn[q] > 0 ? rn[q] / fn[q] : 0.0);
            if (shorts) {
                // Y: the kernel part f - r - a u against f (du is free until the correction)
                HIF_CUDA(launch_kpart(N, nrhs, f, r.as<double>(), h->a.as<double>(), u, du.as<double>(), h->st));
                const std::vector<double> yn = seg_norms(h, du.as<double>(), nrhs);
                Y = 0;
                for (size_t q = 0; q < yn.size(); ++q) Y = std::max(Y, fn[q] > 0 ? yn[q] / fn[q] : 0.0);
            }
            if (env_int("HIF_TRACE", 0))
                std::fprintf(stderr, "[hif] refinement %d: relative residual %.3e (%d digit classes, |bKcu|/|f| %.2e)\n",
                             it, worst, classes, Y);
            if (classes == 8 || short_residual_usable(classes, worst, S * Y, tol, it >= maxit)) break;
            classes = 8;
        }
        hist.push_back(worst);
        if (worst <= tol || it >= maxit) break;
        solve_dev(h, trans, r.as<double>(), du.as<double>(), nrhs);
        HIF_CUDA(launch_axpby(N, nrhs, 1.0, du.as<double>(), N, 1.0, u, N, h->st));
    }
    if (iters) *iters = it;
    if (relres) *relres = worst;
    return worst <= tol ? HIF_OK : HIF_ENOTCONV;
}

// |E|_2 by power iteration on E^T E (Sec. 5) for E_0 = A, E_1 = A - F and
// E_2 = I - A F^{-1}, run side by side as the three columns of one block so
// that each step costs one direct sum with A and one with A^T: v = v0 / |v0|;
// every step w = E v, u = E^T w, the estimate sqrt(|u|), v = u / |u|; a
// column stops when its estimate moved by at most rtol of itself, or after
// maxit steps.  A is the direct sum, F the factored form.
static bool power_norms_dev(hif_handle h, const double* v0, double rtol, int maxit, double* norms, int* iters) {
    const int64_t N = h->N;
    const cudaStream_t st = h->st;
    DevMem V, X, W, U, Tv;
    V.ensure(sizeof(double) * N * 3);
    X.ensure(sizeof(double) * N * 3);
    W.ensure(sizeof(double) * N * 3);
    U.ensure(sizeof(double) * N * 3);
    Tv.ensure(sizeof(double) * N);
    double* vp = V.as<double>();
    double* xp = X.as<double>();
    double* wp = W.as<double>();
    double* up = U.as<double>();
    double* tp = Tv.as<double>();
    HIF_CUDA(cudaMemcpyAsync(tp, v0, sizeof(double) * N,
                             is_device_ptr(v0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    const double n0 = col_norms(h, tp, 1)[0];
    if (!(n0 > 0) || !std::isfinite(n0)) fail(HIF_EINVAL, "start vector must be finite and nonzero");
    for (int c = 0; c < 3; ++c) HIF_CUDA(launch_axpby(N, 1, 1.0 / n0, tp, N, 0.0, vp + N * c, N, st));
    double est[3] = {0.0, 0.0, 0.0};
    bool done[3] = {false, false, false};
    for (int c = 0; c < 3; ++c) iters[c] = 0;
    for (int it = 1; it <= maxit && !(done[0] && done[1] && done[2]); ++it) {
        // W = E V: A [v0, v1, F^{-1} v2], then column 1 minus F v1, column 2 = v2 - (.)
        HIF_CUDA(cudaMemcpyAsync(xp, vp, sizeof(double) * N * 2, cudaMemcpyDeviceToDevice, st));
        fac_dev(h, 0, vp + 2 * N, xp + 2 * N, 1);
        matvec_dev(h, 0, xp, N, wp, N, 3);
        fac_dev(h, 1, vp + N, tp, 1);
        HIF_CUDA(launch_axpby(N, 1, -1.0, tp, N, 1.0, wp + N, N, st));
        HIF_CUDA(launch_axpby(N, 1, 1.0, vp + 2 * N, N, -1.0, wp + 2 * N, N, st));
        // U = E^T W: A^T W, then column 1 minus F^T w1, column 2 = w2 - F^{-T} (.)
        matvec_dev(h, 1, wp, N, up, N, 3);
        fac_dev(h, 3, wp + N, tp, 1);
        HIF_CUDA(launch_axpby(N, 1, -1.0, tp, N, 1.0, up + N, N, st));
        fac_dev(h, 2, up + 2 * N, tp, 1);
        HIF_CUDA(launch_axpby(N, 1, 1.0, wp + 2 * N, N, 0.0, up + 2 * N, N, st));
        HIF_CUDA(launch_axpby(N, 1, -1.0, tp, N, 1.0, up + 2 * N, N, st));
        const std::vector<double> nu = col_norms(h, up, 3);
        for (int c = 0; c < 3; ++c) {
            if (done[c]) continue;
            iters[c] = it;
            if (!std::isfinite(nu[c])) fail(HIF_ENUMERIC, "non-finite power iterate");
            if (nu[c] == 0.0) {
                est[c] = 0.0;
                done[c] = true;
                continue;
            }
            const double nw = std::sqrt(nu[c]);
            HIF_CUDA(launch_axpby(N, 1, 1.0 / nu[c], up + N * c, N, 0.0, vp + N * c, N, st));
            if (est[c] > 0.0 && std::fabs(nw - est[c]) <= rtol * nw) done[c] = true;
            est[c] = nw;
        }
    }
    for (int c = 0; c < 3; ++c) norms[c] = est[c];
    return done[0] && done[1] && done[2];
}

// Right-preconditioned GMRES(m), all columns advanced together, modified
// Gram-Schmidt in FP64; the Hessenberg least-squares problems are solved on
// the host (they are at most (m+1) x m per column).
static hif_status refine_gmres(hif_handle h, int trans, const double* f, double* u, int nrhs, double tol, int maxit,
                               int* iters, double* relres) {
    const int m = 20;
    const int64_t N = h->N;
    const cudaStream_t st = h->st;
    DevMem V, Z, wv, r, tmpc;
    V.ensure(sizeof(double) * N * nrhs * (m + 1));
    Z.ensure(sizeof(double) * N * nrhs * m);
    wv.ensure(sizeof(double) * N * nrhs);
    r.ensure(sizeof(double) * N * nrhs);
    tmpc.ensure(sizeof(double) * nrhs);
    double* Vp = V.as<double>();
    double* Zp = Z.as<double>();
    auto Vc = [&](int j) { return Vp + (int64_t)j * N * nrhs; };
    auto Zc = [&](int j) { return Zp + (int64_t)j * N * nrhs; };
    const std::vector<double> fn = col_norms(h, f, nrhs);
    HIF_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * N * nrhs, st));
    int its = 0;
    double worst = 1.0;
    std::vector<double> beta(nrhs);
    for (int c = 0; c < nrhs; ++c) beta[c] = fn[c];
    HIF_CUDA(cudaMemcpyAsync(r.p, f, sizeof(double) * N * nrhs, cudaMemcpyDeviceToDevice, st));
    while (true) {
        worst = 0;
        for (int c = 0; c < nrhs; ++c) worst = std::max(worst, fn[c] > 0 ? beta[c] / fn[c] : 0.0);
        if (worst <= tol || its >= maxit) break;
        // V_0 = r / beta (column scaling on the device through a tiny kernel: use axpby per column)
        for (int c = 0; c < nrhs; ++c)
            HIF_CUDA(launch_axpby(N, 1, beta[c] > 0 ? 1.0 / beta[c] : 0.0, r.as<double>() + N * c, N, 0.0,
                                  Vc(0) + N * c, N, st));
        std::vector<std::vector<double>> H(nrhs, std::vector<double>((m + 1) * m, 0.0));
        std::vector<std::vector<double>> gvec(nrhs, std::vector<double>(m + 1, 0.0));
        std::vector<std::vector<double>> cs(nrhs, std::vector<double>(m)), sn(nrhs, std::vector<double>(m));
        for (int c = 0; c < nrhs; ++c) gvec[c][0] = beta[c];
        int jdone = 0;
        std::vector<double> dots(nrhs);
        for (int j = 0; j < m; ++j) {
            solve_dev(h, trans, Vc(j), Zc(j), nrhs);
            matvec_dev(h, trans, Zc(j), N, wv.as<double>(), N, nrhs);
            for (int i = 0; i <= j; ++i) {
                HIF_CUDA(launch_col_dots(N, nrhs, Vc(i), N, wv.as<double>(), N, tmpc.as<double>(), st));
                HIF_CUDA(cudaMemcpyAsync(dots.data(), tmpc.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
                HIF_CUDA(cudaStreamSynchronize(st));
                for (int c = 0; c < nrhs; ++c) {
                    H[c][i + (m + 1) * j] = dots[c];
                    HIF_CUDA(launch_axpby(N, 1, -dots[c], Vc(i) + N * c, N, 1.0, wv.as<double>() + N * c, N, st));
                }
            }
            const std::vector<double> hn = col_norms(h, wv.as<double>(), nrhs);
            bool all_conv = true;
            for (int c = 0; c < nrhs; ++c) {
                H[c][j + 1 + (m + 1) * j] = hn[c];
                HIF_CUDA(launch_axpby(N, 1, hn[c] > 0 ? 1.0 / hn[c] : 0.0, wv.as<double>() + N * c, N, 0.0,
                                      Vc(j + 1) + N * c, N, st));
                double* Hc = H[c].data();
                for (int i = 0; i < j; ++i) {
                    const double t0 = cs[c][i] * Hc[i + (m + 1) * j] + sn[c][i] * Hc[i + 1 + (m + 1) * j];
                    Hc[i + 1 + (m + 1) * j] = -sn[c][i] * Hc[i + (m + 1) * j] + cs[c][i] * Hc[i + 1 + (m + 1) * j];
                    Hc[i + (m + 1) * j] = t0;
                }
                const double den = std::hypot(Hc[j + (m + 1) * j], Hc[j + 1 + (m + 1) * j]);
                cs[c][j] = den > 0 ? Hc[j + (m + 1) * j] / den : 1.0;
                sn[c][j] = den > 0 ? Hc[j + 1 + (m + 1) * j] / den : 0.0;
                Hc[j + (m + 1) * j] = cs[c][j] * Hc[j + (m + 1) * j] + sn[c][j] * Hc[j + 1 + (m + 1) * j];
                Hc[j + 1 + (m + 1) * j] = 0.0;
                gvec[c][j + 1] = -sn[c][j] * gvec[c][j];
                gvec[c][j] = cs[c][j] * gvec[c][j];
                if (fn[c] > 0 && std::fabs(gvec[c][j + 1]) / fn[c] > tol) all_conv = false;
            }
            ++its;
            jdone = j + 1;
            if (all_conv || its >= maxit) break;
        }
        // u += Z y per column
        for (int c = 0; c < nrhs; ++c) {
            std::vector<double> y(jdone, 0.0);
            for (int i = jdone - 1; i >= 0; --i) {
                double v = gvec[c][i];
                for (int l = i + 1; l < jdone; ++l) v -= H[c][i + (m + 1) * l] * y[l];
                const double dg = H[c][i + (m + 1) * i];
                y[i] = dg != 0 ? v / dg : 0.0;
            }
            for (int i = 0; i < jdone; ++i)
                HIF_CUDA(launch_axpby(N, 1, y[i], Zc(i) + N * c, N, 1.0, u + N * c, N, st));
        }
        matvec_dev(h, trans, u, N, r.as<double>(), N, nrhs);
        HIF_CUDA(launch_axpby(N, nrhs, 1.0, f, N, -1.0, r.as<double>(), N, st));
        beta = col_norms(h, r.as<double>(), nrhs);
    }
    if (iters) *iters = its;
    if (relres) *relres = worst;
    return worst <= tol ? HIF_OK : HIF_ENOTCONV;
}

template <typename F>
static hif_status guard(F&& fn) {
    try {
        fn();
        return HIF_OK;
    } catch (const Err& e) {
        return e.s;
    } catch (const std::bad_alloc&) {
        return HIF_ENOMEM;
    }
}

// Runs fn on device copies (ld = N) of a caller input and output, copying
// host arrays in and out.
template <typename F>
static void with_dev_io(hif_handle h, const double* in, double* out, int64_t nrhs, int64_t ld, F&& fn) {
    const int64_t N = h->N;
    const cudaStream_t st = h->st;
    DevMem din, dout;
    din.ensure(sizeof(double) * N * nrhs);
    dout.ensure(sizeof(double) * N * nrhs);
    HIF_CUDA(cudaMemcpy2DAsync(din.p, sizeof(double) * N, in, sizeof(double) * ld, sizeof(double) * N, nrhs,
                               is_device_ptr(in) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    fn(din.as<double>(), dout.as<double>());
    HIF_CUDA(cudaMemcpy2DAsync(out, sizeof(double) * ld, dout.p, sizeof(double) * N, sizeof(double) * N, nrhs,
                               is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    HIF_CUDA(cudaStreamSynchronize(st));
}

}  // namespace hif

using namespace hif;

extern "C" {

const char* hif_status_string(hif_status s) {
    switch (s) {
        case HIF_OK: return "HIF_OK";
        case HIF_EINVAL: return "HIF_EINVAL: invalid argument";
        case HIF_ENOMEM: return "HIF_ENOMEM: out of memory";
        case HIF_ESINGULAR: return "HIF_ESINGULAR: singular elimination block";
        case HIF_ENUMERIC: return "HIF_ENUMERIC: non-finite value";
        case HIF_ECUDA: return "HIF_ECUDA: CUDA runtime error";
        case HIF_ETIMEOUT: return "HIF_ETIMEOUT: bounded wait expired";
        case HIF_ENOTCONV: return "HIF_ENOTCONV: tolerance not reached";
    }
    return "unknown hif_status";
}

const char* hif_last_error(void) { return g_last_error; }

uint64_t hif_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

hif_status hif_kernel_timing(int enable, double* ms, int64_t* launches) {
    return guard([&] {
        HIF_CUDA(tc_timing_collect(ms, launches));
        tc_timing_set(enable != 0);
    });
}

hif_status hif_kernel_profile(int enable, hif_profile_entry* out, int cap, int* count) {
    return guard([&] {
        int64_t rg[PROF_COUNT];
        double ms[PROF_COUNT], fl[PROF_COUNT], by[PROF_COUNT];
        HIF_CUDA(prof_collect(rg, ms, fl, by));
        if (count) *count = PROF_COUNT;
        for (int k = 0; out && k < PROF_COUNT && k < cap; ++k) {
            out[k].name = prof_name(k);
            out[k].ranges = rg[k];
            out[k].ms = ms[k];
            out[k].flops = fl[k];
            out[k].bytes = by[k];
        }
        prof_set(enable != 0);
    });
}

hif_status hif_options_default(int dim, hif_options* opt) {
    if (!opt || (dim != 2 && dim != 3)) return HIF_EINVAL;
    std::memset(opt, 0, sizeof(*opt));
    opt->dim = dim;
    opt->leaf_occupancy = 64;
    opt->second_kind = 1;
    opt->precision = 0;
    opt->fractional_levels = 1;
    opt->skip_levels = 0;
    opt->proxy_points = dim == 2 ? 64 : 512;
    opt->proxy_radius = 1.5;
    opt->proxy_dirs = nullptr;
    opt->fp32_tol_floor = std::ldexp(1.0, -17);
    opt->direct_precision = 2;
    opt->use_graphs = 1;
    opt->autotune = 1;
    opt->symmetric = 1;
    opt->ldl = 1;
    opt->root_width = 0.0;
    opt->stream = nullptr;
    return HIF_OK;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton's method on the
// three-term recurrence of the Legendre polynomials).
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            const double dz = p0 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Self-cell integral of the Helmholtz kernel G(r) = (i/4) H_0^(1)(k r) over
// the square of side h centred at the singularity (Sec. 5, Example 3, with
// the quadratures of the volume examples).  The real part is split as
// -log(r)/(2 pi) (the Laplace kernel, whose integral is in closed form) plus
// the bounded rest -Y_0(k r)/4 + log(r)/(2 pi); the rest and the imaginary
// part J_0(k r)/4 are integrated in polar coordinates about the centre,
// 8 int_0^{pi/4} int_0^{h/(2 cos t)} f(r) r dr dt, by 48 x 48-point
// Gauss-Legendre rules.  Bessel functions from the C math library.
static void helmholtz_self(double k, double h, double* re, double* im) {
    std::vector<double> xg, wg;
    gauss_legendre(48, xg, wg);
    double sr = 0.0, si = 0.0;
    for (size_t a = 0; a < xg.size(); ++a) {
        const double t = (xg[a] + 1.0) * kPi / 8.0, wt = wg[a] * kPi / 8.0;
        const double R = 0.5 * h / std::cos(t);
        for (size_t b = 0; b < xg.size(); ++b) {
            const double r = 0.5 * (xg[b] + 1.0) * R, wr = 0.5 * wg[b] * R;
            sr += wt * wr * r * (-0.25 * ::y0(k * r) + std::log(r) / (2.0 * kPi));
            si += wt * wr * r * (0.25 * ::j0(k * r));
        }
    }
    const double lap = -(h * h / (2.0 * kPi)) * (std::log(h) - 0.5 * std::log(2.0) - 1.5 + 0.25 * kPi);
    *re = lap + 8.0 * sr;
    *im = 8.0 * si;
}

static hif_status factor_impl(int count, const hif_problem* probs, int kernel_id, double eps, const hif_options* opt_in,
                              hif_handle* out) {
    if (!out) return HIF_EINVAL;
    *out = nullptr;
    hif_options opt;
    if (opt_in) opt = *opt_in;
    else hif_options_default(2, &opt);
    if (count <= 0 || !probs) return HIF_EINVAL;
    int64_t N = 0;
    for (int q = 0; q < count; ++q) {
        const hif_problem& pr = probs[q];
        if (pr.N <= 0 || !pr.points || !pr.weights || !pr.a || !pr.b || !pr.c) return HIF_EINVAL;
        N += pr.N;
    }
    if (N > (int64_t)2000000000) return HIF_EINVAL;
    if (opt.dim != 2 && opt.dim != 3) return HIF_EINVAL;
    if ((opt.dim == 2 && kernel_id != 0 && kernel_id != 2) || (opt.dim == 3 && kernel_id != 1)) return HIF_EINVAL;
    if (kernel_id == 2 && !(opt.wavenumber > 0.0 && std::isfinite(opt.wavenumber))) return HIF_EINVAL;
    if (!(eps >= 0.0) || !std::isfinite(eps)) return HIF_EINVAL;
    if (opt.leaf_occupancy < 1 || opt.proxy_points < 1 || !(opt.proxy_radius > 0)) return HIF_EINVAL;
    if (opt.precision != 0 && opt.precision != 1) return HIF_EINVAL;
    if (opt.direct_precision < 0 || opt.direct_precision > 2) return HIF_EINVAL;
    if (opt.symmetric != 0 && opt.symmetric != 1) return HIF_EINVAL;
    if (opt.ldl != 0 && opt.ldl != 1) return HIF_EINVAL;
    if (opt.dim == 3 && !opt.proxy_dirs) return HIF_EINVAL;
    auto h = std::make_unique<hif_handle_s>();
    const auto t0 = std::chrono::steady_clock::now();
    hif_status s = guard([&] {
        h->dim = opt.dim;
        h->kernel_id = kernel_id;
        h->precision = opt.precision;
        h->second_kind = opt.second_kind ? 1 : 0;
        h->N = N;
        h->eps = eps;
        h->opt = opt;
        h->st = static_cast<cudaStream_t>(opt.stream);
        {
            int dev = 0;
            HIF_CUDA(cudaGetDevice(&dev));
            HIF_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
        }
        h->elem = opt.precision == 0 ? 8 : 4;
        const int d = opt.dim;
        const cudaStream_t st = h->st;
        // inputs: one concatenated device copy owned by the handle (problem q
        // holds rows [off_q, off_q + N_q)), and host copies of the geometry
        h->x.ensure(sizeof(double) * N * d);
        h->w.ensure(sizeof(double) * N);
        h->a.ensure(sizeof(double) * N);
        h->b.ensure(sizeof(double) * N);
        h->c.ensure(sizeof(double) * N);
        auto take = [&](DevMem& dst, int64_t off, const double* src, size_t cnt) {
            HIF_CUDA(cudaMemcpyAsync(dst.as<double>() + off, src, cnt * sizeof(double),
                                     is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        };
        std::vector<int64_t> soff(count), sn(count);
        int64_t off = 0;
        for (int q = 0; q < count; ++q) {
            const hif_problem& pr = probs[q];
            take(h->x, off * d, pr.points, (size_t)pr.N * d);
            take(h->w, off, pr.weights, (size_t)pr.N);
            take(h->a, off, pr.a, (size_t)pr.N);
            take(h->b, off, pr.b, (size_t)pr.N);
            take(h->c, off, pr.c, (size_t)pr.N);
            auto sg = std::make_unique<Segment>();
            sg->off = off;
            sg->N = pr.N;
            soff[q] = off;
            sn[q] = pr.N;
            h->segs.push_back(std::move(sg));
            off += pr.N;
        }
        upload(h->seg_off, soff, st);
        upload(h->seg_n, sn, st);
        h->hx.resize((size_t)N * d);
        h->hw.resize((size_t)N);
        HIF_CUDA(cudaMemcpyAsync(h->hx.data(), h->x.p, sizeof(double) * N * d, cudaMemcpyDeviceToHost, st));
        HIF_CUDA(cudaMemcpyAsync(h->hw.data(), h->w.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        std::vector<double> ha(N), hbv(N), hc(N);
        HIF_CUDA(cudaMemcpyAsync(ha.data(), h->a.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        HIF_CUDA(cudaMemcpyAsync(hbv.data(), h->b.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        HIF_CUDA(cudaMemcpyAsync(hc.data(), h->c.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        HIF_CUDA(cudaStreamSynchronize(st));
        for (int64_t i = 0; i < N; ++i) {
            if (!std::isfinite(ha[i]) || !std::isfinite(hbv[i]) || !std::isfinite(hc[i]) || !(h->hw[i] > 0) ||
                !std::isfinite(h->hw[i]))
                fail(HIF_ENUMERIC, "non-finite or non-positive input");
            for (int k = 0; k < d; ++k)
                if (!std::isfinite(h->hx[d * i + k])) fail(HIF_ENUMERIC, "non-finite point");
        }
        if (kernel_id == 2) {
            // complex operator (Sec. 5, Example 3) through its real 2 x 2
            // embedding: point j carries the real DOFs 2j (real part) and
            // 2j + 1 (imaginary part); every array is repeated per component,
            // and from here on the handle works on 2N real DOFs
            h->ncomp = 2;
            h->wavenumber = opt.wavenumber;
            auto rep2 = [](const std::vector<double>& v, int per) {
                std::vector<double> o(v.size() * 2);
                const size_t n = v.size() / per;
                for (size_t i = 0; i < n; ++i)
                    for (int r = 0; r < 2; ++r)
                        for (int k = 0; k < per; ++k) o[(2 * i + r) * per + k] = v[i * per + k];
                return o;
            };
            h->hx = rep2(h->hx, d);
            h->hw = rep2(h->hw, 1);
            ha = rep2(ha, 1);
            hbv = rep2(hbv, 1);
            hc = rep2(hc, 1);
            N *= 2;
            h->N = N;
            for (auto& sp : h->segs) {
                sp->off *= 2;
                sp->N *= 2;
            }
            for (int q = 0; q < count; ++q) {
                soff[q] *= 2;
                sn[q] *= 2;
            }
            upload(h->seg_off, soff, st);
            upload(h->seg_n, sn, st);
            upload(h->x, h->hx, st);
            upload(h->w, h->hw, st);
            upload(h->a, ha, st);
            upload(h->b, hbv, st);
            upload(h->c, hc, st);
        }
        // A = diag(a) + diag(b) K diag(c) with K_ij = G_ij w_j is symmetric
        // when b_i w_j c_j = b_j w_i c_i; tested in the sufficient form b = c
        // and equal weights, problem by problem
        for (auto& sp : h->segs) {
            Segment& sg = *sp;
            // (the real embedding of a complex symmetric matrix is not symmetric)
            bool sym = opt.symmetric != 0 && kernel_id != 2;
            for (int64_t i = sg.off; sym && i < sg.off + sg.N; ++i)
                sym = hbv[i] == hc[i] && h->hw[i] == h->hw[sg.off];
            sg.sym = sym;
            h->stats.symmetric_problems += sym ? 1 : 0;
        }
        // proxy directions
        h->P = opt.proxy_points;
        std::vector<double> pd((size_t)h->P * d);
        if (opt.proxy_dirs) {
            if (is_device_ptr(opt.proxy_dirs))
                HIF_CUDA(cudaMemcpy(pd.data(), opt.proxy_dirs, sizeof(double) * pd.size(), cudaMemcpyDeviceToHost));
            else
                std::memcpy(pd.data(), opt.proxy_dirs, sizeof(double) * pd.size());
        } else {
            for (int k = 0; k < h->P; ++k) {
                const double th = 2.0 * kPi * k / h->P;
                pd[2 * k] = std::cos(th);
                pd[2 * k + 1] = std::sin(th);
            }
        }
        if (h->ncomp == 2) {
            // every proxy direction once per component (rows 2e, 2e + 1)
            std::vector<double> pd2((size_t)2 * h->P * d);
            for (int e = 0; e < h->P; ++e)
                for (int r = 0; r < 2; ++r)
                    for (int k = 0; k < d; ++k) pd2[((size_t)2 * e + r) * d + k] = pd[(size_t)e * d + k];
            pd.swap(pd2);
            h->P *= 2;
        }
        upload(h->proxy, pd, st);
        h->kself.ensure(sizeof(double) * N);
        std::vector<double> hks(N);
        if (h->ncomp == 2) {
            std::vector<double> ksi(N);
            double last_w = -1.0, kr = 0.0, ki = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                if (h->hw[i] != last_w) {
                    helmholtz_self(h->wavenumber, std::sqrt(h->hw[i]), &kr, &ki);
                    last_w = h->hw[i];
                }
                hks[i] = kr;
                ksi[i] = ki;
            }
            upload(h->kself, hks, st);
            upload(h->kself_im, ksi, st);
        } else {
            HIF_CUDA(launch_kself(geom(h.get()), h->kself.as<double>(), st));
            HIF_CUDA(cudaMemcpyAsync(hks.data(), h->kself.p, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        }
        HIF_CUDA(cudaStreamSynchronize(st));
        for (auto& sp : h->segs) {
            Segment& sg = *sp;
            if (h->ncomp == 2) continue;               // no grid convolution for the complex kernel
            detect_grid(h.get(), sg);
            if (!sg.grid) continue;
            const int64_t tsz = d == 2 ? (int64_t)sg.gn * sg.gn : (int64_t)sg.gn * sg.gn * sg.gn;
            sg.table.ensure(sizeof(double) * tsz);
            HIF_CUDA(launch_grid_table(sg.table.as<double>(), sg.gn, d, sg.gh, kernel_id,
                                       hks[sg.off] / h->hw[sg.off], st));
            sg.spread = table_spread(sg.gn, d, sg.gh, kernel_id, hks[sg.off] / h->hw[sg.off]);
            sg.table_df.ensure(sizeof(float2) * tsz);
            HIF_CUDA(launch_split_df(sg.table.as<double>(), sg.table_df.as<float2>(), tsz, st));
        }
        h->stats.N = N;
        h->stats.dim = d;
        if (h->precision == 0) {
            run_factor<double>(h.get());
            prepare_sweeps<double>(h.get());
        } else {
            run_factor<float>(h.get());
            prepare_sweeps<float>(h.get());
        }
        HIF_CUDA(cudaStreamSynchronize(st));
    });
    if (s != HIF_OK) return s;
    h->stats.factor_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = h.release();
    return HIF_OK;
}

hif_status hif_factor(const double* points, int64_t N, const double* weights, const double* a, const double* b,
                      const double* c, int kernel_id, double eps, const hif_options* opt, hif_handle* out) {
    const hif_problem pr{points, N, weights, a, b, c};
    return factor_impl(1, &pr, kernel_id, eps, opt, out);
}

hif_status hif_factor_batched(int count, const hif_problem* problems, int kernel_id, double eps,
                              const hif_options* opt, hif_handle* out) {
    return factor_impl(count, problems, kernel_id, eps, opt, out);
}

hif_status hif_apply(hif_handle h, const double* x, double* y, int64_t nrhs, int64_t ld) {
    return guard([&] { apply_op(h, x, y, nrhs, ld, 1); });
}
hif_status hif_apply_transpose(hif_handle h, const double* x, double* y, int64_t nrhs, int64_t ld) {
    return guard([&] { apply_op(h, x, y, nrhs, ld, 3); });
}
hif_status hif_solve(hif_handle h, const double* bb, double* x, int64_t nrhs, int64_t ld) {
    return guard([&] { apply_op(h, bb, x, nrhs, ld, 0); });
}
hif_status hif_solve_transpose(hif_handle h, const double* bb, double* x, int64_t nrhs, int64_t ld) {
    return guard([&] { apply_op(h, bb, x, nrhs, ld, 2); });
}

hif_status hif_matvec(hif_handle h, int trans, const double* x, double* y, int64_t nrhs, int64_t ld) {
    if (!h || !x || !y || nrhs < 0 || ld < (h ? h->N : 0)) return HIF_EINVAL;
    if (nrhs == 0) return HIF_OK;
    return guard([&] {
        with_dev_io(h, x, y, nrhs, ld, [&](const double* dx, double* dy) {
            matvec_dev(h, trans ? 1 : 0, dx, h->N, dy, h->N, (int)nrhs);
        });
    });
}

hif_status hif_matvec_digits(hif_handle h, int trans, int classes, const double* x, double* y, int64_t nrhs,
                             int64_t ld) {
    if (!h || !x || !y || nrhs < 0 || ld < (h ? h->N : 0) || classes < 4 || classes == 7 || classes > 8) {
        std::snprintf(g_last_error, sizeof(g_last_error), "%s",
                      "hif_matvec_digits: invalid argument (classes must be 4, 5, 6 or 8)");
        return HIF_EINVAL;
    }
    if (nrhs == 0) return HIF_OK;
    return guard([&] {
        with_dev_io(h, x, y, nrhs, ld, [&](const double* dx, double* dy) {
            matvec_dev(h, trans ? 1 : 0, dx, h->N, dy, h->N, (int)nrhs, classes);
        });
    });
}

hif_status hif_solve_refined(hif_handle h, int trans, const double* f, double* u, int64_t nrhs, int64_t ld, double tol,
                             int maxit, int method, int* iters, double* relres) {
    if (!h || !f || !u || nrhs < 0 || ld < (h ? h->N : 0) || !(tol > 0) || maxit < 0 || (method != 0 && method != 1))
        return HIF_EINVAL;
    if (nrhs == 0) return HIF_OK;
    hif_status res = HIF_OK;
    hif_status s = guard([&] {
        with_dev_io(h, f, u, nrhs, ld, [&](const double* df, double* du) {
            res = method == 0 ? refine_ir(h, trans ? 1 : 0, df, du, (int)nrhs, tol, maxit, iters, relres)
                              : refine_gmres(h, trans ? 1 : 0, df, du, (int)nrhs, tol, maxit, iters, relres);
        });
    });
    return s != HIF_OK ? s : res;
}

hif_status hif_adjoint_gradients(hif_handle h, const double* u, const double* lam, int64_t nrhs, int64_t ld,
                                 double* grad_a, double* grad_b, double* grad_c) {
    if (!h || !u || !lam || !grad_a || !grad_b || !grad_c || nrhs < 1 || ld < h->N || nrhs > (1 << 20))
        return HIF_EINVAL;
    if (h->ncomp != 1) {
        std::snprintf(g_last_error, sizeof(g_last_error), "hif_adjoint_gradients: real kernels only");
        return HIF_EINVAL;
    }
    return guard([&] {
        const int64_t N = h->N;
        const cudaStream_t st = h->st;
        const int nr = (int)nrhs;
        DevMem U, Lm, Fu, Ftl, G;
        U.ensure(sizeof(double) * N * nr);
        Lm.ensure(sizeof(double) * N * nr);
        Fu.ensure(sizeof(double) * N * nr);
        Ftl.ensure(sizeof(double) * N * nr);
        G.ensure(sizeof(double) * N * 3);
        HIF_CUDA(cudaMemcpy2DAsync(U.p, sizeof(double) * N, u, sizeof(double) * ld, sizeof(double) * N, nr,
                                   is_device_ptr(u) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        HIF_CUDA(cudaMemcpy2DAsync(Lm.p, sizeof(double) * N, lam, sizeof(double) * ld, sizeof(double) * N, nr,
                                   is_device_ptr(lam) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        fac_dev(h, 1, U.as<double>(), Fu.as<double>(), nr);       // F u
        fac_dev(h, 3, Lm.as<double>(), Ftl.as<double>(), nr);     // F^T lambda
        h->status.ensure(sizeof(int));
        HIF_CUDA(cudaMemsetAsync(h->status.p, 0, sizeof(int), st));
        double* g = G.as<double>();
        HIF_CUDA(launch_adjoint_coef(N, nr, h->a.as<double>(), h->b.as<double>(), h->c.as<double>(), U.as<double>(),
                                     Lm.as<double>(), Fu.as<double>(), Ftl.as<double>(), g, g + N, g + 2 * N,
                                     h->status.as<int>(), st));
        int bad = 0;
        HIF_CUDA(cudaMemcpyAsync(&bad, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        double* outs[3] = {grad_a, grad_b, grad_c};
        for (int q = 0; q < 3; ++q)
            HIF_CUDA(cudaMemcpyAsync(outs[q], g + q * N, sizeof(double) * N,
                                     is_device_ptr(outs[q]) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        HIF_CUDA(cudaStreamSynchronize(st));
        if (bad) fail(HIF_EINVAL, "adjoint gradients need nonzero b and c");
    });
}

hif_status hif_error_estimates(hif_handle h, const double* v0, double rtol, int maxit, double* norms, int* iters) {
    if (!h || !v0 || !norms || !(rtol > 0) || maxit < 1) return HIF_EINVAL;
    bool all = true;
    const hif_status s = guard([&] {
        int its[3];
        all = power_norms_dev(h, v0, rtol, maxit, norms, its);
        if (iters)
            for (int c = 0; c < 3; ++c) iters[c] = its[c];
    });
    if (s != HIF_OK) return s;
    return all ? HIF_OK : HIF_ENOTCONV;
}

hif_status hif_eliminated_dofs(hif_handle h, int sublevel, int* out, int64_t cap, int64_t* count) {
    if (!h || !count || sublevel < 0 || sublevel >= (int)h->subs.size()) return HIF_EINVAL;
    const SubFactor& sf = *h->subs[sublevel];
    int64_t n = 0;
    for (const BoxFac& b : sf.hbox) n += b.r;
    *count = n;
    if (!out) return HIF_OK;
    if (cap < n) return HIF_EINVAL;
    return guard([&] {
        if (n == 0) return;
        HIF_CUDA(cudaMemcpyAsync(out, sf.rd.p, sizeof(int) * n,
                                 is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
        HIF_CUDA(cudaStreamSynchronize(h->st));
    });
}

hif_status hif_stats(hif_handle h, hif_stats_t* st) {
    if (!h || !st) return HIF_EINVAL;
    *st = h->stats;
    return HIF_OK;
}

hif_status hif_destroy(hif_handle h) {
    if (!h) return HIF_OK;
    if (h->st) cudaStreamSynchronize(h->st);
    else cudaDeviceSynchronize();
    delete h;
    return HIF_OK;
}

hif_status hif_kernel_block(const double* points, int64_t N, int dim, const double* weights, const double* a,
                            const double* b, const double* c, int kernel_id, const int32_t* rows, int64_t nr,
                            const int32_t* cols, int64_t nc, double* out, int64_t ldo, void* stream) {
    if (N <= 0 || (dim != 2 && dim != 3) || (kernel_id != 0 && kernel_id != 1) || nr < 0 || nc < 0 || ldo < nr ||
        !points || !weights || !a || !b || !c || !rows || !cols || !out)
        return HIF_EINVAL;
    return guard([&] {
        const cudaStream_t st = static_cast<cudaStream_t>(stream);
        InArr px, pw, pa, pb, pc;
        px.set(points, (size_t)N * dim, st);
        pw.set(weights, N, st);
        pa.set(a, N, st);
        pb.set(b, N, st);
        pc.set(c, N, st);
        DevMem dr, dc, dk, dout;
        const int* drp = rows;
        const int* dcp = cols;
        if (!is_device_ptr(rows)) {
            dr.ensure(sizeof(int) * std::max<int64_t>(nr, 1));
            if (nr) HIF_CUDA(cudaMemcpyAsync(dr.p, rows, sizeof(int) * nr, cudaMemcpyHostToDevice, st));
            drp = dr.as<int>();
        }
        if (!is_device_ptr(cols)) {
            dc.ensure(sizeof(int) * std::max<int64_t>(nc, 1));
            if (nc) HIF_CUDA(cudaMemcpyAsync(dc.p, cols, sizeof(int) * nc, cudaMemcpyHostToDevice, st));
            dcp = dc.as<int>();
        }
        dk.ensure(sizeof(double) * N);
        GeomDev g{px.d, pw.d, pa.d, pb.d, pc.d, dk.as<double>(), nullptr, 0.0, N, dim, kernel_id, 1};
        HIF_CUDA(launch_kself(g, dk.as<double>(), st));
        const bool dev_out = is_device_ptr(out);
        double* o = out;
        if (!dev_out) {
            dout.ensure(sizeof(double) * std::max<int64_t>(ldo * nc, 1));
            o = dout.as<double>();
        }
        HIF_CUDA(launch_kernel_block(g, drp, nr, dcp, nc, o, ldo, st));
        if (!dev_out && nr > 0 && nc > 0)
            HIF_CUDA(cudaMemcpyAsync(out, o, sizeof(double) * ldo * nc, cudaMemcpyDeviceToHost, st));
        HIF_CUDA(cudaStreamSynchronize(st));
    });
}

hif_status hif_gemm_batched_f32(int count, const hif_gemm_problem* problems, void* stream) {
    g_last_error[0] = 0;
    if (count < 0 || (count > 0 && !problems)) {
        std::snprintf(g_last_error, sizeof(g_last_error), "hif_gemm_batched_f32: %s",
                      count < 0 ? "negative count" : "NULL problem array");
        return HIF_EINVAL;
    }
    std::vector<TcGemmProb> hp;
    int max_m = 0, max_n = 0;
    for (int i = 0; i < count; ++i) {
        const hif_gemm_problem& q = problems[i];
        const int64_t ra = q.trans_a ? q.k : q.m, rb = q.trans_b ? q.n : q.k;
        const bool bad = q.m < 0 || q.n < 0 || q.k < 0 || (q.beta != 0 && q.beta != 1) ||
                         (q.m > 0 && q.n > 0 && (!q.C || q.ldc < std::max(1, q.m))) ||
                         (q.m > 0 && q.n > 0 && q.k > 0 &&
                          (!q.A || !q.B || q.lda < std::max<int64_t>(1, ra) || q.ldb < std::max<int64_t>(1, rb)));
        if (bad) {
            std::snprintf(g_last_error, sizeof(g_last_error), "hif_gemm_batched_f32: problem %d is invalid", i);
            return HIF_EINVAL;
        }
        if (q.m == 0 || q.n == 0 || (q.k == 0 && q.beta == 1)) continue;
        hp.push_back(TcGemmProb{q.A, q.B, q.C, q.lda, q.ldb, q.ldc, q.m, q.n, q.k, q.trans_a ? 1 : 0,
                                q.trans_b ? 1 : 0, q.alpha, q.beta});
        max_m = std::max(max_m, q.m);
        max_n = std::max(max_n, q.n);
    }
    if (hp.empty()) return HIF_OK;
    return guard([&] {
        const cudaStream_t st = static_cast<cudaStream_t>(stream);
        DevMem dp, ds;
        dp.ensure(sizeof(TcGemmProb) * hp.size());
        ds.ensure(sizeof(int));
        HIF_CUDA(cudaMemsetAsync(ds.p, 0, sizeof(int), st));
        HIF_CUDA(cudaMemcpyAsync(dp.p, hp.data(), sizeof(TcGemmProb) * hp.size(), cudaMemcpyHostToDevice, st));
        for (size_t off = 0; off < hp.size(); off += 65535) {
            const int cnt = (int)std::min<size_t>(65535, hp.size() - off);
            HIF_CUDA(launch_tc_gemm(dp.as<TcGemmProb>() + off, cnt, max_m, max_n, ds.as<int>(), 1, st));
        }
        int flag = 0;
        HIF_CUDA(cudaMemcpyAsync(&flag, ds.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        HIF_CUDA(cudaStreamSynchronize(st));
        if (flag) fail(HIF_ETIMEOUT, "hif_gemm_batched_f32: a bounded wait of the kernel ran out");
    });
}

hif_status hif_id_batched(int count, const double* mats, const int64_t* off, const int32_t* m, const int32_t* n,
                          const double* tol, int32_t* k, int32_t* perm, const int64_t* poff, double* T,
                          const int64_t* toff, void* stream) {
    if (count < 0 || !mats || !off || !m || !n || !tol || !k || !perm || !poff || !T || !toff) return HIF_EINVAL;
    if (count == 0) return HIF_OK;
    return guard([&] {
        const cudaStream_t st = static_cast<cudaStream_t>(stream);
        // all metadata to the device; matrices may be host or device
        std::vector<int64_t> hoff(off, off + count), hpoff(poff, poff + count), htoff(toff, toff + count);
        std::vector<int> hm(m, m + count), hn(n, n + count);
        int64_t mat_end = 0, perm_end = 0, t_end = 0;
        for (int i = 0; i < count; ++i) {
            if (hm[i] < 0 || hn[i] < 0) fail(HIF_EINVAL, "negative size");
            mat_end = std::max(mat_end, hoff[i] + (int64_t)hm[i] * hn[i]);
            perm_end = std::max(perm_end, hpoff[i] + hn[i]);
            t_end = std::max(t_end, htoff[i] + (int64_t)hn[i] * hn[i] / 4 + hn[i]);
        }
        std::vector<double> htol(tol, tol + count);
        DevMem dmats, doff, dm, dn, dtol, dk, dperm, dpoff, dT, dtoff;
        const double* mp = mats;
        if (!is_device_ptr(mats)) {
            dmats.ensure(sizeof(double) * std::max<int64_t>(mat_end, 1));
            HIF_CUDA(cudaMemcpyAsync(dmats.p, mats, sizeof(double) * mat_end, cudaMemcpyHostToDevice, st));
            mp = dmats.as<double>();
        }
        upload(doff, hoff, st);
        upload(dm, hm, st);
        upload(dn, hn, st);
        upload(dtol, htol, st);
        upload(dpoff, hpoff, st);
        upload(dtoff, htoff, st);
        dk.ensure(sizeof(int) * count);
        dperm.ensure(sizeof(int) * std::max<int64_t>(perm_end, 1));
        dT.ensure(sizeof(double) * std::max<int64_t>(t_end, 1));
        HIF_CUDA(launch_id_batched(count, mp, doff.as<int64_t>(), dm.as<int>(), dn.as<int>(), dtol.as<double>(),
                                   dk.as<int>(), dperm.as<int>(), dpoff.as<int64_t>(), dT.as<double>(),
                                   dtoff.as<int64_t>(), st));
        const bool dk_dev = is_device_ptr(k), dp_dev = is_device_ptr(perm), dt_dev = is_device_ptr(T);
        HIF_CUDA(cudaMemcpyAsync(k, dk.p, sizeof(int) * count, dk_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        HIF_CUDA(cudaMemcpyAsync(perm, dperm.p, sizeof(int) * perm_end,
                                 dp_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        HIF_CUDA(cudaMemcpyAsync(T, dT.p, sizeof(double) * t_end, dt_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        HIF_CUDA(cudaStreamSynchronize(st));
    });
}

}  // extern "C"

extern "C" {

hif_status hif_id_batched_noalloc(int count, const double* mats, const int64_t* off, const int32_t* m,
                                  const int32_t* n, const double* tol, int32_t* k, int32_t* perm,
                                  const int64_t* poff, double* T, const int64_t* toff, void* stream) {
    g_last_error[0] = '\0';
    if (count < 0) {
        std::snprintf(g_last_error, sizeof(g_last_error), "hif_id_batched_noalloc: negative count %d", count);
        return HIF_EINVAL;
    }
    if (!mats || !off || !m || !n || !tol || !k || !perm || !poff || !T || !toff) {
        std::snprintf(g_last_error, sizeof(g_last_error), "hif_id_batched_noalloc: a required array is NULL");
        return HIF_EINVAL;
    }
    if (count == 0) return HIF_OK;
    const void* ptrs[] = {mats, off, m, n, tol, k, perm, poff, T, toff};
    for (const void* p : ptrs) {
        if (!is_device_ptr(p)) {
            std::snprintf(g_last_error, sizeof(g_last_error),
                          "hif_id_batched_noalloc: every array must be device memory");
            return HIF_EINVAL;
        }
    }
    int too_big = 0;
    const cudaError_t e = launch_id_batched_noalloc(count, mats, off, m, n, tol, k, perm, poff, T, toff,
                                                    static_cast<cudaStream_t>(stream), &too_big);
    if (e != cudaSuccess) {
        std::snprintf(g_last_error, sizeof(g_last_error), "hif_id_batched_noalloc: %s", cudaGetErrorString(e));
        return HIF_ECUDA;
    }
    if (too_big) {
        std::snprintf(g_last_error, sizeof(g_last_error),
                      "hif_id_batched_noalloc: input exceeds the fixed work space (at most 4096 matrices, "
                      "1024 columns each, sum over matrices of (m|1)*n <= 1048576 doubles)");
        return HIF_EINVAL;
    }
    return HIF_OK;
}

}  // extern "C"
