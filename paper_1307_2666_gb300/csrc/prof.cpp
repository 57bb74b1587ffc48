// Per-kernel-family CUDA-event timing (see prof.h).
#include "prof.h"

#include <atomic>
#include <mutex>
#include <vector>

namespace hif {

namespace {
struct Rec {
    int kind;
    cudaEvent_t e0, e1;
};
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Rec> g_recs;
double g_flops[PROF_COUNT] = {};
double g_bytes[PROF_COUNT] = {};
const char* const kNames[PROF_COUNT] = {
    "fold_kernel", "id_kernel", "elim_kernel", "big_ygen_kernel", "big_rho", "big_qr_step",
    "big_T_kernel", "big_elim_batch", "sweep", "direct_sum", "direct_sum_short"};
}  // namespace

bool prof_enabled() { return g_on.load(std::memory_order_relaxed); }

void prof_set(bool enable) { g_on.store(enable, std::memory_order_relaxed); }

const char* prof_name(int kind) { return kind >= 0 && kind < PROF_COUNT ? kNames[kind] : "?"; }

void prof_add_work(int kind, double flops, double bytes) {
    if (!prof_enabled() || kind < 0 || kind >= PROF_COUNT) return;
    std::lock_guard<std::mutex> lk(g_mu);
    g_flops[kind] += flops;
    g_bytes[kind] += bytes;
}

ProfRange::ProfRange(int kind, cudaStream_t st, double flops, double bytes) : kind_(kind), st_(st) {
    if (!prof_enabled() || kind < 0 || kind >= PROF_COUNT) return;
    // a stream being captured into a graph cannot take timing events
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (cudaEventCreate(&e0_) != cudaSuccess) { e0_ = nullptr; return; }
    if (cudaEventRecord(e0_, st) != cudaSuccess) {
        cudaEventDestroy(e0_);
        e0_ = nullptr;
        return;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_flops[kind] += flops;
    g_bytes[kind] += bytes;
}

ProfRange::~ProfRange() {
    if (!e0_) return;
    cudaEvent_t e1 = nullptr;
    if (cudaEventCreate(&e1) != cudaSuccess || cudaEventRecord(e1, st_) != cudaSuccess) {
        if (e1) cudaEventDestroy(e1);
        cudaEventDestroy(e0_);
        return;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_recs.push_back({kind_, e0_, e1});
}

cudaError_t prof_collect(int64_t* ranges, double* ms, double* flops, double* bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < PROF_COUNT; ++k) {
        ranges[k] = 0;
        ms[k] = 0.0;
        flops[k] = g_flops[k];
        bytes[k] = g_bytes[k];
        g_flops[k] = g_bytes[k] = 0.0;
    }
    for (const Rec& r : g_recs) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.e0, r.e1);
        if (e != cudaSuccess && err == cudaSuccess) err = e;
        ranges[r.kind] += 1;
        ms[r.kind] += t;
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    g_recs.clear();
    return err;
}

}  // namespace hif
