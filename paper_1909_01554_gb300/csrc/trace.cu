// Tracing: a CUDA event pair around every kernel launch while enabled (on the
// launching stream), summed per phase on demand; and a launch counter.
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"

namespace bmm {
namespace {

struct Rec {
    int phase;
    cudaEvent_t a, b;
};

std::mutex g_mu;
std::vector<Rec> g_recs;
std::atomic<bool> g_on{false};
std::atomic<int64_t> g_launches{0};

}  // namespace

void trace_launch_begin(int phase, cudaStream_t s, void** token) {
    *token = nullptr;
    if (!g_on.load(std::memory_order_relaxed)) return;
    Rec* r = new Rec{phase, nullptr, nullptr};
    if (cudaEventCreate(&r->a) != cudaSuccess || cudaEventCreate(&r->b) != cudaSuccess) {
        cudaGetLastError();
        delete r;
        return;
    }
    cudaEventRecord(r->a, s);
    *token = r;
}

void trace_launch_end(void* token, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!token) return;
    Rec* r = (Rec*)token;
    cudaEventRecord(r->b, s);
    std::lock_guard<std::mutex> lk(g_mu);
    g_recs.push_back(*r);
    delete r;
}

}  // namespace bmm

using namespace bmm;

extern "C" {

void bmm_trace_enable(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (enable) {
        for (auto& r : g_recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        g_recs.clear();
    }
    g_on.store(enable != 0);
}

bmm_status bmm_trace_read(int32_t phase, int64_t* launches, double* milliseconds) {
    if (phase < 0 || phase >= BMM_PHASE_COUNT || !launches || !milliseconds)
        return BMM_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    int64_t cnt = 0;
    double ms = 0.0;
    for (auto& r : g_recs) {
        if (r.phase != phase) continue;
        BMM_CUDA_TRY(cudaEventSynchronize(r.b));
        float t = 0.f;
        BMM_CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
        ms += t;
        cnt++;
    }
    *launches = cnt;
    *milliseconds = ms;
    return BMM_OK;
}

int64_t bmm_launch_count(void) { return g_launches.load(); }

}  // extern "C"
