// profile.cu -- launch counting and CUDA-event timing of kernel classes
// (measurement support for the benchmark; no counterpart in the paper).
#include <atomic>
#include <mutex>
#include <string.h>
#include <vector>

#include "pts_internal.cuh"

namespace pts {
namespace {

const char *kNames[kProfClasses] = {"search_topk", "search_full", "rerank", "project", "m_step",
                                    "search_tc", "mlp", "probe", "brute", "irls"};
std::atomic<long long> g_launches{0};
std::atomic<int> g_enabled{0};
std::mutex g_mu;
struct Rec {
    cudaEvent_t a, b;
};
std::vector<Rec> g_recs[kProfClasses];
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void clear_records() {
    for (auto &v : g_recs) {
        for (auto &r : v) {
            g_pool.push_back(r.a);
            g_pool.push_back(r.b);
        }
        v.clear();
    }
}

}  // namespace

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Event timing is switched off while a CUDA graph is being captured (an event recorded into a
// capture would become a graph node, not a timing point); on = true restores the previous state.
void prof_suspend(bool on) {
    static int saved = 0;
    if (!on) {
        saved = g_enabled.exchange(0);
    } else {
        g_enabled.store(saved);
    }
}

void prof_begin(int cls, cudaStream_t st, void **token) {
    *token = nullptr;
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t a = get_event();
    cudaEventRecord(a, st);
    *token = a;
    (void)cls;
}

void prof_end(int cls, cudaStream_t st, void *token) {
    if (!token) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = get_event();
    cudaEventRecord(b, st);
    g_recs[cls].push_back({reinterpret_cast<cudaEvent_t>(token), b});
}

}  // namespace pts

extern "C" {

long long pts_launch_count(void) { return pts::g_launches.load(); }

void pts_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(pts::g_mu);
    pts::clear_records();
    pts::g_enabled.store(on ? 1 : 0);
}

pts_status pts_profile_read(const char *kernel, double *total_ms, long long *launches) {
    if (!kernel || !total_ms || !launches)
        return pts::set_error(PTS_ERR_INVALID_ARG, "pts_profile_read: null pointer");
    int cls = -1;
    for (int i = 0; i < pts::kProfClasses; ++i)
        if (strcmp(kernel, pts::kNames[i]) == 0) cls = i;
    if (cls < 0) return pts::set_error(PTS_ERR_INVALID_ARG, "pts_profile_read: unknown kernel class");
    std::lock_guard<std::mutex> lk(pts::g_mu);
    double ms = 0.0;
    for (auto &r : pts::g_recs[cls]) {
        PTS_CUDA_TRY(cudaEventSynchronize(r.b));
        float t = 0.0f;
        PTS_CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
        ms += t;
    }
    *total_ms = ms;
    *launches = (long long)pts::g_recs[cls].size();
    return PTS_OK;
}

}  // extern "C"
