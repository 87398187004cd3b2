// profile.cu -- launch counting and CUDA-event timing of kernel classes
// (measurement support for the benchmark; no counterpart in the paper).
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string.h>
#include <vector>

#include "pts_internal.cuh"

namespace pts {
namespace {

const char *kNames[kProfClasses] = {"search_topk", "search_full", "rerank", "project", "m_step",
                                    "search_tc", "mlp", "probe", "brute", "irls", "search_tc_list", "search_tcf"};
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

// 8 independent FMA chains per thread, 16 steps unrolled per iteration; a and b keep the values
// bounded (|a| < 1).  The sum is stored only when it equals a value it cannot reach, which keeps
// every chain live without a store per thread.
__global__ void __launch_bounds__(1024, 2) k_fma_peak(int iters, float a, float b, float never, float *out) {
    float x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    if (s == never) out[blockIdx.x] = s;
}

}  // namespace

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_smem_attr(const void *kernel, int bytes) {
    struct Done {
        const void *kernel;
        int device, bytes;
    };
    static std::mutex mu;
    static std::vector<Done> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    for (const Done &d : done)
        if (d.kernel == kernel && d.device == dev && d.bytes >= bytes) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done.push_back({kernel, dev, bytes});
}

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

pts_status pts_fp32_fma_peak(int iters, int reps, void *stream, double *tflops, double *best_ms) {
    if (!tflops || !best_ms || iters < 1 || iters > 1000000 || reps < 1 || reps > 100)
        return pts::set_error(PTS_ERR_INVALID_ARG, "pts_fp32_fma_peak: iters in 1..1e6, reps in 1..100, outputs non-null");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    PTS_CUDA_TRY(cudaGetDevice(&dev));
    PTS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 2 * sms;
    pts::DevBuf<float> out;
    PTS_TRY(out.ensure((size_t)blocks, "fma probe output"));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PTS_CUDA_TRY(cudaEventCreate(&e0));
    PTS_CUDA_TRY(cudaEventCreate(&e1));
    double best = 1e30;
    pts_status rc = PTS_OK;
    for (int r = 0; r <= reps && rc == PTS_OK; ++r) {  // the first launch is a warm-up
        pts::count_launches(1);
        cudaEventRecord(e0, st);
        pts::k_fma_peak<<<blocks, 1024, 0, st>>>(iters, 0.999f, 1e-3f, -1.0f, out.ptr);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = pts::set_error(PTS_ERR_CUDA, "pts_fp32_fma_peak: launch failed");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = std::min(best, (double)ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out.release();
    if (rc != PTS_OK) return rc;
    const double fmas = (double)blocks * 1024.0 * 8.0 * 16.0 * iters;
    *best_ms = best;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return PTS_OK;
}

}  // extern "C"
