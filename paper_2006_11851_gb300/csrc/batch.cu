// batch.cu -- many independent synthesis jobs (one level each, uneven sizes) as one CUDA graph
// (the batched form of the EM loop of section 2.1; no counterpart in the paper).
//
// pts_batch_create runs one search per job to size every workspace the job's mode touches,
// autotunes the tensor-core search's exemplar split per job shape (the candidate with the least
// measured time, cached by shape), then captures all jobs' iterations -- search, IRLS weights
// and energy, M-step -- into one graph, the jobs spread round-robin over n_streams forked
// streams (jobs are independent: each has its own index and workspace).  A job chained to a
// parent (a pyramid's next level) runs on its parent's stream after it, starting from the
// parent's result up-sampled by 2.  Any search mode whose tables the job's index holds may run
// (exact, FP16, FP8, the learned proposal, the k-means tree).  pts_batch_run replays the graph.
// Energies go to device arrays so the graph has no host copy or synchronisation.
#include <algorithm>
#include <map>
#include <string>
#include <mutex>
#include <tuple>
#include <vector>

#include "pts_internal.cuh"

struct pts_batch_s {
    std::vector<pts_job> jobs;
    std::vector<int> parts;
    int iters = 0;
    float r = 2.0f, delta = 1e-3f;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    // each job's index generation when the graph was captured: the graph holds raw pointers into
    // the index's tables and workspace, so a run is refused once any of them has moved
    std::vector<unsigned long long> gens;
};

namespace pts {
namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tune_cache;  // (device, N, Q, K, mode) -> parts

int job_queries(const pts_job &j) {
    const int w = j.index->w;
    return ((j.Ho - w) / j.stride + 1) * ((j.Wo - w) / j.stride + 1);
}

// A CUDA event destroyed with its scope (so an early error return leaks nothing).
struct ScopedEvent {
    cudaEvent_t e = nullptr;
    ~ScopedEvent() {
        if (e) cudaEventDestroy(e);
    }
};

// Times `reps` searches of the job's image with the given exemplar split (ms per search).
pts_status time_search(const pts_job &j, int parts, int reps, cudaStream_t st, float *ms) {
    pts_index idx = j.index;
    Workspace &ws = idx->ws;
    idx->tc_parts_override = parts;
    PTS_TRY(nn_search_impl(idx, j.output, j.Ho, j.Wo, j.stride, j.mode, ws.nn.ptr, ws.d2.ptr, st));
    ScopedEvent a, b;
    PTS_CUDA_TRY(cudaEventCreate(&a.e));
    PTS_CUDA_TRY(cudaEventCreate(&b.e));
    PTS_CUDA_TRY(cudaEventRecord(a.e, st));
    for (int k = 0; k < reps; ++k)
        PTS_TRY(nn_search_impl(idx, j.output, j.Ho, j.Wo, j.stride, j.mode, ws.nn.ptr, ws.d2.ptr, st));
    PTS_CUDA_TRY(cudaEventRecord(b.e, st));
    PTS_CUDA_TRY(cudaEventSynchronize(b.e));
    float t = 0.0f;
    PTS_CUDA_TRY(cudaEventElapsedTime(&t, a.e, b.e));
    *ms = t / reps;
    return PTS_OK;
}

pts_status autotune(pts_batch b, cudaStream_t st) {
    for (size_t k = 0; k < b->jobs.size(); ++k) {
        const pts_job &j = b->jobs[k];
        pts_index idx = j.index;
        if (j.mode != PTS_F16_RERANK && j.mode != PTS_FP8_RERANK) {
            b->parts[k] = 0;
            continue;
        }
        const int Q = job_queries(j), ntc = tc_tiles(idx->N);
        const int K = j.mode == PTS_F16_RERANK ? idx->ktc : idx->kf8;
        const auto key = std::make_tuple(idx->device, idx->N, Q, K, j.mode);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                b->parts[k] = it->second;
                idx->tc_parts_override = it->second;
                // one search with the cached plan still sizes this job's buffers
                PTS_TRY(nn_search_impl(idx, j.output, j.Ho, j.Wo, j.stride, j.mode, idx->ws.nn.ptr,
                                       idx->ws.d2.ptr, st));
                continue;
            }
        }
        // candidates: automatic (the default rule with its tail split) and splits of 1, 2 and 4
        // parts (each part >= 16 tiles)
        std::vector<int> cand = {0, 1, 2, 4};
        int best = cand[0];
        float best_ms = 1e30f;
        for (int p : cand) {
            if (p > 1 && ntc / p < 16) continue;
            float ms = 0.0f;
            PTS_TRY(time_search(j, p, 2, st, &ms));
            if (ms < best_ms) {
                best_ms = ms;
                best = p;
            }
        }
        idx->tc_parts_override = best;
        b->parts[k] = best;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    return PTS_OK;
}

}  // namespace
}  // namespace pts

using namespace pts;

extern "C" {

pts_status pts_batch_create(const pts_job *jobs, int n_jobs, int iters, float r, float delta, int n_streams,
                            int tune, void *stream, pts_batch *out) {
    if (!jobs || !out || n_jobs <= 0) return set_error(PTS_ERR_INVALID_ARG, "pts_batch_create: no jobs");
    if (iters < 0 || !(r > 0.0f && r <= 2.0f) || !(delta > 0.0f))
        return set_error(PTS_ERR_INVALID_ARG, "pts_batch_create: need iters >= 0, 0 < r <= 2, delta > 0");
    if (n_streams < 1 || n_streams > 64) return set_error(PTS_ERR_INVALID_ARG, "pts_batch_create: 1..64 streams");
    *out = nullptr;
    for (int k = 0; k < n_jobs; ++k) {
        const pts_job &j = jobs[k];
        if (!j.index || !j.output || !j.energy) return set_error(PTS_ERR_INVALID_ARG, "pts_batch_create: null job field");
        unsigned long long g = 0;
        if (!index_generation(j.index, &g))
            return set_error(PTS_ERR_INVALID_ARG, "pts_batch_create: a job's index is not a live index");
        if (j.mode < PTS_EXACT_F32 || j.mode > PTS_EXACT_TC)
            return set_error(PTS_ERR_INVALID_ARG, "pts_batch_create: unknown job mode");
        if (j.mode == PTS_PROPOSAL && !j.index->prop.ready)
            return set_error(PTS_ERR_INVALID_ARG, "pts_batch_create: a proposal job's index has no trained proposal");
        if (j.mode == PTS_KMTREE && !j.index->tree.ready)
            return set_error(PTS_ERR_INVALID_ARG, "pts_batch_create: a tree job's index has no k-means tree");
        if (j.parent < -1 || j.parent >= k)
            return set_error(PTS_ERR_INVALID_ARG, "pts_batch_create: a parent must be an earlier job (or -1)");
        if (j.parent >= 0) {
            const pts_job &pj = jobs[j.parent];
            if (j.index->C != 3 || pj.index->C != 3 || 2 * pj.Ho != j.Ho || 2 * pj.Wo != j.Wo)
                return set_error(PTS_ERR_INVALID_ARG,
                                 "pts_batch_create: a chained job needs RGB indices and twice its parent's size");
        }
        PTS_TRY(check_grid_public(j.Ho, j.Wo, j.index->w, j.stride, "pts_batch_create"));
        for (int m = 0; m < k; ++m)
            if (jobs[m].index == j.index)
                return set_error(PTS_ERR_INVALID_ARG, "pts_batch_create: two jobs share an index (its workspace)");
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    pts_batch b = new pts_batch_s();
    b->jobs.assign(jobs, jobs + n_jobs);
    b->parts.assign(n_jobs, 0);
    b->iters = iters;
    b->r = r;
    b->delta = delta;
    // the autotuner sets each index's split for the capture; the caller's settings come back after
    std::vector<int> saved_parts(n_jobs);
    for (int k = 0; k < n_jobs; ++k) saved_parts[k] = jobs[k].index->tc_parts_override;
    auto restore_parts = [&]() {
        for (int k = 0; k < n_jobs; ++k) jobs[k].index->tc_parts_override = saved_parts[k];
    };
    auto fail = [&](pts_status s) {
        restore_parts();
        pts_batch_destroy(b);
        return s;
    };
    // size every buffer a job touches (a capture must not allocate), then tune the split
    for (const pts_job &j : b->jobs) {
        pts_index idx = j.index;
        pts_status s = ensure_workspace(idx, job_queries(j));
        if (s == PTS_OK) s = nn_search_impl(idx, j.output, j.Ho, j.Wo, j.stride, j.mode, idx->ws.nn.ptr, idx->ws.d2.ptr, st);
        if (s != PTS_OK) return fail(s);
    }
    if (tune) {
        pts_status s = autotune(b, st);
        if (s != PTS_OK) return fail(s);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(set_error(PTS_ERR_CUDA, "pts_batch_create: sync"));

    // capture: fork the jobs over n_streams streams and join them back
    std::vector<cudaStream_t> ss(n_streams, nullptr);
    std::vector<cudaEvent_t> ev(n_streams + 1, nullptr);
    cudaStream_t cap = nullptr;
    pts_status s = PTS_OK;
    bool capturing = false;
    do {
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
            s = set_error(PTS_ERR_CUDA, "pts_batch_create: stream");
            break;
        }
        for (int i = 0; i < n_streams && s == PTS_OK; ++i)
            if (cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking) != cudaSuccess)
                s = set_error(PTS_ERR_CUDA, "pts_batch_create: stream");
        for (int i = 0; i <= n_streams && s == PTS_OK; ++i)
            if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess)
                s = set_error(PTS_ERR_CUDA, "pts_batch_create: event");
        if (s != PTS_OK) break;
        prof_suspend(false);
        const long long l0 = pts_launch_count();
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            prof_suspend(true);
            s = set_error(PTS_ERR_CUDA, "pts_batch_create: begin capture");
            break;
        }
        capturing = true;
        cudaEventRecord(ev[n_streams], cap);
        for (int i = 0; i < n_streams; ++i) cudaStreamWaitEvent(ss[i], ev[n_streams], 0);
        // roots go round-robin over the streams; a chained job runs on its parent's stream, after it
        std::vector<int> stream_of(b->jobs.size(), 0);
        int next_root = 0;
        for (size_t k = 0; k < b->jobs.size(); ++k)
            stream_of[k] = b->jobs[k].parent >= 0 ? stream_of[b->jobs[k].parent] : (next_root++ % n_streams);
        for (size_t k = 0; k < b->jobs.size() && s == PTS_OK; ++k) {
            const pts_job &j = b->jobs[k];
            pts_index idx = j.index;
            Workspace &ws = idx->ws;
            cudaStream_t js = ss[stream_of[k]];
            const int Q = job_queries(j);
            if (j.parent >= 0) {
                const pts_job &pj = b->jobs[j.parent];
                launch_upsample2(pj.output, pj.Ho, pj.Wo, j.output, js);
            }
            for (int t = 0; t <= iters && s == PTS_OK; ++t) {
                s = nn_search_impl(idx, j.output, j.Ho, j.Wo, j.stride, j.mode, ws.nn.ptr, ws.d2.ptr, js);
                if (s != PTS_OK) break;
                launch_irls(ws.d2.ptr, Q, r, delta, ws.wts.ptr, j.energy + t, ws.partial.ptr, ws.ticket.ptr, js);
                if (t < iters)
                    launch_m_step(ws.nn.ptr, ws.wts.ptr, idx->exemplar4.ptr, idx->We, idx->nx, idx->N, idx->C, idx->w, j.Ho,
                                  j.Wo, j.stride, j.output, idx->status.ptr, js);
            }
        }
        for (int i = 0; i < n_streams; ++i) {
            cudaEventRecord(ev[i], ss[i]);
            cudaStreamWaitEvent(cap, ev[i], 0);
        }
        const cudaError_t ec = cudaStreamEndCapture(cap, &b->graph);
        capturing = false;
        prof_suspend(true);
        b->launches = pts_launch_count() - l0;
        if (s != PTS_OK) break;
        if (ec != cudaSuccess) {
            s = set_error(PTS_ERR_CUDA, std::string("pts_batch_create: capture: ") + cudaGetErrorString(ec));
            break;
        }
        if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
            s = set_error(PTS_ERR_CUDA, "pts_batch_create: graph instantiation");
    } while (false);
    if (capturing) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(cap, &g);
        if (g) cudaGraphDestroy(g);
        prof_suspend(true);
    }
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t x : ss)
        if (x) cudaStreamDestroy(x);
    if (cap) cudaStreamDestroy(cap);
    if (s != PTS_OK) return fail(s);
    restore_parts();
    b->gens.resize(b->jobs.size());
    for (size_t k = 0; k < b->jobs.size(); ++k)
        if (!index_generation(b->jobs[k].index, &b->gens[k]))
            return fail(set_error(PTS_ERR_INVALID_ARG, "pts_batch_create: a job's index is not a live index"));
    *out = b;
    return PTS_OK;
}

pts_status pts_batch_run(pts_batch b, void *stream) {
    if (!b || !b->exec) return set_error(PTS_ERR_INVALID_ARG, "pts_batch_run: no batch");
    for (size_t k = 0; k < b->jobs.size(); ++k) {
        unsigned long long g = 0;
        if (!index_generation(b->jobs[k].index, &g) || g != b->gens[k])
            return set_error(PTS_ERR_INVALID_ARG,
                             "pts_batch_run: job " + std::to_string(k) +
                                 "'s index was destroyed or its buffers moved since pts_batch_create; create the "
                                 "batch again");
    }
    count_launches((int)b->launches);
    PTS_CUDA_TRY(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)));
    return PTS_OK;
}

pts_status pts_batch_info(pts_batch b, long long *launches_per_run, int *parts_out) {
    if (!b) return set_error(PTS_ERR_INVALID_ARG, "pts_batch_info: no batch");
    if (launches_per_run) *launches_per_run = b->launches;
    if (parts_out)
        for (size_t k = 0; k < b->parts.size(); ++k) parts_out[k] = b->parts[k];
    return PTS_OK;
}

void pts_batch_destroy(pts_batch b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}

pts_status synthesize_batched(const pts_job *jobs, int n_jobs, int iters, float r, float delta, void *stream) {
    pts_batch b = nullptr;
    PTS_TRY(pts_batch_create(jobs, n_jobs, iters, r, delta, std::min(n_jobs, 8), 1, stream, &b));
    pts_status s = pts_batch_run(b, stream);
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    pts_batch_destroy(b);
    if (s != PTS_OK) return s;
    if (e != cudaSuccess) return cuda_error(e, "synthesize_batched");
    for (int k = 0; k < n_jobs; ++k) PTS_TRY(pts_index_device_status(jobs[k].index, stream));
    return PTS_OK;
}

}  // extern "C"
