// capi.cu -- the C ABI (include/pts.h): argument checks, the index object,
// workspace management and the E-step / EM drivers that sequence the kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "pts_internal.cuh"

namespace pts {

namespace {
thread_local std::string g_last_error;

// Rounding slack of the PCA lower bound: tau_q = c sqrt(D) 2^-24 (||u_q||^2 +
// max_n ||u_n||^2).  FP32 dot products of length D carry errors that grow like
// sqrt(D) units in the last place in practice (Higham, "Accuracy and
// Stability of Numerical Algorithms", section 3.1), relative to the operand
// norms; c = 8 leaves a wide margin.
constexpr float kTauC = 8.0f;
constexpr int kWarmMinTiles = 100;  // exemplar tiles below which the FP16 search starts cold

// Margin added to a warm-start bound for the FP16 tensor-core search.  The
// bound is computed from the very FP16 operands the tensor cores multiply
// (their products are exact in FP32), so it only differs from the search's
// values by the FP32 summation order: at most 2 K 2^-24 sum|terms| with
// K <= 128 and sum|terms| <= ||u_q||^2 + 2 max_n ||u_n||^2.  2^-13 doubles that.
constexpr float kWarmEps = 1.0f / 8192.0f;

// The exact search runs its PCA-space pass only when the d components keep at least this
// fraction of the exemplar's variance; below it most queries fail the certificate and the pass
// is wasted, so every query goes straight to the full-dimension pass.
constexpr double kPcaPassMinVar = 0.85;

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// tau_q / (||u_q||^2 + max_n ||u_n||^2) for a bound from the FP16 tensor-core search: operand
// rounding (1 + 2^-11)^2 - 1 < 2^-10 per product of sum |products| <= ||u_q||^2 + max ||u_n||^2,
// the FP32 sum of K <= 128 terms, the FP16 storage of a kept score as an offset from its group
// minimum (2^-11 of an offset no larger than the score range), and the FP32 slack of the
// full-dimension distance; 2^-8 covers the first three.
float f16_slack(pts_index idx) { return 1.0f / 256.0f + kTauC * sqrtf((float)idx->D) * 5.9604645e-8f; }

pts_status check_grid(int H, int W, int w, int stride, const char *what) {
    if (stride != 1 && stride != 2 && stride != 4)
        return set_error(PTS_ERR_INVALID_ARG, std::string(what) + ": stride must be 1, 2 or 4");
    if (w < 1 || w > H || w > W)
        return set_error(PTS_ERR_INVALID_ARG, std::string(what) + ": window larger than the image");
    if ((H - w) % stride || (W - w) % stride || w % stride)
        return set_error(PTS_ERR_INVALID_ARG,
                         std::string(what) + ": (H-w), (W-w) and w must be multiples of the stride");
    return PTS_OK;
}

}  // namespace

pts_status check_grid_public(int H, int W, int w, int stride, const char *what) {
    return check_grid(H, W, w, stride, what);
}

pts_status ensure_workspace(pts_index idx, int Q) {
    Workspace &ws = idx->ws;
    if (Q <= ws.q_cap && ws.counters.ptr) return PTS_OK;
    const int cap = std::max(Q, 1024);
    const size_t qpad = (size_t)ceil_div(cap, kBQ) * kBQ;
    PTS_TRY(ws.qcoord.ensure(qpad * std::max(idx->da, idx->da_fast), "query vectors"));
    PTS_TRY(ws.qnorm.ensure(qpad, "query norms"));
    PTS_TRY(ws.tau.ensure(qpad, "query slack"));
    PTS_TRY(ws.cand_idx.ensure((size_t)cap * kTopK, "candidate indices"));
    PTS_TRY(ws.cand_lb.ensure((size_t)cap * kTopK, "candidate bounds"));
    PTS_TRY(ws.fail_list.ensure(cap, "fail list"));
    PTS_TRY(ws.fail2_list.ensure(cap, "second fail list"));
    PTS_TRY(ws.qfull.ensure(qpad * std::max(padded_dim(idx->D), padded_dim(idx->da_fast)), "full query vectors"));
    PTS_TRY(ws.best64.ensure(cap, "packed minima"));
    PTS_TRY(ws.thr0.ensure(2 * (size_t)cap, "warm-start bounds"));
    PTS_TRY(ws.pca_thr.ensure((size_t)cap, "PCA-pass bounds"));
    PTS_TRY(ws.counters.ensure(4, "counters"));
    PTS_TRY(ws.nn.ensure(cap, "nn"));
    PTS_TRY(ws.d2.ensure(cap, "d2"));
    PTS_TRY(ws.wts.ensure(cap, "weights"));
    PTS_TRY(ws.partial.ensure(kIrlsGrid, "reduction partials"));
    if (!ws.ticket.ptr) {
        PTS_TRY(ws.ticket.ensure(1, "reduction ticket"));
        PTS_CUDA_TRY(cudaMemset(ws.ticket.ptr, 0, sizeof(unsigned int)));
    }
    ws.q_cap = cap;
    return PTS_OK;
}

pts_status read_status(pts_index idx, cudaStream_t st) {
    int h = 0;
    PTS_CUDA_TRY(cudaMemcpyAsync(&h, idx->status.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h & (kDevErrBounds | kDevErrTimeout | kDevErrNumeric)) {
        PTS_CUDA_TRY(cudaMemsetAsync(idx->status.ptr, 0, sizeof(int), st));
        PTS_CUDA_TRY(cudaStreamSynchronize(st));
        if (h & kDevErrTimeout) return set_error(PTS_ERR_TIMEOUT, "a bounded device wait gave up");
        if (h & kDevErrBounds) return set_error(PTS_ERR_DEVICE, "an index input was out of range");
        return set_error(PTS_ERR_DEVICE, "a factorisation met a non-positive pivot");
    }
    return PTS_OK;
}

// Exact search for the queries listed in in_list (count on the device): full-dimension GEMM
// top-32, certified re-rank (what stays uncertified goes to out_list), direct scan of those.
pts_status exact_on_list(pts_index idx, const RerankArgs &ra, int *in_list, unsigned int *in_count, int *out_list,
                         unsigned int *out_count, unsigned int *brute_count, int32_t *nn_out, float *d2_out,
                         cudaStream_t st) {
    Workspace &ws = idx->ws;
    PTS_TRY(ws.part_v.ensure(full_part_capacity(ra.Q), "part lists"));
    PTS_TRY(ws.part_i.ensure(full_part_capacity(ra.Q), "part lists"));
    idx->last.full_splits = launch_search_full(ra.X, ra.Wo, idx->C, idx->w, ra.stride, ra.qx, idx->mu.ptr, in_list,
                                               in_count, ra.Q, ws.qfull.ptr, idx->efull.ptr, idx->enorm.ptr,
                                               idx->ntiles, ws.qnorm.ptr, ws.cand_idx.ptr, ws.cand_lb.ptr,
                                               ws.part_v.ptr, ws.part_i.ptr, idx->status.ptr, st, idx->N,
                                               &ws.full_pdist);
    launch_rerank(ra, in_list, in_count, ws.cand_idx.ptr, ws.cand_lb.ptr, ws.tau.ptr, 1, nn_out, d2_out, out_list,
                  out_count, ws.best64.ptr, idx->status.ptr, st);
    launch_brute_fallback(ra, out_list, out_count, brute_count, ws.best64.ptr, idx->status.ptr, st);
    launch_resolve(out_list, out_count, ws.best64.ptr, ra.Q, nn_out, d2_out, st);
    return PTS_OK;
}

// the learned proposal: network -> 4 clusters -> probe -> re-rank -> exact fallback
pts_status search_proposal(pts_index idx, const float *X, int Ho, int Wo, int stride, int Q, int32_t *nn_out,
                           float *d2_out, cudaStream_t st) {
    Workspace &ws = idx->ws;
    ProposalState &pr = idx->prop;
    if (!pr.ready) return set_error(PTS_ERR_INVALID_ARG, "nn_search: no proposal trained on this index");
    launch_project(X, Ho, Wo, idx->C, idx->w, stride, idx->mu.ptr, idx->basisT.ptr, idx->d_fast, idx->da_fast, 0,
                   ws.qcoord.ptr, ws.qnorm.ptr, ws.tau.ptr, f16_slack(idx), idx->umax.ptr, st, &ws.proj_part);
    PTS_TRY(pr.top.ensure((size_t)std::max(Q, 1) * 4, "probed clusters"));
    launch_mlp_top4(pr.infer, ws.qcoord.ptr, Q, std::min(idx->d, 64), idx->da_fast, pr.top.ptr, idx->status.ptr, st);
    // probe: the tensor-core search restricted, per (query, cluster) pair, to the cluster's tiles
    const int maxb = ivf_max_blocks(Q, pr.C);
    PTS_TRY(pr.ivf_cnt.ensure(pr.C, "probe counts"));
    PTS_TRY(pr.ivf_poff.ensure(pr.C, "probe offsets"));
    PTS_TRY(pr.ivf_cursor.ensure(pr.C, "probe cursors"));
    PTS_TRY(pr.ivf_nblk.ensure(1, "probe blocks"));
    PTS_TRY(pr.pair_q.ensure((size_t)4 * std::max(Q, 1), "probe pairs"));
    PTS_TRY(pr.pair_r.ensure((size_t)4 * std::max(Q, 1), "probe pairs"));
    PTS_TRY(pr.ivf_blk.ensure((size_t)maxb, "probe block table"));
    PTS_TRY(pr.ivf_qtile.ensure((size_t)maxb * 128 * idx->ktc, "probe query tiles"));
    PTS_TRY(pr.ivf_part_v.ensure((size_t)std::max(Q, 1) * 4 * kTopK, "probe lists"));
    PTS_TRY(pr.ivf_part_i.ensure((size_t)std::max(Q, 1) * 4 * kTopK, "probe lists"));
    PTS_TRY(pr.ivf_kept.ensure(tc_kept_bytes(Q, 4), "probe kept groups"));
    IvfBuffers ib{pr.ivf_cnt.ptr, pr.ivf_poff.ptr, pr.ivf_cursor.ptr, pr.ivf_nblk.ptr, pr.pair_q.ptr,
                  pr.pair_r.ptr, pr.ivf_blk.ptr, pr.ivf_qtile.ptr, pr.ivf_part_v.ptr, pr.ivf_part_i.ptr,
                  pr.ivf_kept.ptr};
    launch_ivf_probe(pr.top.ptr, Q, pr.C, pr.off.ptr, ws.qcoord.ptr, ws.qnorm.ptr, idx->d_fast, idx->da_fast, idx->ktc,
                     pr.etc_ivf.ptr, tc_tiles(idx->N), idx->N, pr.members.ptr, ib, ws.cand_idx.ptr, ws.cand_lb.ptr,
                     idx->status.ptr, st);
    const int qx = (Wo - idx->w) / stride + 1;
    RerankArgs ra{X, Ho, Wo, stride, qx, idx->exemplar.ptr, idx->We, idx->w, idx->nx, idx->N, Q, idx->C,
                  idx->exemplar4.ptr};
    PTS_CUDA_TRY(cudaMemsetAsync(ws.counters.ptr, 0, 4 * sizeof(unsigned int), st));
    launch_rerank(ra, nullptr, nullptr, ws.cand_idx.ptr, ws.cand_lb.ptr, ws.tau.ptr, 2, nn_out, d2_out,
                  ws.fail_list.ptr, ws.counters.ptr + 3, ws.best64.ptr, idx->status.ptr, st);
    launch_fallback(nn_out, d2_out, Q, pr.assign.ptr, pr.median.ptr, pr.factor, idx->N, ws.fail_list.ptr,
                    ws.counters.ptr + 0, st);
    // the fallback: the FP16 tensor-core search over every window for the listed queries
    PTS_TRY(ws.qtile.ensure((size_t)tc_query_blocks(Q) * 128 * idx->ktc, "query operand tiles"));
    launch_pack_queries(ws.qcoord.ptr, Q, idx->d_fast, idx->da_fast, idx->ktc, ws.qtile.ptr, st, ws.fail_list.ptr,
                        ws.counters.ptr + 0);
    PTS_TRY(ws.kept.ensure(tc_kept_bytes(Q, 1), "kept groups"));
    launch_search_tc(ws.qtile.ptr, ws.qnorm.ptr, Q, idx->ktc, idx->etc.ptr, tc_tiles(idx->N), 1, nullptr,
                     ws.cand_idx.ptr, ws.cand_lb.ptr, nullptr, nullptr, idx->status.ptr, st, ws.fail_list.ptr,
                     ws.counters.ptr + 0, 0, nullptr, nullptr, idx->N, ws.kept.ptr);
    launch_rerank(ra, ws.fail_list.ptr, ws.counters.ptr + 0, ws.cand_idx.ptr, ws.cand_lb.ptr, ws.tau.ptr, 2, nn_out,
                  d2_out, ws.fail2_list.ptr, ws.counters.ptr + 1, ws.best64.ptr, idx->status.ptr, st);
    return PTS_OK;
}

// the paper's k-means tree: descent to a leaf, exact re-rank of its windows
pts_status search_kmtree(pts_index idx, const float *X, int Ho, int Wo, int stride, int Q, int32_t *nn_out,
                         float *d2_out, cudaStream_t st) {
    KmTree &tr = idx->tree;
    if (!tr.ready) return set_error(PTS_ERR_INVALID_ARG, "nn_search: no k-means tree built on this index");
    Workspace &ws = idx->ws;
    launch_project(X, Ho, Wo, idx->C, idx->w, stride, idx->mu.ptr, idx->basisT.ptr, idx->d, idx->da, 0, ws.qcoord.ptr,
                   ws.qnorm.ptr, ws.tau.ptr, 0.0f, idx->umax.ptr, st, &ws.proj_part);
    PTS_TRY(tr.leaf_of_query.ensure((size_t)std::max(Q, 1), "tree leaves of the queries"));
    launch_tree_search(tr, ws.qcoord.ptr, idx->da, Q, ws.cand_idx.ptr, ws.cand_lb.ptr, tr.leaf_of_query.ptr, st);
    const int qx = (Wo - idx->w) / stride + 1;
    RerankArgs ra{X, Ho, Wo, stride, qx, idx->exemplar.ptr, idx->We, idx->w, idx->nx, idx->N, Q, idx->C,
                  idx->exemplar4.ptr};
    launch_rerank(ra, nullptr, nullptr, ws.cand_idx.ptr, ws.cand_lb.ptr, ws.tau.ptr, 0, nn_out, d2_out,
                  ws.fail_list.ptr, ws.counters.ptr, ws.best64.ptr, idx->status.ptr, st);
    return PTS_OK;
}

// the E-step in exact mode (see include/pts.h)
pts_status search_exact(pts_index idx, const float *X, int Ho, int Wo, int stride, int Q,
                        int32_t *nn_out, float *d2_out, cudaStream_t st) {
    Workspace &ws = idx->ws;
    // the bound's components: the index's d_fast (the larger PCA) or its first d
    const bool fast = idx->exact_fast == 1 && idx->d_fast > idx->d && idx->et_fast_rows.ptr;
    const int bd = fast ? idx->d_fast : idx->d, bda = fast ? idx->da_fast : idx->da;
    const float *bet = fast ? idx->et_fast.ptr : idx->et.ptr;
    const float *brows = fast ? idx->et_fast_rows.ptr : idx->et_rows.ptr;
    const double bvar = fast ? idx->var_fast : idx->var_retained;
    const float tau_scale = kTauC * sqrtf((float)idx->D) * 5.9604645e-8f;
    const int qx = (Wo - idx->w) / stride + 1;
    RerankArgs ra{X, Ho, Wo, stride, qx, idx->exemplar.ptr, idx->We, idx->w, idx->nx, idx->N, Q, idx->C,
                  idx->exemplar4.ptr};
    unsigned int *fail_count = ws.counters.ptr + 0;
    unsigned int *fail2_count = ws.counters.ptr + 1;
    unsigned int *brute_count = ws.counters.ptr + 2;
    unsigned int *fail3_count = ws.counters.ptr + 3;
    idx->last_cascade = 0;
    PTS_CUDA_TRY(cudaMemsetAsync(ws.counters.ptr, 0, 4 * sizeof(unsigned int), st));
    if (bvar < kPcaPassMinVar) {
        // the bound would certify few queries: every query goes to the full-dimension pass (its
        // bound needs only ||u_q||^2 and the slack)
        launch_project(X, Ho, Wo, idx->C, idx->w, stride, idx->mu.ptr, idx->basisT.ptr, 0, idx->da, 0, nullptr,
                       ws.qnorm.ptr, ws.tau.ptr, tau_scale, idx->umax.ptr, st);
        launch_list_all(ws.fail_list.ptr, fail_count, Q, st);
    } else {
        launch_project(X, Ho, Wo, idx->C, idx->w, stride, idx->mu.ptr, idx->basisT.ptr, bd, bda, 0,
                       ws.qcoord.ptr, ws.qnorm.ptr, ws.tau.ptr, tau_scale, idx->umax.ptr, st, &ws.proj_part);
        const int pp = pca_parts(Q, idx->ntiles);
        if (pp > 1) {
            PTS_TRY(ws.part_v.ensure((size_t)Q * pp * kTopK, "part lists"));
            PTS_TRY(ws.part_i.ensure((size_t)Q * pp * kTopK, "part lists"));
        }
        // the candidates of the previous search on this grid (any mode) bound the 32nd best
        const bool warm = ws.warm_q == Q && ws.warm_ho == Ho && ws.warm_wo == Wo && ws.warm_stride == stride;
        if (warm) {
            launch_warm_pca(ws.cand_idx.ptr, ws.qcoord.ptr, bda, brows, idx->enorm.ptr, Q, idx->N,
                            ws.pca_thr.ptr, st);
        }
        launch_search_topk(ws.qcoord.ptr, ws.qnorm.ptr, Q, bda, bd + 1, bet, idx->enorm.ptr,
                           idx->ntiles, ws.cand_idx.ptr, ws.cand_lb.ptr, idx->status.ptr, st, pp, ws.part_v.ptr,
                           ws.part_i.ptr, warm ? ws.pca_thr.ptr : nullptr);
        // pass 1: PCA bounds -> top-32 -> exact re-rank, certified or listed
        launch_rerank(ra, nullptr, nullptr, ws.cand_idx.ptr, ws.cand_lb.ptr, ws.tau.ptr, 1, nn_out,
                      d2_out, ws.fail_list.ptr, fail_count, ws.best64.ptr, idx->status.ptr, st);
        // pass 1b, for the listed queries only: the same bound with the index's d_fast components
        // (the larger PCA the tensor-core searches use), certified the same way
        if (!fast && idx->exact_fast == 0 && idx->d_fast > idx->d && idx->var_fast >= kPcaPassMinVar &&
            idx->da_fast % 32 == 0) {
            idx->last_cascade = 1;
            launch_project(X, Ho, Wo, idx->C, idx->w, stride, idx->mu.ptr, idx->basisT.ptr, idx->d_fast,
                           idx->da_fast, 0, ws.qcoord.ptr, ws.qnorm.ptr, ws.tau.ptr, tau_scale, idx->umax.ptr, st,
                           &ws.proj_part);
            PTS_TRY(ws.part_v.ensure(full_part_capacity(Q), "part lists"));
            PTS_TRY(ws.part_i.ensure(full_part_capacity(Q), "part lists"));
            launch_search_rows(ws.qcoord.ptr, idx->da_fast, idx->d_fast + 1, ws.fail_list.ptr, fail_count, Q,
                               idx->da_fast,
                               ws.qfull.ptr, idx->et_fast.ptr, idx->enorm.ptr, idx->ntiles, ws.qnorm.ptr,
                               ws.cand_idx.ptr, ws.cand_lb.ptr, ws.part_v.ptr, ws.part_i.ptr, idx->status.ptr, st);
            launch_rerank(ra, ws.fail_list.ptr, fail_count, ws.cand_idx.ptr, ws.cand_lb.ptr, ws.tau.ptr, 1, nn_out,
                          d2_out, ws.fail2_list.ptr, fail2_count, ws.best64.ptr, idx->status.ptr, st);
            PTS_TRY(exact_on_list(idx, ra, ws.fail2_list.ptr, fail2_count, ws.fail_list.ptr, fail3_count, brute_count,
                                  nn_out, d2_out, st));
            return PTS_OK;
        }
    }
    PTS_TRY(exact_on_list(idx, ra, ws.fail_list.ptr, fail_count, ws.fail2_list.ptr, fail2_count, brute_count, nn_out,
                          d2_out, st));
    return PTS_OK;
}

// The nearest windows of Eq. 4 through the full-dimension FP16 GEMM (search_tcf.cu): scores of
// every pair, the 32 best per query re-ranked in FP32 and certified with the GEMM's rounding
// slack; the rest takes the FP32 full pass of exact mode.  Slack per unit of ||u_q||^2 + max_n
// ||u_n||^2 (scores -2 (2^-12 a_hat . 2^-12 b_hat) + ||u_n||^2 with a_hat = fl16(2^12 u_q)):
//   FP16 operands: |a_hat b_hat - a b| <= (2^-10 + 2^-22) |a b| for normal values, and the terms
//     of values below the FP16 normal range add at most D 2^-31 in all, which is below
//     2^-10 max_n ||u_n||^2 when that is >= D 2^-21 (checked): 2^-9 + 2^-22 in all, after
//     sum |a_i b_i| <= (||u_q||^2 + ||u_n||^2) / 2 and the factor 2 of the score;
//   FP32 accumulation of D products, each addition within 2^-22 of its partial sum (a
//     truncating accumulator included): D 2^-22 (1 + 2^-10);
//   the epilogue's FMA and the bound's addition of ||u_q||^2: 2^-21;
//   the FP32 norms and the FP32 re-rank: exact mode's model, kTauC sqrt(D) 2^-24.
float tcf_slack(int D) {
    return (float)((std::ldexp(1.0, -9) + (D + 2) * std::ldexp(1.0, -22)) * (1.0 + std::ldexp(1.0, -10)) +
                   kTauC * std::sqrt((double)D) * std::ldexp(1.0, -24));
}

// FP16 full-dimension tiles of the exemplar, built on the first PTS_EXACT_TC search (one
// synchronisation); tcf_state -1 when they cannot be used
// The FP16 search's query rows into ws.qtile, with ||u||^2 (norm) and tau: on the tensor cores
// (their FP16 hi/lo basis tiles built on first use) unless asked otherwise or the image is past
// the kernel's 32-bit offsets, else by the FP32 SIMT projection.
pts_status project_f16_rows(pts_index idx, const float *X, int Ho, int Wo, int stride, int tensor_cores, float *norm,
                            cudaStream_t st) {
    Workspace &ws = idx->ws;
    if (tensor_cores && project_tc16_fits(Ho, Wo, idx->C)) {
        if (!idx->basis16_ready) {
            PTS_TRY(idx->basis16.ensure(basis16_bytes(idx->D), "FP16 basis tiles"));
            launch_pack_basis16(idx->basisT.ptr, idx->D, idx->d_fast, idx->basis16.ptr, st);
            idx->basis16_ready = true;
        }
        launch_project_tc16(X, Ho, Wo, idx->C, idx->w, stride, idx->mu.ptr, idx->basis16.ptr, idx->d_fast, idx->ktc,
                            ws.qtile.ptr, norm, ws.tau.ptr, f16_slack(idx), idx->umax.ptr, idx->status.ptr, st,
                            &ws.proj_part);
    } else {
        launch_project_tile16(X, Ho, Wo, idx->C, idx->w, stride, idx->mu.ptr, idx->basisT.ptr, idx->d_fast, idx->ktc,
                              ws.qtile.ptr, norm, ws.tau.ptr, f16_slack(idx), idx->umax.ptr, st, &ws.proj_part);
    }
    return PTS_OK;
}

pts_status ensure_tcf_tiles(pts_index idx, cudaStream_t st) {
    if (idx->tcf_state != 0) return PTS_OK;
    if (!((double)idx->unorm2_max >= idx->D * std::ldexp(1.0, -21))) {
        idx->tcf_state = -1;
        return PTS_OK;
    }
    const size_t n = (size_t)tcf_tiles(idx->N) * 256 * tcf_k(idx->D);
    PTS_TRY(idx->efull16.ensure(n, "FP16 full-dimension tiles"));
    DevBuf<int> over;
    PTS_TRY(over.ensure(1, "range flag"));
    PTS_CUDA_TRY(cudaMemsetAsync(over.ptr, 0, sizeof(int), st));
    launch_pack_exemplar_full16(idx->exemplar.ptr, idx->We, idx->C, idx->w, idx->nx, idx->N, idx->mu.ptr,
                                idx->efull16.ptr, over.ptr, st);
    int h = 0;
    PTS_CUDA_TRY(cudaMemcpyAsync(&h, over.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    idx->tcf_state = h ? -1 : 1;
    if (h) idx->efull16.release();
    return PTS_OK;
}

// PTS_EXACT_TC runs the FP32 route when its scores (Q x 256-window tiles x 4 bytes) would pass
// this size: their write and read then cost more than the FP32 route's bounds save.
constexpr size_t kTcfScoreBytes = 256u << 20;

pts_status search_exact_tc(pts_index idx, const float *X, int Ho, int Wo, int stride, int Q, int32_t *nn_out,
                           float *d2_out, cudaStream_t st) {
    const int npad = tcf_tiles(idx->N) * 256;
    if ((size_t)Q * npad * sizeof(float) > kTcfScoreBytes)
        return search_exact(idx, X, Ho, Wo, stride, Q, nn_out, d2_out, st);
    PTS_TRY(ensure_tcf_tiles(idx, st));
    if (idx->tcf_state != 1) return search_exact(idx, X, Ho, Wo, stride, Q, nn_out, d2_out, st);
    Workspace &ws = idx->ws;
    const float tau_scale = kTauC * sqrtf((float)idx->D) * 5.9604645e-8f;
    const int qx = (Wo - idx->w) / stride + 1;
    RerankArgs ra{X, Ho, Wo, stride, qx, idx->exemplar.ptr, idx->We, idx->w, idx->nx, idx->N, Q, idx->C,
                  idx->exemplar4.ptr};
    unsigned int *fail_count = ws.counters.ptr + 0;
    unsigned int *fail2_count = ws.counters.ptr + 1;
    unsigned int *brute_count = ws.counters.ptr + 2;
    idx->last_cascade = 0;
    PTS_TRY(ws.qtile16.ensure((size_t)tcf_query_blocks(Q) * 128 * tcf_k(idx->D), "FP16 query tiles"));
    PTS_TRY(ws.tau_tc.ensure((size_t)std::max(Q, 1), "FP16 slack"));
    PTS_TRY(ws.full_pdist.ensure((size_t)std::max(Q, 1) * npad, "full-dimension scores"));
    PTS_CUDA_TRY(cudaMemsetAsync(ws.counters.ptr, 0, 4 * sizeof(unsigned int), st));
    // the FP16 query tiles, ||u_q||^2, exact mode's slack (the FP32 pass uses it) and the GEMM's
    // slack in one pass over the windows, then the GEMM and the 32 best scores of every query
    launch_pack_queries_full16(X, Wo, idx->C, idx->w, stride, qx, Q, idx->mu.ptr, ws.qtile16.ptr, ws.qnorm.ptr,
                               ws.tau.ptr, tau_scale, ws.tau_tc.ptr, tcf_slack(idx->D), idx->umax.ptr, st);
    launch_gemm_tcf(ws.qtile16.ptr, Q, idx->C, idx->w, idx->efull16.ptr, idx->N, idx->enorm.ptr, ws.qnorm.ptr,
                    ws.full_pdist.ptr, ws.cand_idx.ptr, ws.cand_lb.ptr, idx->status.ptr, st);
    launch_rerank(ra, nullptr, nullptr, ws.cand_idx.ptr, ws.cand_lb.ptr, ws.tau_tc.ptr, 1, nn_out, d2_out,
                  ws.fail_list.ptr, fail_count, ws.best64.ptr, idx->status.ptr, st);
    PTS_TRY(exact_on_list(idx, ra, ws.fail_list.ptr, fail_count, ws.fail2_list.ptr, fail2_count, brute_count, nn_out,
                          d2_out, st));
    return PTS_OK;
}

pts_status nn_search_impl(pts_index idx, const float *X, int Ho, int Wo, int stride, int mode,
                          int32_t *nn_out, float *d2_out, cudaStream_t st) {
    PTS_TRY(check_grid(Ho, Wo, idx->w, stride, "nn_search"));
    if (!X || !nn_out || !d2_out) return set_error(PTS_ERR_INVALID_ARG, "nn_search: null pointer");
    const long Ql = (long)((Ho - idx->w) / stride + 1) * ((Wo - idx->w) / stride + 1);
    if (Ql > (1L << 30)) return set_error(PTS_ERR_INVALID_ARG, "nn_search: too many queries");
    const int Q = (int)Ql;
    PTS_TRY(ensure_workspace(idx, Q));
    idx->last_mode = mode;
    idx->last.queries = Q;
    idx->last.full_splits = 0;
    switch (mode) {
        case PTS_EXACT_F32:
            PTS_TRY(search_exact(idx, X, Ho, Wo, stride, Q, nn_out, d2_out, st));
            break;
        case PTS_F16_RERANK: {
            Workspace &ws = idx->ws;
            // the projection writes the FP16 query tiles itself (no FP32 coordinates in between)
            PTS_TRY(ws.qtile.ensure((size_t)tc_query_blocks(Q) * kTcQueryRows * idx->ktc, "query operand tiles"));
            PTS_TRY(project_f16_rows(idx, X, Ho, Wo, stride, 1, ws.qnorm.ptr, st));
            const int ntc = tc_tiles(idx->N);
            // 0: automatic -- the default split rule, one part plus the tail split of launch_search_tc
            const int auto_parts = tc_parts(Q, ntc);
            const int nparts = idx->tc_parts_override > 0 ? std::min(idx->tc_parts_override, ntc)
                                                          : (auto_parts > 1 ? auto_parts : 0);
            // the candidate lists of the previous search on this grid seed the bound, where the search
            // is long enough for the bound to save more than it costs (measured: at 243 tiles it saves
            // 0.12 ms of a fine-level search for about 0.05; at 50 tiles 2 us for about 10)
            const bool warm = ntc >= kWarmMinTiles && ws.warm_q == Q && ws.warm_ho == Ho && ws.warm_wo == Wo &&
                              ws.warm_stride == stride;
            if (warm)
                launch_warm_threshold(ws.cand_idx.ptr, ws.qtile.ptr, ws.qnorm.ptr, idx->etc.ptr, idx->umax.ptr, Q, idx->ktc,
                                      idx->N, kWarmEps, ws.thr0.ptr, st);
            PTS_TRY(ws.kept.ensure(tc_kept_bytes_search(Q, ntc, nparts), "kept groups"));
            launch_search_tc(ws.qtile.ptr, ws.qnorm.ptr, Q, idx->ktc, idx->etc.ptr, ntc, nparts,
                             warm ? ws.thr0.ptr : nullptr, ws.cand_idx.ptr, ws.cand_lb.ptr, ws.part_v.ptr,
                             ws.part_i.ptr, idx->status.ptr, st, nullptr, nullptr, 0, nullptr, nullptr, idx->N,
                             ws.kept.ptr);
            RerankArgs ra{X, Ho, Wo, stride, (Wo - idx->w) / stride + 1, idx->exemplar.ptr, idx->We, idx->w,
                          idx->nx, idx->N, Q, idx->C, idx->exemplar4.ptr};
            // candidates in ascending bound order; stop where bound - slack exceeds the best
            launch_rerank(ra, nullptr, nullptr, ws.cand_idx.ptr, ws.cand_lb.ptr, ws.tau.ptr, 2, nn_out, d2_out,
                          ws.fail_list.ptr, ws.counters.ptr, ws.best64.ptr, idx->status.ptr, st);
            break;
        }
        case PTS_PROPOSAL:
            PTS_TRY(search_proposal(idx, X, Ho, Wo, stride, Q, nn_out, d2_out, st));
            break;
        case PTS_EXACT_TC:
            PTS_TRY(search_exact_tc(idx, X, Ho, Wo, stride, Q, nn_out, d2_out, st));
            break;
        case PTS_KMTREE:
            PTS_TRY(search_kmtree(idx, X, Ho, Wo, stride, Q, nn_out, d2_out, st));
            break;
        case PTS_FP8_RERANK: {
            // FP8 E4M3 operands with per-dimension scales (the epilogue adds the FP32 norms); the
            // bound's rounding error is too large for a useful early exit, so every candidate is
            // re-ranked
            Workspace &ws = idx->ws;
            launch_project(X, Ho, Wo, idx->C, idx->w, stride, idx->mu.ptr, idx->basisT.ptr, idx->d_fast, idx->da_fast, 0,
                           ws.qcoord.ptr, ws.qnorm.ptr, ws.tau.ptr, 0.0f, idx->umax.ptr, st, &ws.proj_part);
            const int ntc = tc_tiles(idx->N);
            // 0: automatic -- the default split rule, one part plus the tail split of launch_search_tc
            const int auto_parts = tc_parts(Q, ntc);
            const int nparts = idx->tc_parts_override > 0 ? std::min(idx->tc_parts_override, ntc)
                                                          : (auto_parts > 1 ? auto_parts : 0);
            PTS_TRY(ws.qtile8.ensure((size_t)tc_query_blocks(Q) * 128 * idx->kf8, "fp8 query tiles"));
            PTS_TRY(ws.qscale.ensure((size_t)std::max(Q, 1), "fp8 query scales"));
            launch_pack_queries_f8(ws.qcoord.ptr, Q, idx->d_fast, idx->da_fast, idx->kf8, idx->f8scale.ptr,
                                   ws.qtile8.ptr, ws.qscale.ptr, st);
            PTS_TRY(ws.kept.ensure(tc_kept_bytes_search(Q, ntc, nparts), "kept groups"));
            launch_search_tc(ws.qtile8.ptr, ws.qnorm.ptr, Q, idx->kf8, idx->etc8.ptr, ntc, nparts, nullptr,
                             ws.cand_idx.ptr, ws.cand_lb.ptr, ws.part_v.ptr, ws.part_i.ptr, idx->status.ptr, st,
                             nullptr, nullptr, 1, ws.qscale.ptr, idx->enorm.ptr, idx->N, ws.kept.ptr);
            RerankArgs ra{X, Ho, Wo, stride, (Wo - idx->w) / stride + 1, idx->exemplar.ptr, idx->We, idx->w,
                          idx->nx, idx->N, Q, idx->C, idx->exemplar4.ptr};
            launch_rerank(ra, nullptr, nullptr, ws.cand_idx.ptr, ws.cand_lb.ptr, ws.tau.ptr, 0, nn_out, d2_out,
                          ws.fail_list.ptr, ws.counters.ptr, ws.best64.ptr, idx->status.ptr, st);
            break;
        }
        default:
            return set_error(PTS_ERR_INVALID_ARG, "nn_search: unknown mode");
    }
    PTS_CUDA_TRY(cudaGetLastError());
    idx->ws.warm_q = Q;
    idx->ws.warm_ho = Ho;
    idx->ws.warm_wo = Wo;
    idx->ws.warm_stride = stride;
    return PTS_OK;
}


// ---------------------------------------------------------------------------
// registry of live indices and their buffer generations
// ---------------------------------------------------------------------------
namespace {
std::mutex g_registry_mu;
std::vector<pts_index> g_live_indices;
unsigned long long g_generation = 0;
}  // namespace

void register_index(pts_index idx) {
    std::lock_guard<std::mutex> lk(g_registry_mu);
    idx->generation = ++g_generation;
    g_live_indices.push_back(idx);
}

void unregister_index(pts_index idx) {
    std::lock_guard<std::mutex> lk(g_registry_mu);
    g_live_indices.erase(std::remove(g_live_indices.begin(), g_live_indices.end(), idx), g_live_indices.end());
}

bool index_generation(pts_index idx, unsigned long long *gen) {
    std::lock_guard<std::mutex> lk(g_registry_mu);
    for (pts_index p : g_live_indices)
        if (p == idx) {
            *gen = p->generation;
            return true;
        }
    return false;
}

void note_buffer_moved(const void *buf) {
    const char *b = static_cast<const char *>(buf);
    std::lock_guard<std::mutex> lk(g_registry_mu);
    for (pts_index p : g_live_indices) {
        const char *lo = reinterpret_cast<const char *>(p);
        if (b >= lo && b < lo + sizeof(pts_index_s)) {
            p->generation = ++g_generation;
            return;
        }
    }
}

pts_status set_error(pts_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

pts_status cuda_error(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return PTS_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// device memory: cudaMalloc / cudaFree, or the allocator registered by pts_set_allocator
// ---------------------------------------------------------------------------
namespace {
struct Allocator {
    pts_alloc_fn alloc = nullptr;
    pts_free_fn release = nullptr;
    void *user = nullptr;
};
std::mutex g_alloc_mu;
Allocator g_alloc;                 // empty: cudaMalloc / cudaFree
std::atomic<long long> g_live{0};  // library allocations not yet freed
}  // namespace

pts_status dev_alloc(void **p, size_t bytes, const char *what) {
    *p = nullptr;
    // the lock spans the allocation, so the allocator cannot be swapped while one is being made
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_alloc.alloc) {
        *p = g_alloc.alloc(bytes, nullptr, g_alloc.user);
        if (!*p) return set_error(PTS_ERR_OOM, std::string("registered allocator failed for ") + what);
    } else {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            *p = nullptr;
            cudaGetLastError();
            return set_error(PTS_ERR_OOM, std::string("cudaMalloc failed for ") + what);
        }
    }
    g_live.fetch_add(1);
    return PTS_OK;
}

void dev_free(void *p) {
    if (!p) return;
    Allocator a;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
    }
    // while this allocation is still counted live, pts_set_allocator cannot swap the allocator
    if (a.release) {
        cudaDeviceSynchronize();
        a.release(p, nullptr, a.user);
    } else {
        cudaFree(p);
    }
    g_live.fetch_sub(1);
}

}  // namespace pts

using namespace pts;

extern "C" {

const char *pts_last_error(void) { return g_last_error.c_str(); }

const char *pts_version(void) { return "pts-gb300 0.1 (sm_103a)"; }

pts_status pts_set_allocator(pts_alloc_fn alloc, pts_free_fn release, void *user) {
    if ((alloc == nullptr) != (release == nullptr))
        return set_error(PTS_ERR_INVALID_ARG, "pts_set_allocator: give both functions or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_live.load() != 0)
        return set_error(PTS_ERR_INVALID_ARG,
                         "pts_set_allocator: the library still holds device memory (" + std::to_string(g_live.load()) +
                             " allocations); destroy every index and batch first");
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.user = alloc ? user : nullptr;
    return PTS_OK;
}

long long pts_live_allocations(void) { return g_live.load(); }

pts_status pca_fit(const float *exemplar, int He, int We, int w, int d, double var_frac,
                   float *mean_out, float *basis_out, double *eigvals_out, int *d_out, void *stream) {
    return pca_fit_channels(exemplar, He, We, 3, w, d, var_frac, mean_out, basis_out, eigvals_out, d_out, stream);
}

pts_status pca_fit_channels(const float *exemplar, int He, int We, int C, int w, int d, double var_frac,
                            float *mean_out, float *basis_out, double *eigvals_out, int *d_out, void *stream) {
    if (!exemplar || !basis_out) return set_error(PTS_ERR_INVALID_ARG, "pca_fit: null pointer");
    if (C != 3 && C != 4) return set_error(PTS_ERR_INVALID_ARG, "pca_fit: channels must be 3 or 4");
    if (w < 1 || w > He || w > We) return set_error(PTS_ERR_INVALID_ARG, "pca_fit: bad window");
    if (d > kMaxDPca) return set_error(PTS_ERR_INVALID_ARG, "pca_fit: d > 128");
    if (d <= 0 && !(var_frac > 0.0 && var_frac <= 1.0))
        return set_error(PTS_ERR_INVALID_ARG, "pca_fit: var_frac must be in (0, 1]");
    cudaStream_t st = as_stream(stream);
    DevBuf<int> status;
    PTS_TRY(status.ensure(1, "status"));
    PTS_CUDA_TRY(cudaMemsetAsync(status.ptr, 0, sizeof(int), st));
    int dd = 0;
    pts_status s = pca_fit_device(exemplar, He, We, C, w, d, var_frac, 0, mean_out, basis_out,
                                  eigvals_out, &dd, nullptr, nullptr, nullptr, nullptr, status.ptr, st);
    if (s == PTS_OK) {
        int h = 0;
        cudaMemcpy(&h, status.ptr, sizeof(int), cudaMemcpyDeviceToHost);
        if (h) s = set_error(PTS_ERR_DEVICE, "pca_fit: eigen-solver did not converge cleanly");
    }
    status.release();
    if (d_out) *d_out = dd;
    return s;
}

pts_status build_exemplar_index(const float *exemplar, int He, int We, int w,
                                const pts_index_params *params, void *stream, pts_index *out) {
    if (!out || !exemplar || !params)
        return set_error(PTS_ERR_INVALID_ARG, "build_exemplar_index: null pointer");
    *out = nullptr;
    if (w < 1 || w > He || w > We)
        return set_error(PTS_ERR_INVALID_ARG, "build_exemplar_index: bad window");
    if (params->d > kMaxD) return set_error(PTS_ERR_INVALID_ARG, "build_exemplar_index: d > 64");
    if (params->d_fast > kMaxDFast)
        return set_error(PTS_ERR_INVALID_ARG, "build_exemplar_index: d_fast > 124");
    const long N = (long)(He - w + 1) * (We - w + 1);
    if (N < 2 || N > (1L << 30))
        return set_error(PTS_ERR_INVALID_ARG, "build_exemplar_index: bad exemplar size");
    const int C = params->channels == 0 ? 3 : params->channels;
    if (C != 3 && C != 4) return set_error(PTS_ERR_INVALID_ARG, "build_exemplar_index: channels must be 3 or 4");
    cudaStream_t st = as_stream(stream);
    pts_index idx = new pts_index_s();
    register_index(idx);
    auto fail = [&](pts_status s) {
        pts_index_destroy(idx);
        return s;
    };
    cudaGetDevice(&idx->device);
    idx->He = He;
    idx->We = We;
    idx->w = w;
    idx->C = C;
    idx->D = C * w * w;
    idx->ny = He - w + 1;
    idx->nx = We - w + 1;
    idx->N = (int)N;
    pts_status s;
    if ((s = idx->exemplar.ensure((size_t)He * We * C, "exemplar")) != PTS_OK) return fail(s);
    if ((s = idx->exemplar4.ensure((size_t)He * We, "exemplar rgba")) != PTS_OK) return fail(s);
    if ((s = idx->status.ensure(1, "status")) != PTS_OK) return fail(s);
    if ((s = idx->mu.ensure(idx->D, "mean")) != PTS_OK) return fail(s);
    if ((s = idx->basis.ensure((size_t)kMaxDPca * idx->D, "basis")) != PTS_OK) return fail(s);
    if ((s = idx->eig.ensure(kMaxDPca, "eigenvalues")) != PTS_OK) return fail(s);
    if ((s = idx->umax.ensure(1, "norm max")) != PTS_OK) return fail(s);
    cudaError_t e = cudaMemcpyAsync(idx->exemplar.ptr, exemplar, sizeof(float) * He * We * C,
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(cuda_error(e, "copy exemplar"));
    launch_rgba(idx->exemplar.ptr, (long)He * We, C, idx->exemplar4.ptr, st);
    cudaMemsetAsync(idx->status.ptr, 0, sizeof(int), st);
    // one PCA serves both searches: the exact search uses its first d components, the
    // tensor-core and proposal searches the first d_fast (components are ordered by variance)
    const long rank_cap = std::min<long>(idx->D, N - 1);
    int d_fast = params->d_fast > 0 ? params->d_fast : kMaxDFast;
    d_fast = (int)std::min<long>(d_fast, rank_cap);
    const int d_req = params->d > 0 ? params->d : kMaxD;
    const int d_pca = (int)std::min<long>(std::max(d_req, d_fast), rank_cap);
    int dd = 0;
    double trace = 0.0;
    s = pca_fit_device(idx->exemplar.ptr, He, We, C, w, d_pca, params->var_frac, params->max_iters,
                       idx->mu.ptr, idx->basis.ptr, idx->eig.ptr, &dd, &idx->var_retained,
                       &idx->eig_top, &idx->eig_iters, &trace, idx->status.ptr, st);
    if (s != PTS_OK) return fail(s);
    if ((s = idx->basisT.ensure((size_t)idx->D * kMaxDPca, "transposed basis")) != PTS_OK) return fail(s);
    launch_basis_transpose(idx->basis.ptr, dd, idx->D, idx->basisT.ptr, st);
    if (params->d > 0) {
        dd = std::min(params->d, dd);
    } else {  // smallest d (<= 64) whose eigenvalues reach var_frac of the trace
        std::vector<double> ev(dd);
        cudaMemcpy(ev.data(), idx->eig.ptr, sizeof(double) * dd, cudaMemcpyDeviceToHost);
        double acc = 0.0;
        int pick = std::min(dd, kMaxD);
        for (int j = 0; j < std::min(dd, kMaxD); ++j) {
            acc += ev[j];
            if (acc >= params->var_frac * trace) {
                pick = j + 1;
                break;
            }
        }
        dd = pick;
    }
    {
        std::vector<double> ev(dd);
        cudaMemcpy(ev.data(), idx->eig.ptr, sizeof(double) * dd, cudaMemcpyDeviceToHost);
        double kept = 0.0;
        for (double v : ev) kept += v;
        idx->var_retained = trace > 0 ? kept / trace : 0.0;
    }
    idx->d = dd;
    idx->d_fast = std::max(1, d_fast);
    idx->da_fast = (idx->d_fast + 1 + 3) & ~3;
    idx->da = (dd + 1 + 3) & ~3;
    idx->ntiles = ceil_div(N, kBN);
    if ((s = idx->et.ensure((size_t)idx->ntiles * idx->da * kBN, "exemplar vectors")) != PTS_OK)
        return fail(s);
    if ((s = idx->enorm.ensure((size_t)idx->ntiles * kBN, "exemplar norms")) != PTS_OK) return fail(s);
    launch_exemplar_pad(idx->et.ptr, idx->enorm.ptr, idx->N, idx->ntiles, idx->da, st);
    launch_project(idx->exemplar.ptr, He, We, C, w, 1, idx->mu.ptr, idx->basisT.ptr, dd, idx->da, 1,
                   idx->et.ptr, idx->enorm.ptr, nullptr, 0.0f, nullptr, st);
    launch_norm_max(idx->enorm.ptr, idx->N, idx->umax.ptr, st);
    if ((s = idx->et_rows.ensure((size_t)idx->N * idx->da, "window-major exemplar vectors")) != PTS_OK)
        return fail(s);
    launch_tiles_to_rows(idx->et.ptr, idx->N, idx->da, idx->et_rows.ptr, st);
    if ((s = idx->efull.ensure((size_t)idx->ntiles * padded_dim(idx->D) * kBN, "full exemplar vectors")) !=
        PTS_OK)
        return fail(s);
    launch_exemplar_full(idx->exemplar.ptr, We, C, w, idx->nx, idx->N, idx->mu.ptr, idx->efull.ptr,
                         idx->ntiles, st);
    // fast-mode search vectors: d_fast coordinates + the residual beyond them
    if ((s = idx->et_fast.ensure((size_t)idx->ntiles * idx->da_fast * kBN, "fast exemplar vectors")) != PTS_OK)
        return fail(s);
    {
        DevBuf<float> norm_tmp;
        if ((s = norm_tmp.ensure((size_t)idx->ntiles * kBN, "norm scratch")) != PTS_OK) return fail(s);
        launch_exemplar_pad(idx->et_fast.ptr, norm_tmp.ptr, idx->N, idx->ntiles, idx->da_fast, st);
        launch_project(idx->exemplar.ptr, He, We, C, w, 1, idx->mu.ptr, idx->basisT.ptr, idx->d_fast, idx->da_fast, 1,
                       idx->et_fast.ptr, norm_tmp.ptr, nullptr, 0.0f, nullptr, st);
        cudaStreamSynchronize(st);
        norm_tmp.release();
    }
    if ((s = idx->et_fast_rows.ensure((size_t)idx->N * idx->da_fast, "window-major fast exemplar vectors")) != PTS_OK)
        return fail(s);
    launch_tiles_to_rows(idx->et_fast.ptr, idx->N, idx->da_fast, idx->et_fast_rows.ptr, st);
    {
        std::vector<double> ev(idx->d_fast);
        cudaMemcpy(ev.data(), idx->eig.ptr, sizeof(double) * idx->d_fast, cudaMemcpyDeviceToHost);
        double kept = 0.0;
        for (double v : ev) kept += v;
        idx->var_fast = trace > 0 ? kept / trace : 0.0;
    }
    idx->ktc = tc_padded_k(idx->d_fast);
    if ((s = idx->etc.ensure((size_t)tc_tiles(idx->N) * tc_tile_rows() * idx->ktc, "fp16 exemplar tiles")) != PTS_OK)
        return fail(s);
    launch_pack_exemplar(idx->et_fast.ptr, idx->enorm.ptr, idx->N, idx->d_fast, idx->da_fast, idx->ktc, idx->etc.ptr,
                         st);
    idx->kf8 = tc_padded_k8(idx->d_fast);
    if ((s = idx->etc8.ensure((size_t)tc_tiles(idx->N) * tc_tile_rows() * idx->kf8, "fp8 exemplar tiles")) != PTS_OK)
        return fail(s);
    if ((s = idx->f8scale.ensure((size_t)idx->d_fast + 1, "fp8 scales")) != PTS_OK) return fail(s);
    launch_fp8_tables(idx->et_fast.ptr, idx->N, idx->d_fast, idx->da_fast, idx->kf8, idx->f8scale.ptr, idx->etc8.ptr,
                      st);
    e = cudaMemcpyAsync(&idx->unorm2_max, idx->umax.ptr, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return fail(cuda_error(e, "read norm max"));
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(cuda_error(e, "build_exemplar_index"));
    if ((s = read_status(idx, st)) != PTS_OK) return fail(s);
    *out = idx;
    return PTS_OK;
}

void pts_index_destroy(pts_index idx) {
    if (!idx) return;
    unregister_index(idx);
    cudaDeviceSynchronize();
    Workspace &ws = idx->ws;
    ws.qcoord.release();
    ws.qnorm.release();
    ws.tau.release();
    ws.cand_idx.release();
    ws.cand_lb.release();
    ws.fail_list.release();
    ws.fail2_list.release();
    ws.qfull.release();
    ws.full_pdist.release();
    ws.best64.release();
    ws.counters.release();
    ws.nn.release();
    ws.d2.release();
    ws.wts.release();
    ws.energy.release();
    ws.partial.release();
    ws.ticket.release();
    ws.thr0.release();
    ws.pca_thr.release();
    ws.qtile.release();
    ws.qtile8.release();
    ws.qscale.release();
    ws.proj_part.release();
    ws.kept.release();
    ws.part_v.release();
    ws.part_i.release();
    ws.hist.release();
    ws.nn_prev.release();
    ws.diff.release();
    idx->exemplar.release();
    idx->exemplar4.release();
    idx->mu.release();
    idx->basis.release();
    idx->basisT.release();
    idx->eig.release();
    idx->et.release();
    idx->et_rows.release();
    idx->enorm.release();
    idx->efull.release();
    idx->etc.release();
    idx->etc8.release();
    idx->f8scale.release();
    idx->et_fast.release();
    idx->et_fast_rows.release();
    {
        ProposalState &pr = idx->prop;
        pr.centroids.release();
        pr.assign.release();
        pr.counts.release();
        pr.off.release();
        pr.members.release();
        pr.median.release();
        pr.top.release();
        pr.etc_ivf.release();
        for (auto *b : {&pr.ivf_cnt, &pr.ivf_poff, &pr.ivf_cursor, &pr.ivf_nblk, &pr.pair_q, &pr.pair_r, &pr.ivf_part_i})
            b->release();
        pr.ivf_blk.release();
        pr.ivf_qtile.release();
        pr.ivf_part_v.release();
        pr.ivf_kept.release();
        pr.infer.wp1.release();
        pr.infer.wp2.release();
        pr.infer.wp3.release();
        pr.infer.b3p.release();
        KmTree &tr = idx->tree;
        for (auto *b : {&tr.child, &tr.leaf_begin, &tr.leaf_end, &tr.perm, &tr.tmp, &tr.leaf_of_query}) b->release();
        tr.cent.release();
        tr.label.release();
        MlpState &m = pr.mlp;
        for (auto *b : {&m.params, &m.grads, &m.adam_m, &m.adam_v, &m.a1, &m.a2, &m.z, &m.dh, &m.loss}) b->release();
        for (auto *b : {&m.wb, &m.wt, &m.xb, &m.xt, &m.h1b, &m.h1t, &m.h2b, &m.h2t, &m.dzb, &m.dzt, &m.dab, &m.dat})
            b->release();
        m.labels.release();
    }
    idx->umax.release();
    idx->status.release();
    delete idx;
}

pts_status pts_index_get_info(pts_index idx, pts_index_info *info) {
    if (!idx || !info) return set_error(PTS_ERR_INVALID_ARG, "pts_index_get_info: null pointer");
    info->He = idx->He;
    info->We = idx->We;
    info->w = idx->w;
    info->D = idx->D;
    info->N = idx->N;
    info->d = idx->d;
    info->da = idx->da;
    info->d_fast = idx->d_fast;
    info->var_retained = idx->var_retained;
    info->eig_top = idx->eig_top;
    info->eig_iters = idx->eig_iters;
    info->unorm2_max = idx->unorm2_max;
    info->channels = idx->C;
    const bool fast = idx->exact_fast == 1 && idx->d_fast > idx->d;
    info->exact_dims = fast ? idx->d_fast : idx->d;
    info->exact_var = fast ? idx->var_fast : idx->var_retained;
    return PTS_OK;
}

pts_status pts_index_set_exact_bound(pts_index idx, int fast) {
    if (!idx || fast < 0 || fast > 2) return set_error(PTS_ERR_INVALID_ARG, "pts_index_set_exact_bound: bad argument");
    idx->exact_fast = fast;
    return PTS_OK;
}

pts_status pts_index_set_tc_parts(pts_index idx, int parts) {
    if (!idx || parts < 0) return set_error(PTS_ERR_INVALID_ARG, "pts_index_set_tc_parts: null index or parts < 0");
    idx->tc_parts_override = parts;
    return PTS_OK;
}

pts_status pts_build_kmeans_tree(pts_index idx, int iters, void *stream) {
    if (!idx || iters < 1 || iters > 100)
        return set_error(PTS_ERR_INVALID_ARG, "pts_build_kmeans_tree: null index or iters outside 1..100");
    idx->tree.ready = 0;
    return build_kmtree(idx->tree, idx->et_rows.ptr, idx->N, idx->da, idx->d, iters, as_stream(stream));
}

pts_status pts_kmtree_info(pts_index idx, int *n_internal, int *n_leaves, int *depth) {
    if (!idx || !idx->tree.ready) return set_error(PTS_ERR_INVALID_ARG, "pts_kmtree_info: no k-means tree built");
    if (n_internal) *n_internal = idx->tree.n_internal;
    if (n_leaves) *n_leaves = idx->tree.n_leaves;
    if (depth) *depth = idx->tree.depth;
    return PTS_OK;
}

pts_status pts_kmtree_export(pts_index idx, int *child, int *leaf_begin, int *leaf_end, int *perm, float *cent,
                             void *stream) {
    if (!idx || !idx->tree.ready) return set_error(PTS_ERR_INVALID_ARG, "pts_kmtree_export: no k-means tree built");
    const KmTree &tr = idx->tree;
    cudaStream_t st = as_stream(stream);
    if (child)
        PTS_CUDA_TRY(cudaMemcpyAsync(child, tr.child.ptr, sizeof(int) * 4 * tr.n_internal, cudaMemcpyDeviceToHost, st));
    if (leaf_begin)
        PTS_CUDA_TRY(cudaMemcpyAsync(leaf_begin, tr.leaf_begin.ptr, sizeof(int) * tr.n_leaves, cudaMemcpyDeviceToHost,
                                     st));
    if (leaf_end)
        PTS_CUDA_TRY(cudaMemcpyAsync(leaf_end, tr.leaf_end.ptr, sizeof(int) * tr.n_leaves, cudaMemcpyDeviceToHost, st));
    if (perm) PTS_CUDA_TRY(cudaMemcpyAsync(perm, tr.perm.ptr, sizeof(int) * tr.N, cudaMemcpyDeviceToHost, st));
    if (cent)
        PTS_CUDA_TRY(cudaMemcpyAsync(cent, tr.cent.ptr, sizeof(float) * 4 * (size_t)tr.n_internal * tr.d,
                                     cudaMemcpyDeviceToHost, st));
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    return PTS_OK;
}

pts_status pts_kmtree_last_leaves(pts_index idx, int *leaves, int Q, void *stream) {
    if (!idx || !leaves || Q < 0) return set_error(PTS_ERR_INVALID_ARG, "pts_kmtree_last_leaves: bad argument");
    if (!idx->tree.ready || idx->tree.leaf_of_query.count < (size_t)Q)
        return set_error(PTS_ERR_INVALID_ARG, "pts_kmtree_last_leaves: no tree search of that size");
    cudaStream_t st = as_stream(stream);
    PTS_CUDA_TRY(cudaMemcpyAsync(leaves, idx->tree.leaf_of_query.ptr, sizeof(int) * Q, cudaMemcpyDeviceToHost, st));
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    return PTS_OK;
}

pts_status pts_index_device_status(pts_index idx, void *stream) {
    if (!idx) return set_error(PTS_ERR_INVALID_ARG, "pts_index_device_status: null index");
    return read_status(idx, as_stream(stream));
}

pts_status nn_search(pts_index idx, const float *output, int Ho, int Wo, int stride, int mode,
                     int32_t *nn_out, float *dist2_out, void *stream) {
    if (!idx) return set_error(PTS_ERR_INVALID_ARG, "nn_search: null index");
    return nn_search_impl(idx, output, Ho, Wo, stride, mode, nn_out, dist2_out, as_stream(stream));
}

pts_status pts_index_search_stats(pts_index idx, pts_search_stats *stats, void *stream) {
    if (!idx || !stats) return set_error(PTS_ERR_INVALID_ARG, "pts_index_search_stats: null pointer");
    cudaStream_t st = as_stream(stream);
    *stats = idx->last;
    stats->fallback_queries = 0;
    const bool exact_route = idx->last_mode == PTS_EXACT_F32 || idx->last_mode == PTS_EXACT_TC;
    if (idx->ws.counters.ptr && (exact_route || idx->last_mode == PTS_PROPOSAL)) {
        unsigned int c[4] = {0, 0, 0, 0};
        PTS_CUDA_TRY(cudaMemcpyAsync(c, idx->ws.counters.ptr, sizeof(c), cudaMemcpyDeviceToHost, st));
        PTS_CUDA_TRY(cudaStreamSynchronize(st));
        stats->second_certified = 0;
        stats->second_queries = 0;
        if (exact_route) {
            // PTS_EXACT_TC: c[0] queries the FP16 GEMM's candidates left uncertified (the first
            // bound's role), c[1] of those still uncertified after the full pass
            stats->range_queries = c[0];
            stats->certified = stats->queries - c[0];
            // with the second bound: c[1] of the c[0] queries reached the full pass, c[3] of those
            // stayed uncertified
            stats->full_queries = idx->last_cascade ? c[1] : c[0];
            stats->second_certified = idx->last_cascade ? c[0] - c[1] : 0;
            stats->second_queries = idx->last_cascade ? c[0] : 0;
            stats->range_pairs = idx->last_cascade ? c[3] : c[1];
        } else {
            stats->fallback_queries = c[0];
            stats->range_queries = 0;
            stats->certified = 0;
            stats->full_queries = 0;
            stats->range_pairs = c[1];
        }
        stats->brute_queries = c[2];
    }
    return PTS_OK;
}

pts_status irls_weights(const float *dist2, int Q, float r, float delta, float *weights_out,
                        double *energy_out, void *stream) {
    if (!dist2 || Q < 0) return set_error(PTS_ERR_INVALID_ARG, "irls_weights: bad input");
    if (!(r > 0.0f && r <= 2.0f) || !(delta > 0.0f))
        return set_error(PTS_ERR_INVALID_ARG, "irls_weights: need 0 < r <= 2 and delta > 0");
    cudaStream_t st = as_stream(stream);
    DevBuf<double> partial;
    DevBuf<unsigned int> ticket;
    PTS_TRY(partial.ensure(kIrlsGrid, "partials"));
    PTS_TRY(ticket.ensure(1, "ticket"));
    PTS_CUDA_TRY(cudaMemsetAsync(ticket.ptr, 0, sizeof(unsigned int), st));
    launch_irls(dist2, Q, r, delta, weights_out, energy_out, partial.ptr, ticket.ptr, st);
    cudaError_t e = cudaStreamSynchronize(st);
    partial.release();
    ticket.release();
    if (e != cudaSuccess) return cuda_error(e, "irls_weights");
    return PTS_OK;
}

pts_status m_step(pts_index idx, const int32_t *nn, const float *weights, int Ho, int Wo,
                  int stride, float *output, void *stream) {
    if (!idx || !nn || !output) return set_error(PTS_ERR_INVALID_ARG, "m_step: null pointer");
    PTS_TRY(check_grid(Ho, Wo, idx->w, stride, "m_step"));
    launch_m_step(nn, weights, idx->exemplar4.ptr, idx->We, idx->nx, idx->N, idx->C, idx->w, Ho, Wo, stride,
                  output, idx->status.ptr, as_stream(stream));
    PTS_CUDA_TRY(cudaGetLastError());
    return PTS_OK;
}

pts_status m_step_hist(pts_index idx, const int32_t *nn, const float *weights, int Ho, int Wo, int stride, int nbins,
                       const float *current, float *output, void *stream) {
    if (!idx || !nn || !output || !current) return set_error(PTS_ERR_INVALID_ARG, "m_step_hist: null pointer");
    if (nbins < 2 || nbins > kMaxHistBins) return set_error(PTS_ERR_INVALID_ARG, "m_step_hist: nbins in 2..256");
    if (idx->C != 3) return set_error(PTS_ERR_INVALID_ARG, "m_step_hist: histogram weights need an RGB index");
    PTS_TRY(check_grid(Ho, Wo, idx->w, stride, "m_step_hist"));
    cudaStream_t st = as_stream(stream);
    Workspace &ws = idx->ws;
    PTS_TRY(ws.hist.ensure(6 * kMaxHistBins, "histograms"));
    unsigned int *cx = ws.hist.ptr, *cz = ws.hist.ptr + 3 * kMaxHistBins;
    const long nx = (long)Ho * Wo, nz = (long)idx->He * idx->We;
    launch_hist3(current, nx, nbins, cx, st);
    launch_hist3(idx->exemplar.ptr, nz, nbins, cz, st);
    launch_m_step_hist(nn, weights, idx->exemplar4.ptr, idx->We, idx->nx, idx->N, idx->w, Ho, Wo, stride, nbins, cx, nx,
                       cz, nz, output, idx->status.ptr, st);
    PTS_CUDA_TRY(cudaGetLastError());
    return PTS_OK;
}

pts_status pts_histogram_match(pts_index idx, float *image, int H, int W, int nbins, void *stream) {
    if (!idx || !image) return set_error(PTS_ERR_INVALID_ARG, "pts_histogram_match: null pointer");
    if (nbins < 2 || nbins > kMaxHistBins)
        return set_error(PTS_ERR_INVALID_ARG, "pts_histogram_match: nbins in 2..256");
    if (idx->C != 3) return set_error(PTS_ERR_INVALID_ARG, "pts_histogram_match: needs an RGB index");
    if (H < 1 || W < 1) return set_error(PTS_ERR_INVALID_ARG, "pts_histogram_match: empty image");
    cudaStream_t st = as_stream(stream);
    Workspace &ws = idx->ws;
    PTS_TRY(ws.hist.ensure(6 * kMaxHistBins, "histograms"));
    unsigned int *cx = ws.hist.ptr, *cz = ws.hist.ptr + 3 * kMaxHistBins;
    const long nx = (long)H * W, nz = (long)idx->He * idx->We;
    launch_hist3(image, nx, nbins, cx, st);
    launch_hist3(idx->exemplar.ptr, nz, nbins, cz, st);
    launch_hist_match(image, nx, nbins, cx, nx, cz, nz, st);
    PTS_CUDA_TRY(cudaGetLastError());
    return PTS_OK;
}

// the EM loop of synthesize_level; nbins > 0 takes the M-step of m_step_hist
static pts_status synthesize_impl(pts_index idx, float *output, int Ho, int Wo, int stride, int iters, float r,
                                  float delta, int mode, int nbins, double *energy_out, void *stream,
                                  const char *name, double *energy_dev = nullptr) {
    if (!idx || !output || !energy_out) return set_error(PTS_ERR_INVALID_ARG, std::string(name) + ": null pointer");
    if (iters < 0) return set_error(PTS_ERR_INVALID_ARG, std::string(name) + ": iters < 0");
    if (!(r > 0.0f && r <= 2.0f) || !(delta > 0.0f))
        return set_error(PTS_ERR_INVALID_ARG, std::string(name) + ": need 0 < r <= 2 and delta > 0");
    if (nbins != 0 && (nbins < 2 || nbins > kMaxHistBins))
        return set_error(PTS_ERR_INVALID_ARG, std::string(name) + ": nbins in 2..256");
    if (nbins != 0 && idx->C != 3)
        return set_error(PTS_ERR_INVALID_ARG, std::string(name) + ": histogram weights need an RGB index");
    PTS_TRY(check_grid(Ho, Wo, idx->w, stride, name));
    cudaStream_t st = as_stream(stream);
    const int Q = ((Ho - idx->w) / stride + 1) * ((Wo - idx->w) / stride + 1);
    PTS_TRY(ensure_workspace(idx, Q));
    Workspace &ws = idx->ws;
    PTS_TRY(ws.energy.ensure(iters + 1, "energies"));
    double *energy = energy_dev ? energy_dev : ws.energy.ptr;
    unsigned int *cx = nullptr, *cz = nullptr;
    const long nx = (long)Ho * Wo, nz = (long)idx->He * idx->We;
    if (nbins) {
        PTS_TRY(ws.hist.ensure(6 * kMaxHistBins, "histograms"));
        cx = ws.hist.ptr;
        cz = ws.hist.ptr + 3 * kMaxHistBins;
        launch_hist3(idx->exemplar.ptr, nz, nbins, cz, st);
    }
    for (int t = 0; t <= iters; ++t) {
        PTS_TRY(nn_search_impl(idx, output, Ho, Wo, stride, mode, ws.nn.ptr, ws.d2.ptr, st));
        launch_irls(ws.d2.ptr, Q, r, delta, ws.wts.ptr, energy + t, ws.partial.ptr, ws.ticket.ptr, st);
        if (t == iters) break;
        if (nbins) {
            launch_hist3(output, nx, nbins, cx, st);  // of the image the E-step matched
            launch_m_step_hist(ws.nn.ptr, ws.wts.ptr, idx->exemplar4.ptr, idx->We, idx->nx, idx->N, idx->w, Ho, Wo,
                               stride, nbins, cx, nx, cz, nz, output, idx->status.ptr, st);
        } else {
            launch_m_step(ws.nn.ptr, ws.wts.ptr, idx->exemplar4.ptr, idx->We, idx->nx, idx->N, idx->C, idx->w, Ho,
                          Wo, stride, output, idx->status.ptr, st);
        }
    }
    PTS_CUDA_TRY(cudaGetLastError());
    if (energy_dev) return PTS_OK;  // asynchronous: the caller reads the device status later
    PTS_CUDA_TRY(cudaMemcpyAsync(energy_out, ws.energy.ptr, sizeof(double) * (iters + 1),
                                 cudaMemcpyDeviceToHost, st));
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    return read_status(idx, st);
}

pts_status synthesize_level_async(pts_index idx, float *output, int Ho, int Wo, int stride, int iters, float r,
                                  float delta, int mode, double *energy_dev, void *stream) {
    if (!energy_dev) return set_error(PTS_ERR_INVALID_ARG, "synthesize_level_async: null pointer");
    return synthesize_impl(idx, output, Ho, Wo, stride, iters, r, delta, mode, 0, energy_dev, stream,
                           "synthesize_level_async", energy_dev);
}

pts_status synthesize_level(pts_index idx, float *output, int Ho, int Wo, int stride, int iters, float r, float delta,
                            int mode, double *energy_out, void *stream) {
    return synthesize_impl(idx, output, Ho, Wo, stride, iters, r, delta, mode, 0, energy_out, stream,
                           "synthesize_level");
}

pts_status synthesize_level_converge(pts_index idx, float *output, int Ho, int Wo, int stride, int max_iters, float r,
                                     float delta, int mode, int nbins, double *energy_out, int *iters_out,
                                     void *stream) {
    const char *name = "synthesize_level_converge";
    if (!idx || !output || !energy_out || !iters_out)
        return set_error(PTS_ERR_INVALID_ARG, std::string(name) + ": null pointer");
    if (max_iters < 0) return set_error(PTS_ERR_INVALID_ARG, std::string(name) + ": max_iters < 0");
    if (!(r > 0.0f && r <= 2.0f) || !(delta > 0.0f))
        return set_error(PTS_ERR_INVALID_ARG, std::string(name) + ": need 0 < r <= 2 and delta > 0");
    if (nbins != 0 && (nbins < 2 || nbins > kMaxHistBins))
        return set_error(PTS_ERR_INVALID_ARG, std::string(name) + ": nbins 0 or in 2..256");
    if (nbins != 0 && idx->C != 3)
        return set_error(PTS_ERR_INVALID_ARG, std::string(name) + ": histogram weights need an RGB index");
    PTS_TRY(check_grid(Ho, Wo, idx->w, stride, name));
    cudaStream_t st = as_stream(stream);
    const int Q = ((Ho - idx->w) / stride + 1) * ((Wo - idx->w) / stride + 1);
    PTS_TRY(ensure_workspace(idx, Q));
    Workspace &ws = idx->ws;
    PTS_TRY(ws.energy.ensure(max_iters + 1, "energies"));
    PTS_TRY(ws.nn_prev.ensure((size_t)std::max(Q, 1), "previous windows"));
    PTS_TRY(ws.diff.ensure(1, "changed windows"));
    unsigned int *cx = nullptr, *cz = nullptr;
    const long nx = (long)Ho * Wo, nz = (long)idx->He * idx->We;
    if (nbins) {
        PTS_TRY(ws.hist.ensure(6 * kMaxHistBins, "histograms"));
        cx = ws.hist.ptr;
        cz = ws.hist.ptr + 3 * kMaxHistBins;
        launch_hist3(idx->exemplar.ptr, nz, nbins, cz, st);
    }
    int it = 0;
    PTS_TRY(nn_search_impl(idx, output, Ho, Wo, stride, mode, ws.nn.ptr, ws.d2.ptr, st));
    launch_irls(ws.d2.ptr, Q, r, delta, ws.wts.ptr, ws.energy.ptr, ws.partial.ptr, ws.ticket.ptr, st);
    while (it < max_iters) {
        if (nbins) {
            launch_hist3(output, nx, nbins, cx, st);
            launch_m_step_hist(ws.nn.ptr, ws.wts.ptr, idx->exemplar4.ptr, idx->We, idx->nx, idx->N, idx->w, Ho, Wo,
                               stride, nbins, cx, nx, cz, nz, output, idx->status.ptr, st);
        } else {
            launch_m_step(ws.nn.ptr, ws.wts.ptr, idx->exemplar4.ptr, idx->We, idx->nx, idx->N, idx->C, idx->w, Ho, Wo, stride,
                          output, idx->status.ptr, st);
        }
        PTS_CUDA_TRY(cudaMemcpyAsync(ws.nn_prev.ptr, ws.nn.ptr, sizeof(int) * Q, cudaMemcpyDeviceToDevice, st));
        ++it;
        PTS_TRY(nn_search_impl(idx, output, Ho, Wo, stride, mode, ws.nn.ptr, ws.d2.ptr, st));
        launch_irls(ws.d2.ptr, Q, r, delta, ws.wts.ptr, ws.energy.ptr + it, ws.partial.ptr, ws.ticket.ptr, st);
        launch_count_diff(ws.nn.ptr, ws.nn_prev.ptr, Q, ws.diff.ptr, st);
        unsigned int changed = 0;
        PTS_CUDA_TRY(cudaMemcpyAsync(&changed, ws.diff.ptr, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
        PTS_CUDA_TRY(cudaStreamSynchronize(st));
        if (changed == 0) break;
    }
    PTS_CUDA_TRY(cudaGetLastError());
    PTS_CUDA_TRY(cudaMemcpyAsync(energy_out, ws.energy.ptr, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost, st));
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    *iters_out = it;
    return read_status(idx, st);
}

pts_status synthesize_level_hist(pts_index idx, float *output, int Ho, int Wo, int stride, int iters, float r,
                                 float delta, int mode, int nbins, double *energy_out, void *stream) {
    if (nbins == 0) return set_error(PTS_ERR_INVALID_ARG, "synthesize_level_hist: nbins in 2..256");
    return synthesize_impl(idx, output, Ho, Wo, stride, iters, r, delta, mode, nbins, energy_out, stream,
                           "synthesize_level_hist");
}

pts_status pts_project_queries(pts_index idx, const float *output, int Ho, int Wo, int stride, float *y_out,
                               void *stream) {
    if (!idx || !output || !y_out) return set_error(PTS_ERR_INVALID_ARG, "pts_project_queries: null pointer");
    PTS_TRY(check_grid(Ho, Wo, idx->w, stride, "pts_project_queries"));
    const int Q = ((Ho - idx->w) / stride + 1) * ((Wo - idx->w) / stride + 1);
    PTS_TRY(ensure_workspace(idx, Q));
    cudaStream_t st = as_stream(stream);
    Workspace &ws = idx->ws;
    launch_project(output, Ho, Wo, idx->C, idx->w, stride, idx->mu.ptr, idx->basisT.ptr, idx->d, idx->da, 0, ws.qcoord.ptr,
                   ws.qnorm.ptr, ws.tau.ptr, 0.0f, idx->umax.ptr, st);
    PTS_CUDA_TRY(cudaMemcpy2DAsync(y_out, sizeof(float) * idx->d, ws.qcoord.ptr, sizeof(float) * idx->da,
                                   sizeof(float) * idx->d, Q, cudaMemcpyDeviceToDevice, st));
    return PTS_OK;
}

pts_status pts_index_pca(pts_index idx, float *mean_out, float *basis_out, void *stream) {
    if (!idx || !mean_out || !basis_out) return set_error(PTS_ERR_INVALID_ARG, "pts_index_pca: null pointer");
    cudaStream_t st = as_stream(stream);
    PTS_CUDA_TRY(cudaMemcpyAsync(mean_out, idx->mu.ptr, sizeof(float) * idx->D, cudaMemcpyDeviceToDevice, st));
    PTS_CUDA_TRY(cudaMemcpyAsync(basis_out, idx->basis.ptr, sizeof(float) * idx->D * idx->d_fast,
                                 cudaMemcpyDeviceToDevice, st));
    return PTS_OK;
}

pts_status pts_query_rows_f16(pts_index idx, const float *output, int Ho, int Wo, int stride, int tensor_cores,
                              uint16_t *rows_out, float *norm_out, void *stream) {
    if (!idx || !output || !rows_out || !norm_out)
        return set_error(PTS_ERR_INVALID_ARG, "pts_query_rows_f16: null pointer");
    PTS_TRY(check_grid(Ho, Wo, idx->w, stride, "pts_query_rows_f16"));
    const int Q = ((Ho - idx->w) / stride + 1) * ((Wo - idx->w) / stride + 1);
    PTS_TRY(ensure_workspace(idx, Q));
    cudaStream_t st = as_stream(stream);
    Workspace &ws = idx->ws;
    PTS_TRY(ws.qtile.ensure((size_t)tc_query_blocks(Q) * kTcQueryRows * idx->ktc, "query operand tiles"));
    PTS_TRY(project_f16_rows(idx, output, Ho, Wo, stride, tensor_cores, norm_out, st));
    launch_tile16_rows(ws.qtile.ptr, Q, idx->ktc, reinterpret_cast<__half *>(rows_out), st);
    return PTS_OK;
}

pts_status pts_proposal_top4(pts_index idx, const float *output, int Ho, int Wo, int stride, int fused,
                             int32_t *top_out, void *stream) {
    if (!idx || !output || !top_out) return set_error(PTS_ERR_INVALID_ARG, "pts_proposal_top4: null pointer");
    ProposalState &pr = idx->prop;
    if (!pr.ready) return set_error(PTS_ERR_INVALID_ARG, "pts_proposal_top4: no proposal trained on this index");
    PTS_TRY(check_grid(Ho, Wo, idx->w, stride, "pts_proposal_top4"));
    cudaStream_t st = as_stream(stream);
    const int Q = ((Ho - idx->w) / stride + 1) * ((Wo - idx->w) / stride + 1);
    PTS_TRY(ensure_workspace(idx, Q));
    Workspace &ws = idx->ws;
    launch_project(output, Ho, Wo, idx->C, idx->w, stride, idx->mu.ptr, idx->basisT.ptr, idx->d_fast, idx->da_fast, 0,
                   ws.qcoord.ptr, ws.qnorm.ptr, ws.tau.ptr, 0.0f, idx->umax.ptr, st, &ws.proj_part);
    if (fused) {
        launch_mlp_top4(pr.infer, ws.qcoord.ptr, Q, std::min(idx->d, 64), idx->da_fast, top_out, idx->status.ptr, st);
    } else {
        PTS_TRY(pr.mlp.ensure(pr.C, std::min(Q, kMlpChunk), st));
        for (int q0 = 0; q0 < Q; q0 += kMlpChunk) {
            const int B = std::min(kMlpChunk, Q - q0);
            mlp_gather(pr.mlp, ws.qcoord.ptr + (size_t)q0 * idx->da_fast, std::min(idx->d, 64), idx->da_fast, nullptr,
                       0, B, nullptr, st);
            mlp_forward(pr.mlp, B, 0, idx->status.ptr, st);
            launch_top4(pr.mlp.z.ptr, B, pr.C, top_out + (size_t)q0 * 4, st);
        }
    }
    PTS_CUDA_TRY(cudaGetLastError());
    return PTS_OK;
}

pts_status pts_proposal_info(pts_index idx, int *n_clusters, int *sizes_out, int *assign_out) {
    if (!idx || !n_clusters) return set_error(PTS_ERR_INVALID_ARG, "pts_proposal_info: null pointer");
    ProposalState &pr = idx->prop;
    if (!pr.ready) return set_error(PTS_ERR_INVALID_ARG, "pts_proposal_info: no proposal trained on this index");
    PTS_CUDA_TRY(cudaSetDevice(idx->device));
    *n_clusters = pr.C;
    PTS_CUDA_TRY(cudaDeviceSynchronize());
    if (sizes_out) PTS_CUDA_TRY(cudaMemcpy(sizes_out, pr.counts.ptr, sizeof(int) * pr.C, cudaMemcpyDeviceToHost));
    if (assign_out) PTS_CUDA_TRY(cudaMemcpy(assign_out, pr.assign.ptr, sizeof(int) * idx->N, cudaMemcpyDeviceToHost));
    return PTS_OK;
}

pts_status pts_train_proposal(pts_index idx, const float *y, const int32_t *nn, const float *d2, int n,
                              const pts_proposal_params *prm, double *loss_out, void *stream) {
    if (!idx || !y || !nn || !d2 || !prm) return set_error(PTS_ERR_INVALID_ARG, "pts_train_proposal: null pointer");
    const int C = prm->n_clusters;
    if (C < 4 || C > 1024 || C > idx->N) return set_error(PTS_ERR_INVALID_ARG, "pts_train_proposal: bad n_clusters");
    const int iters = prm->kmeans_iters > 0 ? prm->kmeans_iters : 25;
    const int epochs = prm->epochs > 0 ? prm->epochs : 8;
    const int batch = prm->batch > 0 ? prm->batch : 4096;
    if (batch % 8) return set_error(PTS_ERR_INVALID_ARG, "pts_train_proposal: batch must be a multiple of 8");
    if (n < batch) return set_error(PTS_ERR_INVALID_ARG, "pts_train_proposal: fewer pairs than one batch");
    const float lr = prm->lr > 0 ? prm->lr : 1e-3f;
    const float wd = prm->weight_decay > 0 ? prm->weight_decay : 1e-4f;
    cudaStream_t st = as_stream(stream);
    ProposalState &pr = idx->prop;
    pr.ready = 0;
    pr.C = C;
    pr.factor = prm->fallback_factor > 0 ? prm->fallback_factor : 1.2f;
    const int N = idx->N, d = idx->d, da = idx->da;
    // SplitMix64 stream of the method's random draws (k-means++ uniforms, init, batch order)
    uint64_t state = prm->seed;
    auto next_u64 = [&]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto uniform = [&]() { return (double)(next_u64() >> 11) * (1.0 / 9007199254740992.0); };
    DevBuf<float> Y, cost;
    PTS_TRY(Y.ensure((size_t)N * d, "proposal points"));
    PTS_TRY(cost.ensure(N, "kmeans cost"));
    PTS_TRY(pr.centroids.ensure((size_t)C * d, "centroids"));
    PTS_TRY(pr.assign.ensure(N, "cluster of each window"));
    PTS_TRY(pr.counts.ensure(C, "cluster sizes"));
    PTS_TRY(pr.off.ensure(C + 1, "cluster offsets"));
    PTS_TRY(pr.members.ensure(N, "cluster members"));
    PTS_TRY(pr.median.ensure(C, "cluster medians"));
    launch_extract_y(idx->et.ptr, N, da, d, Y.ptr, st);
    std::vector<double> u(C);
    for (int i = 0; i < C; ++i) u[i] = uniform();
    PTS_TRY(kmeans_device(Y.ptr, N, d, C, u.data(), iters, pr.centroids.ptr, pr.assign.ptr, cost.ptr, pr.counts.ptr,
                          pr.off.ptr, pr.members.ptr, nullptr, st));
    // the exemplar's FP16 search tiles with the windows in cluster order, for the probe
    PTS_TRY(pr.etc_ivf.ensure((size_t)tc_tiles(N) * tc_tile_rows() * idx->ktc, "cluster-ordered tiles"));
    launch_pack_exemplar(idx->et_fast.ptr, idx->enorm.ptr, N, idx->d_fast, idx->da_fast, idx->ktc, pr.etc_ivf.ptr, st,
                         pr.members.ptr);
    DevBuf<int> lab;
    DevBuf<float> dist;
    PTS_TRY(lab.ensure(n, "pair labels"));
    PTS_TRY(dist.ensure(n, "pair distances"));
    PTS_TRY(cluster_medians(nn, d2, n, pr.assign.ptr, N, C, lab.ptr, dist.ptr, pr.median.ptr, st));
    // network: Kaiming-normal weights (Box-Muller on the same stream), zero biases
    MlpState &m = pr.mlp;
    PTS_TRY(m.ensure(C, std::max(batch, kMlpChunk), st));
    const long np = mlp_param_count(C);
    std::vector<float> hp(np, 0.0f);
    auto normal = [&]() {
        const double u1 = uniform(), u2 = uniform();
        return std::sqrt(-2.0 * std::log1p(-u1)) * std::cos(6.283185307179586 * u2);
    };
    long o = 0;
    const int fan_in[3] = {64, kMlpH, kMlpH}, fan_out[3] = {kMlpH, kMlpH, C};
    for (int l = 0; l < 3; ++l) {
        const double sdev = std::sqrt(2.0 / fan_in[l]);
        for (long i = 0; i < (long)fan_out[l] * fan_in[l]; ++i) hp[o + i] = (float)(sdev * normal());
        o += (long)fan_out[l] * fan_in[l] + fan_out[l];
    }
    PTS_CUDA_TRY(cudaMemcpyAsync(m.params.ptr, hp.data(), sizeof(float) * np, cudaMemcpyHostToDevice, st));
    PTS_CUDA_TRY(cudaMemsetAsync(m.adam_m.ptr, 0, sizeof(float) * np, st));
    PTS_CUDA_TRY(cudaMemsetAsync(m.adam_v.ptr, 0, sizeof(float) * np, st));
    mlp_refresh_bf16(m, st);
    DevBuf<int> perm;
    PTS_TRY(perm.ensure(n, "batch order"));
    std::vector<int> hperm(n);
    std::vector<float> hloss(batch);
    const int steps_per_epoch = n / batch;
    const long total_steps = (long)steps_per_epoch * epochs;
    long step = 0;
    for (int e = 0; e < epochs; ++e) {
        for (int i = 0; i < n; ++i) hperm[i] = i;
        for (int i = n - 1; i > 0; --i) std::swap(hperm[i], hperm[(int)(uniform() * (i + 1))]);
        PTS_CUDA_TRY(cudaMemcpyAsync(perm.ptr, hperm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        double esum = 0.0;
        for (int b = 0; b < steps_per_epoch; ++b) {
            ++step;
            const float lr_t = lr * 0.5f * (1.0f + cosf(3.14159265f * (float)(step - 1) / (float)total_steps));
            mlp_gather(m, y, d, d, perm.ptr, b * batch, batch, lab.ptr, st);
            mlp_forward(m, batch, 1, idx->status.ptr, st);
            mlp_backward(m, batch, m.labels.ptr, idx->status.ptr, st);
            mlp_adamw(m, lr_t, wd, (int)step, st);
            mlp_refresh_bf16(m, st);
            if (b == steps_per_epoch - 1) {
                PTS_CUDA_TRY(cudaMemcpyAsync(hloss.data(), m.loss.ptr, sizeof(float) * batch, cudaMemcpyDeviceToHost, st));
                PTS_CUDA_TRY(cudaStreamSynchronize(st));
                for (int i = 0; i < batch; ++i) esum += hloss[i];
            }
        }
        if (loss_out) loss_out[e] = esum / batch;  // loss of the epoch's last batch
    }
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    PTS_TRY(read_status(idx, st));
    PTS_TRY(mlp_pack_infer(pr.mlp, pr.infer, st));
    pr.ready = 1;
    return PTS_OK;
}

pts_status pts_kmeans(const float *points, int n, int d, int k, const double *u, int iters, float *centroids_out,
                      int32_t *assign_out, int *iters_out, void *stream) {
    if (!points || !u || !centroids_out || !assign_out) return set_error(PTS_ERR_INVALID_ARG, "pts_kmeans: null pointer");
    cudaStream_t st = as_stream(stream);
    DevBuf<float> cost;
    DevBuf<int> counts, off, members;
    PTS_TRY(cost.ensure(n, "kmeans cost"));
    PTS_TRY(counts.ensure(k, "kmeans counts"));
    PTS_TRY(off.ensure(k + 1, "kmeans offsets"));
    PTS_TRY(members.ensure(n, "kmeans members"));
    return kmeans_device(points, n, d, k, u, iters > 0 ? iters : 25, centroids_out, assign_out, cost.ptr, counts.ptr,
                         off.ptr, members.ptr, iters_out, st);
}

pts_status pts_mlp_grad(int C, const float *params, const float *X, const int32_t *labels, int B, float *grads_out,
                        double *loss_out, void *stream) {
    if (!params || !X || !labels || !grads_out || !loss_out) return set_error(PTS_ERR_INVALID_ARG, "pts_mlp_grad: null pointer");
    if (C < 1 || C > 1024 || B < 8 || B % 8) return set_error(PTS_ERR_INVALID_ARG, "pts_mlp_grad: bad sizes");
    cudaStream_t st = as_stream(stream);
    MlpState m;
    PTS_TRY(m.ensure(C, B, st));
    DevBuf<int> status;
    PTS_TRY(status.ensure(1, "status"));
    PTS_CUDA_TRY(cudaMemsetAsync(status.ptr, 0, sizeof(int), st));
    const long np = mlp_param_count(C);
    PTS_CUDA_TRY(cudaMemcpyAsync(m.params.ptr, params, sizeof(float) * np, cudaMemcpyDeviceToDevice, st));
    mlp_refresh_bf16(m, st);
    mlp_gather(m, X, 64, 64, nullptr, 0, B, labels, st);
    mlp_forward(m, B, 1, status.ptr, st);
    mlp_backward(m, B, m.labels.ptr, status.ptr, st);
    PTS_CUDA_TRY(cudaMemcpyAsync(grads_out, m.grads.ptr, sizeof(float) * np, cudaMemcpyDeviceToDevice, st));
    std::vector<float> hl(B);
    PTS_CUDA_TRY(cudaMemcpyAsync(hl.data(), m.loss.ptr, sizeof(float) * B, cudaMemcpyDeviceToHost, st));
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    double s = 0.0;
    for (int i = 0; i < B; ++i) s += hl[i];
    *loss_out = s / B;
    int h = 0;
    PTS_CUDA_TRY(cudaMemcpy(&h, status.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) return set_error(PTS_ERR_TIMEOUT, "pts_mlp_grad: a completion wait gave up");
    return PTS_OK;
}

pts_status pts_gemm_selftest(int M, int N, int K, double *max_rel_err) {
    if (!max_rel_err) return set_error(PTS_ERR_INVALID_ARG, "pts_gemm_selftest: null pointer");
    return gemm_selftest(M, N, K, max_rel_err);
}

pts_status pts_tc_selftest(int N, int K, int f16, double *max_abs_err, double *max_abs_ref) {
    if (!max_abs_err || !max_abs_ref) return set_error(PTS_ERR_INVALID_ARG, "pts_tc_selftest: null pointer");
    return tc_selftest(N, K, f16, max_abs_err, max_abs_ref);
}

pts_status pts_downsample2(const float *in, int H, int W, float *out, void *stream) {
    if (!in || !out || H < 1 || W < 1) return set_error(PTS_ERR_INVALID_ARG, "pts_downsample2");
    launch_downsample2(in, H, W, out, as_stream(stream));
    PTS_CUDA_TRY(cudaGetLastError());
    return PTS_OK;
}

pts_status pts_upsample2(const float *in, int H, int W, float *out, void *stream) {
    if (!in || !out || H < 1 || W < 1) return set_error(PTS_ERR_INVALID_ARG, "pts_upsample2");
    launch_upsample2(in, H, W, out, as_stream(stream));
    PTS_CUDA_TRY(cudaGetLastError());
    return PTS_OK;
}

}  // extern "C"
