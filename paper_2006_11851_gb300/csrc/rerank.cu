// rerank.cu -- exact full-dimension distances of Eq. 4 for candidate lists.
//
// k_rerank       one warp per query (all queries, or those of a device-side
//                list): evaluates the query's candidates in increasing order of
//                their bound and keeps the lexicographically smallest (d2, n).
//                With certify != 0 it stops at the first candidate whose bound
//                minus the slack tau_q exceeds the best distance found (no later
//                candidate can win).  With certify == 1
//                (exact mode) the result is final when d2_best <= B_32 - tau_q:
//                every window outside the list has a bound >= B_32, hence a
//                distance >= d2_best.  Otherwise the query joins the fail list
//                with its best so far packed into best64.
// k_brute        direct scan of every exemplar window for each listed query
//                (one CTA per query); used for what no pass could certify.
// k_resolve      writes nn/d2 of listed queries from the packed minima.
//
// Distances are sums of squared FP32 differences read straight from the two
// images (a window row is C w contiguous floats in HWC layout, C channels), reduced across
// the warp by a fixed butterfly, so the result is deterministic.  Windows of 8, 16 and 32
// pixels go through k_rerank_px, which reads the exemplar's RGBA copy (one 16-byte load per
// pixel); its per-lane order of terms differs from k_rerank's, so the last bits of a distance
// depend on the window width's kernel, never on the mode or the run.
#include <algorithm>

#include "pts_internal.cuh"

namespace pts {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Full-dimension squared distance between the query window at (y0, x0) of X
// and exemplar window n, one warp, lanes striding over each window row.
__device__ __forceinline__ float window_dist2(const RerankArgs &a, int y0, int x0, int n, int lane) {
    const int ey = n / a.ex, ex0 = n - ey * a.ex;
    const int row = a.C * a.w;
    const float *xq = a.X + ((size_t)y0 * a.Wo + x0) * a.C;
    const float *zn = a.Z + ((size_t)ey * a.We + ex0) * a.C;
    float s = 0.0f;
    for (int dy = 0; dy < a.w; ++dy) {
        const float *xr = xq + (size_t)dy * a.Wo * a.C;
        const float *zr = zn + (size_t)dy * a.We * a.C;
        for (int e = lane; e < row; e += 32) {
            const float t = __ldg(xr + e) - __ldg(zr + e);
            s = fmaf(t, t, s);
        }
    }
    return warp_sum(s);
}

__global__ void __launch_bounds__(256) k_rerank(RerankArgs a, const int *__restrict__ qlist,
                                                const unsigned int *__restrict__ qcount,
                                                const int *__restrict__ cand_idx,
                                                const float *__restrict__ cand_lb,
                                                const float *__restrict__ tau, int certify,
                                                int *__restrict__ nn_out, float *__restrict__ d2_out,
                                                int *__restrict__ fail_list,
                                                unsigned int *__restrict__ fail_count,
                                                unsigned long long *__restrict__ best64,
                                                int *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int q = wid;
    if (qlist) {
        if (wid >= (int)*qcount) return;
        q = qlist[wid];
    }
    if (q < 0 || q >= a.Q) return;
    const int y0 = (q / a.qx) * a.stride, x0 = (q % a.qx) * a.stride;
    const int my_idx = cand_idx[(size_t)q * kTopK + lane];
    const float my_lb = cand_lb[(size_t)q * kTopK + lane];
    const float tq = certify ? tau[q] : 0.0f;
    float best = INFINITY;
    int best_n = -1;
    for (int i = 0; i < kTopK; ++i) {
        const int n = __shfl_sync(kFull, my_idx, i);
        const float lb = __shfl_sync(kFull, my_lb, i);
        if (n < 0) break;  // fewer than 32 windows exist
        if (n >= a.N) {
            if (lane == 0) atomicOr(status, kDevErrBounds);
            continue;
        }
        if (certify && lb - tq > best) break;  // bounds are ascending
        const float d = window_dist2(a, y0, x0, n, lane);
        if (d < best || (d == best && n < best_n)) {
            best = d;
            best_n = n;
        }
    }
    const int last_idx = __shfl_sync(kFull, my_idx, kTopK - 1);
    const float last_lb = __shfl_sync(kFull, my_lb, kTopK - 1);
    const bool done = certify != 1 || last_idx < 0 || best <= last_lb - tq;
    if (lane == 0) {
        if (done) {
            nn_out[q] = best_n;
            d2_out[q] = best;
        } else {
            const unsigned int slot = atomicAdd(fail_count, 1u);
            fail_list[slot] = q;
            best64[q] = pack_dist_idx(best, best_n);
        }
    }
}

// k_rerank for a window width known at compile time: the query window is loaded into registers
// once, and each candidate's rows are fully unrolled, two candidates at a time, so their loads are
// in flight together.  Per lane the terms are summed in the order of window_dist2 (row by row,
// element lane + 32p within a row) and reduced by the same butterfly: the distances are bitwise
// those of k_rerank.  Evaluating the second candidate of a pair that k_rerank would have skipped
// cannot change the minimum (its distance exceeds the best so far).
template <int W, int CH>
__global__ void __launch_bounds__(256) k_rerank_w(RerankArgs a, const int *__restrict__ qlist,
                                                  const unsigned int *__restrict__ qcount,
                                                  const int *__restrict__ cand_idx,
                                                  const float *__restrict__ cand_lb,
                                                  const float *__restrict__ tau, int certify,
                                                  int *__restrict__ nn_out, float *__restrict__ d2_out,
                                                  int *__restrict__ fail_list,
                                                  unsigned int *__restrict__ fail_count,
                                                  unsigned long long *__restrict__ best64,
                                                  int *__restrict__ status) {
    constexpr int R = CH * W, PER = (R + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int q = wid;
    if (qlist) {
        if (wid >= (int)*qcount) return;
        q = qlist[wid];
    }
    if (q < 0 || q >= a.Q) return;
    const int y0 = (q / a.qx) * a.stride, x0 = (q % a.qx) * a.stride;
    const float *xq = a.X + ((size_t)y0 * a.Wo + x0) * CH;
    float xv[W][PER];
#pragma unroll
    for (int dy = 0; dy < W; ++dy)
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int e = lane + 32 * p;
            xv[dy][p] = e < R ? __ldg(xq + (size_t)dy * a.Wo * CH + e) : 0.0f;
        }
    const int my_idx = cand_idx[(size_t)q * kTopK + lane];
    const float my_lb = cand_lb[(size_t)q * kTopK + lane];
    const float tq = certify ? tau[q] : 0.0f;
    float best = INFINITY;
    int best_n = -1;
    const size_t zrow = (size_t)a.We * CH;
    for (int i = 0; i < kTopK; i += 2) {
        int n0 = __shfl_sync(kFull, my_idx, i);
        int n1 = __shfl_sync(kFull, my_idx, i + 1);
        const float lb0 = __shfl_sync(kFull, my_lb, i);
        if (n0 < 0) break;  // fewer than 32 windows exist
        if (certify && lb0 - tq > best) break;  // bounds are ascending
        if (n0 >= a.N) {
            if (lane == 0) atomicOr(status, kDevErrBounds);
            n0 = -1;
        }
        if (n1 >= a.N) {
            if (lane == 0) atomicOr(status, kDevErrBounds);
            n1 = -1;
        }
        const int m0 = n0 < 0 ? 0 : n0, m1 = n1 < 0 ? 0 : n1;
        const int ey0 = m0 / a.ex, ey1 = m1 / a.ex;
        const float *z0 = a.Z + ((size_t)ey0 * a.We + (m0 - ey0 * a.ex)) * CH;
        const float *z1 = a.Z + ((size_t)ey1 * a.We + (m1 - ey1 * a.ex)) * CH;
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int dy = 0; dy < W; ++dy)
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                const int e = lane + 32 * p;
                if (e < R) {
                    const float t0 = xv[dy][p] - __ldg(z0 + dy * zrow + e);
                    const float t1 = xv[dy][p] - __ldg(z1 + dy * zrow + e);
                    s0 = fmaf(t0, t0, s0);
                    s1 = fmaf(t1, t1, s1);
                }
            }
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        if (n0 >= 0 && (s0 < best || (s0 == best && n0 < best_n))) {
            best = s0;
            best_n = n0;
        }
        if (n1 >= 0 && (s1 < best || (s1 == best && n1 < best_n))) {
            best = s1;
            best_n = n1;
        }
    }
    const int last_idx = __shfl_sync(kFull, my_idx, kTopK - 1);
    const float last_lb = __shfl_sync(kFull, my_lb, kTopK - 1);
    const bool done = certify != 1 || last_idx < 0 || best <= last_lb - tq;
    if (lane == 0) {
        if (done) {
            nn_out[q] = best_n;
            d2_out[q] = best;
        } else {
            const unsigned int slot = atomicAdd(fail_count, 1u);
            fail_list[slot] = q;
            best64[q] = pack_dist_idx(best, best_n);
        }
    }
}

// k_rerank for windows of W x W pixels (W * W a multiple of 32) with the exemplar read as one
// 16-byte (r, g, b, s-or-0) load per pixel: lane l holds query pixels l, l + 32, ..., and sums
// its pixels' channel terms in that order before the butterfly, so each candidate costs a lane
// W * W / 32 vector loads.  P candidates are evaluated together; those beyond the first of a
// group that k_rerank would have skipped have distances above the best so far and change
// nothing.  The distances are deterministic FP32 sums (a different order from k_rerank's).
template <int W, int CH, int P>
__global__ void __launch_bounds__(256) k_rerank_px(RerankArgs a, const int *__restrict__ qlist,
                                                   const unsigned int *__restrict__ qcount,
                                                   const int *__restrict__ cand_idx,
                                                   const float *__restrict__ cand_lb,
                                                   const float *__restrict__ tau, int certify,
                                                   int *__restrict__ nn_out, float *__restrict__ d2_out,
                                                   int *__restrict__ fail_list,
                                                   unsigned int *__restrict__ fail_count,
                                                   unsigned long long *__restrict__ best64,
                                                   int *__restrict__ status) {
    static_assert((W * W) % 32 == 0 && (CH == 3 || CH == 4), "pixel-parallel re-rank shape");
    constexpr int PX = W * W / 32;
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int q = wid;
    if (qlist) {
        if (wid >= (int)*qcount) return;
        q = qlist[wid];
    }
    if (q < 0 || q >= a.Q) return;
    const int y0 = (q / a.qx) * a.stride, x0 = (q % a.qx) * a.stride;
    float xq[PX][CH];
#pragma unroll
    for (int j = 0; j < PX; ++j) {
        const int p = lane + 32 * j, dy = p / W, dx = p % W;
        const float *src = a.X + ((size_t)(y0 + dy) * a.Wo + x0 + dx) * CH;
#pragma unroll
        for (int c = 0; c < CH; ++c) xq[j][c] = __ldg(src + c);
    }
    const int my_idx = cand_idx[(size_t)q * kTopK + lane];
    const float my_lb = cand_lb[(size_t)q * kTopK + lane];
    const float tq = certify ? tau[q] : 0.0f;
    float best = INFINITY;
    int best_n = -1;
    for (int i = 0; i < kTopK; i += P) {
        int n[P];
#pragma unroll
        for (int c = 0; c < P; ++c) n[c] = __shfl_sync(kFull, my_idx, i + c);
        const float lb0 = __shfl_sync(kFull, my_lb, i);
        if (n[0] < 0) break;  // fewer than 32 windows exist
        if (certify && lb0 - tq > best) break;  // bounds are ascending
        const float4 *z[P];
#pragma unroll
        for (int c = 0; c < P; ++c) {
            if (n[c] >= a.N) {
                if (lane == 0) atomicOr(status, kDevErrBounds);
                n[c] = -1;
            }
            const int m = n[c] < 0 ? 0 : n[c], ey = m / a.ex;
            z[c] = a.Z4 + (size_t)ey * a.We + (m - ey * a.ex);
        }
        float s[P];
#pragma unroll
        for (int c = 0; c < P; ++c) s[c] = 0.0f;
#pragma unroll
        for (int j = 0; j < PX; ++j) {
            const int p = lane + 32 * j, off = (p / W) * a.We + p % W;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const float4 e = __ldg(z[c] + off);
                float t = xq[j][0] - e.x;
                s[c] = fmaf(t, t, s[c]);
                t = xq[j][1] - e.y;
                s[c] = fmaf(t, t, s[c]);
                t = xq[j][2] - e.z;
                s[c] = fmaf(t, t, s[c]);
                if constexpr (CH == 4) {
                    t = xq[j][CH - 1] - e.w;
                    s[c] = fmaf(t, t, s[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < P; ++c) {
            const float d = warp_sum(s[c]);
            if (n[c] >= 0 && (d < best || (d == best && n[c] < best_n))) {
                best = d;
                best_n = n[c];
            }
        }
    }
    const int last_idx = __shfl_sync(kFull, my_idx, kTopK - 1);
    const float last_lb = __shfl_sync(kFull, my_lb, kTopK - 1);
    const bool done = certify != 1 || last_idx < 0 || best <= last_lb - tq;
    if (lane == 0) {
        if (done) {
            nn_out[q] = best_n;
            d2_out[q] = best;
        } else {
            const unsigned int slot = atomicAdd(fail_count, 1u);
            fail_list[slot] = q;
            best64[q] = pack_dist_idx(best, best_n);
        }
    }
}

// One CTA per listed query; each thread scores whole windows.
__global__ void __launch_bounds__(256) k_brute(RerankArgs a, const int *__restrict__ fail_list,
                                               const unsigned int *__restrict__ fail_count,
                                               unsigned int *__restrict__ brute_count,
                                               unsigned long long *__restrict__ best64,
                                               int *__restrict__ status) {
    const unsigned int nf = *fail_count;
    __shared__ unsigned long long red[256];
    for (unsigned int f = blockIdx.x; f < nf; f += gridDim.x) {
        const int q = fail_list[f];
        if (q < 0 || q >= a.Q) {
            if (threadIdx.x == 0) atomicOr(status, kDevErrBounds);
            continue;
        }
        if (threadIdx.x == 0) atomicAdd(brute_count, 1u);
        const int y0 = (q / a.qx) * a.stride, x0 = (q % a.qx) * a.stride;
        unsigned long long mine = ~0ull;
        for (int n = threadIdx.x; n < a.N; n += blockDim.x) {
            const int ey = n / a.ex, ex0 = n - ey * a.ex;
            float s = 0.0f;
            for (int dy = 0; dy < a.w; ++dy) {
                const float *xr = a.X + ((size_t)(y0 + dy) * a.Wo + x0) * a.C;
                const float *zr = a.Z + ((size_t)(ey + dy) * a.We + ex0) * a.C;
                for (int e = 0; e < a.C * a.w; ++e) {
                    const float t = __ldg(xr + e) - __ldg(zr + e);
                    s = fmaf(t, t, s);
                }
            }
            const unsigned long long pk = pack_dist_idx(s, n);
            mine = pk < mine ? pk : mine;
        }
        red[threadIdx.x] = mine;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                const unsigned long long other = red[threadIdx.x + o];
                if (other < red[threadIdx.x]) red[threadIdx.x] = other;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) best64[q] = red[0];
        __syncthreads();
    }
}

__global__ void k_resolve(const int *__restrict__ fail_list,
                          const unsigned int *__restrict__ fail_count,
                          const unsigned long long *__restrict__ best64, int Q,
                          int *__restrict__ nn_out, float *__restrict__ d2_out) {
    const unsigned int nf = *fail_count;
    for (unsigned int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf;
         f += gridDim.x * blockDim.x) {
        const int q = fail_list[f];
        if (q < 0 || q >= Q) continue;
        const unsigned long long pk = best64[q];
        nn_out[q] = static_cast<int>(pk & 0xffffffffu);
        d2_out[q] = __uint_as_float(static_cast<unsigned int>(pk >> 32));
    }
}

__global__ void k_list_all(int *__restrict__ list, unsigned int *__restrict__ count, int Q) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) list[q] = q;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = (unsigned int)Q;
}

}  // namespace

void launch_list_all(int *list, unsigned int *count, int Q, cudaStream_t st) {
    count_launches(1);
    k_list_all<<<std::max(1, std::min(152 * 4, ceil_div(Q, 256))), 256, 0, st>>>(list, count, Q);
}

void launch_rerank(const RerankArgs &a, const int *qlist, const unsigned int *qcount,
                   const int *cand_idx, const float *cand_lb, const float *tau, int certify,
                   int *nn_out, float *d2_out, int *fail_list, unsigned int *fail_count,
                   unsigned long long *best64, int *status, cudaStream_t st) {
    if (a.Q == 0) return;
    const int grid = ceil_div((long)a.Q * 32, 256);
    ProfScope ps(kProfRerank, st, 1);
#define PTS_RERANK_ARGS a, qlist, qcount, cand_idx, cand_lb, tau, certify, nn_out, d2_out, fail_list, fail_count, \
                        best64, status
    switch (a.C * 64 + a.w) {
        case 3 * 64 + 4: k_rerank_w<4, 3><<<grid, 256, 0, st>>>(PTS_RERANK_ARGS); break;
        case 3 * 64 + 8: k_rerank_px<8, 3, 4><<<grid, 256, 0, st>>>(PTS_RERANK_ARGS); break;
        case 3 * 64 + 16: k_rerank_px<16, 3, 2><<<grid, 256, 0, st>>>(PTS_RERANK_ARGS); break;
        case 3 * 64 + 32: k_rerank_px<32, 3, 2><<<grid, 256, 0, st>>>(PTS_RERANK_ARGS); break;
        case 4 * 64 + 4: k_rerank_w<4, 4><<<grid, 256, 0, st>>>(PTS_RERANK_ARGS); break;
        case 4 * 64 + 8: k_rerank_px<8, 4, 4><<<grid, 256, 0, st>>>(PTS_RERANK_ARGS); break;
        case 4 * 64 + 16: k_rerank_px<16, 4, 2><<<grid, 256, 0, st>>>(PTS_RERANK_ARGS); break;
        default: k_rerank<<<grid, 256, 0, st>>>(PTS_RERANK_ARGS); break;
    }
#undef PTS_RERANK_ARGS
}

void launch_brute_fallback(const RerankArgs &a, const int *fail_list,
                           const unsigned int *fail_count, unsigned int *brute_count,
                           unsigned long long *best64, int *status, cudaStream_t st) {
    ProfScope ps(kProfBrute, st, 1);
    k_brute<<<152 * 2, 256, 0, st>>>(a, fail_list, fail_count, brute_count, best64, status);
}

void launch_resolve(const int *fail_list, const unsigned int *fail_count,
                    const unsigned long long *best64, int Q, int *nn_out, float *d2_out,
                    cudaStream_t st) {
    count_launches(1);
    k_resolve<<<152, 256, 0, st>>>(fail_list, fail_count, best64, Q, nn_out, d2_out);
}

}  // namespace pts
