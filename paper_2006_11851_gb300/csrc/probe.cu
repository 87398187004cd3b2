// probe.cu -- the learned-proposal search phase (E-step).  The network ranks the k-means
// clusters for each query; the query is compared with the members of its 4 best-ranked
// clusters only (the FP16 tensor-core search restricted to the tiles of each cluster, with the
// exemplar windows stored in cluster order: launch_ivf_probe in search_tc.cu), and the 32
// smallest PCA-space bounds are re-ranked in full dimension.  A query whose re-ranked distance
// exceeds 1.2 x the median nearest-neighbour distance of its chosen window's cluster goes to
// the FP16 search over every window instead (the fallback).
//
//   k_top4     one warp per query: each lane keeps the 4 largest logits of its stripe, then
//              4 rounds of warp arg-max (largest logit, smallest cluster id on ties).
//   k_fallback lists the queries whose result fails the median test.
#include "pts_internal.cuh"

namespace pts {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__global__ void __launch_bounds__(256) k_top4(const float *__restrict__ logits, int Q, int C, int *__restrict__ top) {
    const int lane = threadIdx.x & 31;
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    const float *z = logits + (size_t)q * C;
    float v[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
    int id[4] = {0x7fffffff, 0x7fffffff, 0x7fffffff, 0x7fffffff};
    for (int c = lane; c < C; c += 32) {
        const float x = z[c];
        // insert (x, c) into the descending (value, ascending id) list of 4
        if (x > v[3]) {
            v[3] = x;
            id[3] = c;
#pragma unroll
            for (int k = 3; k > 0; --k)
                if (v[k] > v[k - 1]) {
                    const float tv = v[k];
                    v[k] = v[k - 1];
                    v[k - 1] = tv;
                    const int ti = id[k];
                    id[k] = id[k - 1];
                    id[k - 1] = ti;
                }
        }
    }
    int head = 0;  // next unused entry of this lane's list
    for (int r = 0; r < 4; ++r) {
        float bv = -INFINITY;
        int bi = 0x7fffffff;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k == head) {
                bv = v[k];
                bi = id[k];
            }
        float wv = bv;
        int wi = bi;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(kFull, wv, o);
            const int oi = __shfl_xor_sync(kFull, wi, o);
            if (ov > wv || (ov == wv && oi < wi)) {
                wv = ov;
                wi = oi;
            }
        }
        if (bi == wi) ++head;
        if (lane == 0) top[(size_t)q * 4 + r] = wi < C ? wi : 0;
    }
}

__global__ void k_fallback(const int *__restrict__ nn, const float *__restrict__ d2, int Q,
                           const int *__restrict__ assign, const float *__restrict__ median, float factor, int N,
                           int *__restrict__ list, unsigned int *__restrict__ count) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
        const int n = nn[q];
        const bool bad = n < 0 || n >= N || !(sqrtf(fmaxf(d2[q], 0.0f)) <= factor * median[assign[n]]);
        if (bad) list[atomicAdd(count, 1u)] = q;
    }
}

}  // namespace

void launch_top4(const float *logits, int Q, int C, int *top, cudaStream_t st) {
    count_launches(1);
    k_top4<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(logits, Q, C, top);
}

void launch_fallback(const int *nn, const float *d2, int Q, const int *assign, const float *median, float factor,
                     int N, int *list, unsigned int *count, cudaStream_t st) {
    count_launches(1);
    k_fallback<<<152, 256, 0, st>>>(nn, d2, Q, assign, median, factor, N, list, count);
}

}  // namespace pts
