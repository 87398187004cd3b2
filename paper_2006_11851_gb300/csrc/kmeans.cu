// kmeans.cu -- the flat k-means partition of the exemplar's PCA vectors behind the learned
// proposal (it takes the place of the paper's k-means search tree, section 2.2), and the
// cluster-sorted data the probe reads.
//
//   seeding   k-means++ (Arthur & Vassilvitskii 2007) with caller-supplied uniforms u[i]:
//             center 0 = point floor(u[0] n); center i = the first point (index order) whose
//             running sum of D^2 reaches u[i] * sum D^2 (D^2 in FP64 to the nearest chosen
//             center; points with D^2 = 0 are skipped; floor(u[i] n) if the sum is 0).
//   Lloyd     assignment to the nearest centroid (direct FP32 differences, smallest id on ties);
//             update to the FP64 mean of the members summed in point order; an empty cluster
//             takes the unused point of largest assignment cost (smallest index on ties).
//   CSR       members of each cluster in point order (one CTA per cluster compacts them).
#include <math.h>

#include <vector>

#include "pts_internal.cuh"

namespace pts {
namespace {

__global__ void k_kpp_update(const float *__restrict__ Y, int n, int d, int center, int first,
                             double *__restrict__ D2) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            const double t = (double)Y[(size_t)j * d + k] - (double)Y[(size_t)center * d + k];
            s += t * t;
        }
        D2[j] = first ? s : fmin(D2[j], s);
    }
}

// one CTA of 1024 threads: pick the next center from the running sums of D2
__global__ void __launch_bounds__(1024) k_kpp_select(const double *__restrict__ D2, int n, double u,
                                                     int *__restrict__ out) {
    __shared__ double part[1024];
    __shared__ int best;
    const int t = threadIdx.x;
    const int chunk = (n + 1023) / 1024;
    const int j0 = t * chunk, j1 = min(n, j0 + chunk);
    double s = 0.0;
    for (int j = j0; j < j1; ++j) s += D2[j];
    part[t] = s;
    if (t == 0) best = n;
    __syncthreads();
    // inclusive scan of the thread sums (Hillis-Steele)
    for (int o = 1; o < 1024; o <<= 1) {
        const double v = t >= o ? part[t - o] : 0.0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    const double total = part[1023];
    if (total <= 0.0) {
        if (t == 0) *out = min(n - 1, (int)(u * n));
        return;
    }
    const double target = u * total;
    double run = t > 0 ? part[t - 1] : 0.0;
    for (int j = j0; j < j1; ++j) {
        run += D2[j];
        if (run >= target && D2[j] > 0.0) {
            atomicMin(&best, j);
            break;
        }
    }
    __syncthreads();
    if (t == 0) *out = best < n ? best : n - 1;
}

__global__ void k_gather_rows(const float *__restrict__ Y, int d, const int *__restrict__ idx, int k,
                              float *__restrict__ C) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k * d; i += gridDim.x * blockDim.x)
        C[i] = Y[(size_t)idx[i / d] * d + (i % d)];
}

// nearest centroid; centroids staged through shared memory in chunks of 64
__global__ void __launch_bounds__(256) k_assign(const float *__restrict__ Y, int n, int d,
                                                const float *__restrict__ C, int k, int *__restrict__ assign,
                                                float *__restrict__ cost, int *__restrict__ changed) {
    extern __shared__ float sc[];  // [64][d]
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    float y[kMaxD];
    if (j < n)
        for (int t = 0; t < d; ++t) y[t] = Y[(size_t)j * d + t];
    float best = INFINITY;
    int bi = 0;
    for (int c0 = 0; c0 < k; c0 += 64) {
        const int cn = min(64, k - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < cn * d; i += blockDim.x) sc[i] = C[(size_t)c0 * d + i];
        __syncthreads();
        if (j < n)
            for (int c = 0; c < cn; ++c) {
                float s = 0.0f;
                for (int t = 0; t < d; ++t) {
                    const float e = y[t] - sc[c * d + t];
                    s = fmaf(e, e, s);
                }
                if (s < best) {
                    best = s;
                    bi = c0 + c;
                }
            }
    }
    if (j < n) {
        if (changed && assign[j] != bi) atomicOr(changed, 1);
        assign[j] = bi;
        if (cost) cost[j] = best;
    }
}

__global__ void k_count(const int *__restrict__ assign, int n, int *__restrict__ counts) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        atomicAdd(&counts[assign[j]], 1);
}

// exclusive scan of k counts into offsets[0..k] (one CTA, sequential per thread chunk)
__global__ void __launch_bounds__(1024) k_offsets(const int *__restrict__ counts, int k, int *__restrict__ off) {
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int chunk = (k + 1023) / 1024;
    const int c0 = t * chunk, c1 = min(k, c0 + chunk);
    int s = 0;
    for (int c = c0; c < c1; ++c) s += counts[c];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = t > 0 ? part[t - 1] : 0;
    for (int c = c0; c < c1; ++c) {
        off[c] = run;
        run += counts[c];
    }
    if (t == 1023) off[k] = part[1023];
}

// one CTA per cluster: members in point order, written at off[c]
__global__ void __launch_bounds__(256) k_compact(const int *__restrict__ key, int n, const int *__restrict__ off,
                                                 int *__restrict__ members) {
    const int c = blockIdx.x;
    __shared__ int wsum[8];
    __shared__ int base;
    if (threadIdx.x == 0) base = off[c];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j0 = 0; j0 < n; j0 += 256) {
        const int j = j0 + threadIdx.x;
        const bool mine = j < n && key[j] == c;
        const unsigned b = __ballot_sync(0xffffffffu, mine);
        if (lane == 0) wsum[w] = __popc(b);
        __syncthreads();
        int before = 0;
        for (int i = 0; i < w; ++i) before += wsum[i];
        if (mine) members[base + before + __popc(b & ((1u << lane) - 1u))] = j;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int i = 0; i < 8; ++i) tot += wsum[i];
            base += tot;
        }
        __syncthreads();
    }
}

// centroid = FP64 mean of the members (point order); empty clusters left for k_reseed
__global__ void k_centroids(const float *__restrict__ Y, int d, const int *__restrict__ off,
                            const int *__restrict__ members, float *__restrict__ C) {
    const int c = blockIdx.x, t = threadIdx.x;
    const int a = off[c], b = off[c + 1];
    if (t >= d || b == a) return;
    double s = 0.0;
    for (int i = a; i < b; ++i) s += (double)Y[(size_t)members[i] * d + t];
    C[(size_t)c * d + t] = (float)(s / (b - a));
}

// empty clusters in order take the unused point of largest cost (one thread)
__global__ void k_reseed(const float *__restrict__ Y, int n, int d, const int *__restrict__ counts, int k,
                         const float *__restrict__ cost, unsigned char *__restrict__ used, float *__restrict__ C) {
    if (blockIdx.x || threadIdx.x) return;
    for (int j = 0; j < n; ++j) used[j] = 0;
    for (int c = 0; c < k; ++c) {
        if (counts[c] > 0) continue;
        int far = -1;
        for (int j = 0; j < n; ++j)
            if (!used[j] && (far < 0 || cost[j] > cost[far])) far = j;
        if (far < 0) continue;
        used[far] = 1;
        for (int t = 0; t < d; ++t) C[(size_t)c * d + t] = Y[(size_t)far * d + t];
    }
}

// exemplar PCA coordinates [N][d] from the tiled search vectors (-2 y)
__global__ void k_extract_y(const float *__restrict__ et, int N, int da, int d, float *__restrict__ Y) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (long)N * d; i += (long)gridDim.x * blockDim.x) {
        const int n = (int)(i / d), k = (int)(i % d);
        Y[i] = -0.5f * et[((size_t)(n / kBN) * da + k) * kBN + (n % kBN)];
    }
}

// member search vectors in cluster order, row-major [N][da], and their norms
__global__ void k_pair_labels(const int *__restrict__ nn, const float *__restrict__ d2, int n,
                              const int *__restrict__ assign, int N, int *__restrict__ lab, float *__restrict__ dist) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int m = nn[i];
        lab[i] = (m >= 0 && m < N) ? assign[m] : 0;
        dist[i] = sqrtf(fmaxf(d2[i], 0.0f));
    }
}

// median of each bucket (values gathered in pair order): sort up to kMedCap values of the
// bucket (every ceil(count / kMedCap)-th one when larger) in shared memory
constexpr int kMedCap = 8192;
__global__ void __launch_bounds__(1024) k_bucket_median(const float *__restrict__ vals, const int *__restrict__ off,
                                                        const int *__restrict__ members, int min_count,
                                                        float fallback, float *__restrict__ med) {
    __shared__ float s[kMedCap];
    const int c = blockIdx.x;
    const int a = off[c], b = off[c + 1];
    const int cnt = b - a;
    if (cnt < min_count) {
        if (threadIdx.x == 0) med[c] = fallback;
        return;
    }
    const int step = (cnt + kMedCap - 1) / kMedCap;
    const int m = (cnt + step - 1) / step;
    int p2 = 1;
    while (p2 < m) p2 <<= 1;
    for (int i = threadIdx.x; i < p2; i += blockDim.x) s[i] = i < m ? vals[members[a + i * step]] : INFINITY;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    if ((s[i] > s[l]) == up) {
                        const float t = s[i];
                        s[i] = s[l];
                        s[l] = t;
                    }
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) med[c] = (m & 1) ? s[m / 2] : 0.5f * (s[m / 2 - 1] + s[m / 2]);
}

}  // namespace

pts_status kmeans_device(const float *Y, int n, int d, int k, const double *u, int iters, float *C, int *assign,
                         float *cost, int *counts, int *off, int *members, int *iters_used, cudaStream_t st) {
    if (n < k || k < 1 || d < 1 || d > kMaxD) return set_error(PTS_ERR_INVALID_ARG, "kmeans: need 1 <= k <= n, d <= 64");
    DevBuf<double> D2;
    DevBuf<int> idx, changed;
    DevBuf<unsigned char> used;
    PTS_TRY(D2.ensure(n, "kmeans D2"));
    PTS_TRY(idx.ensure(k, "kmeans seeds"));
    PTS_TRY(changed.ensure(1, "kmeans flag"));
    PTS_TRY(used.ensure(n, "kmeans used"));
    // seeding: the first center, then one selection per further center
    const int first = std::min(n - 1, (int)(u[0] * n));
    PTS_CUDA_TRY(cudaMemcpyAsync(idx.ptr, &first, sizeof(int), cudaMemcpyHostToDevice, st));
    count_launches(1);
    k_kpp_update<<<152 * 2, 256, 0, st>>>(Y, n, d, first, 1, D2.ptr);
    std::vector<int> hidx(k);
    hidx[0] = first;
    for (int i = 1; i < k; ++i) {
        count_launches(2);
        k_kpp_select<<<1, 1024, 0, st>>>(D2.ptr, n, u[i], idx.ptr + i);
        PTS_CUDA_TRY(cudaMemcpyAsync(&hidx[i], idx.ptr + i, sizeof(int), cudaMemcpyDeviceToHost, st));
        PTS_CUDA_TRY(cudaStreamSynchronize(st));
        k_kpp_update<<<152 * 2, 256, 0, st>>>(Y, n, d, hidx[i], 0, D2.ptr);
    }
    count_launches(1);
    k_gather_rows<<<64, 256, 0, st>>>(Y, d, idx.ptr, k, C);
    const size_t smem = sizeof(float) * 64 * d;
    int it = 0;
    for (it = 0; it < iters; ++it) {
        PTS_CUDA_TRY(cudaMemsetAsync(changed.ptr, 0, sizeof(int), st));
        count_launches(1);
        k_assign<<<ceil_div(n, 256), 256, smem, st>>>(Y, n, d, C, k, assign, cost, it > 0 ? changed.ptr : nullptr);
        int h = 1;
        if (it > 0) {
            PTS_CUDA_TRY(cudaMemcpyAsync(&h, changed.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
            PTS_CUDA_TRY(cudaStreamSynchronize(st));
        }
        if (!h) break;
        PTS_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * k, st));
        count_launches(5);
        k_count<<<152, 256, 0, st>>>(assign, n, counts);
        k_offsets<<<1, 1024, 0, st>>>(counts, k, off);
        k_compact<<<k, 256, 0, st>>>(assign, n, off, members);
        k_centroids<<<k, 64, 0, st>>>(Y, d, off, members, C);
        k_reseed<<<1, 1, 0, st>>>(Y, n, d, counts, k, cost, used.ptr, C);
    }
    // final assignment and CSR for the centroids returned
    count_launches(5);
    k_assign<<<ceil_div(n, 256), 256, smem, st>>>(Y, n, d, C, k, assign, cost, nullptr);
    PTS_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * k, st));
    k_count<<<152, 256, 0, st>>>(assign, n, counts);
    k_offsets<<<1, 1024, 0, st>>>(counts, k, off);
    k_compact<<<k, 256, 0, st>>>(assign, n, off, members);
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    PTS_CUDA_TRY(cudaGetLastError());
    if (iters_used) *iters_used = it;
    return PTS_OK;
}

void launch_extract_y(const float *et, int N, int da, int d, float *Y, cudaStream_t st) {
    count_launches(1);
    k_extract_y<<<152 * 4, 256, 0, st>>>(et, N, da, d, Y);
}

pts_status cluster_medians(const int *nn, const float *d2, int n, const int *assign, int N, int C, int *lab,
                           float *dist, float *median, cudaStream_t st) {
    DevBuf<int> counts, off, members;
    PTS_TRY(counts.ensure(C, "median counts"));
    PTS_TRY(off.ensure(C + 1, "median offsets"));
    PTS_TRY(members.ensure(n, "median buckets"));
    count_launches(1);
    k_pair_labels<<<152 * 4, 256, 0, st>>>(nn, d2, n, assign, N, lab, dist);
    // the global median (one bucket with every pair) is the fallback of sparse clusters
    DevBuf<int> zero, goff, gmem;
    PTS_TRY(zero.ensure(n, "median all"));
    PTS_TRY(goff.ensure(2, "median all offsets"));
    PTS_TRY(gmem.ensure(n, "median all members"));
    PTS_CUDA_TRY(cudaMemsetAsync(zero.ptr, 0, sizeof(int) * n, st));
    DevBuf<int> one;
    PTS_TRY(one.ensure(1, "median one"));
    PTS_CUDA_TRY(cudaMemsetAsync(one.ptr, 0, sizeof(int), st));
    count_launches(6);
    k_count<<<152, 256, 0, st>>>(zero.ptr, n, one.ptr);
    k_offsets<<<1, 1024, 0, st>>>(one.ptr, 1, goff.ptr);
    k_compact<<<1, 256, 0, st>>>(zero.ptr, n, goff.ptr, gmem.ptr);
    DevBuf<float> gmed;
    PTS_TRY(gmed.ensure(1, "median global"));
    k_bucket_median<<<1, 1024, 0, st>>>(dist, goff.ptr, gmem.ptr, 1, 0.0f, gmed.ptr);
    float hg = 0.0f;
    PTS_CUDA_TRY(cudaMemcpyAsync(&hg, gmed.ptr, sizeof(float), cudaMemcpyDeviceToHost, st));
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    PTS_CUDA_TRY(cudaMemsetAsync(counts.ptr, 0, sizeof(int) * C, st));
    k_count<<<152, 256, 0, st>>>(lab, n, counts.ptr);
    k_offsets<<<1, 1024, 0, st>>>(counts.ptr, C, off.ptr);
    count_launches(2);
    k_compact<<<C, 256, 0, st>>>(lab, n, off.ptr, members.ptr);
    k_bucket_median<<<C, 1024, 0, st>>>(dist, off.ptr, members.ptr, 5, hg, median);
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    return PTS_OK;
}

}  // namespace pts
