// kmtree.cu -- the paper's own search structure (section 2.2), kept as a baseline beside the
// learned proposal: a hierarchical k-means tree over the exemplar windows' PCA coordinates with
// k = 4, each node split recursively until it holds fewer than k windows, searched by greedy
// descent (the nearest of a node's 4 centroids, down to a leaf) and an exact re-rank of the
// leaf's windows.
//
// Build, level by level: one CTA per node to split.  It seeds the 4 centroids with the node's
// windows at 1/8, 3/8, 5/8 and 7/8 of its range, runs a fixed number of Lloyd iterations
// (assignment to the nearest centroid, the smaller index on ties; the update sums in window order,
// so the tree is deterministic; an emptied cluster keeps its centroid), assigns once more to the
// final centroids and partitions the node's range stably by cluster.  The host reads the
// children's sizes and decides, for each child, internal node (>= 4 windows and smaller than its
// parent) or leaf, before the next level.
//
// Layout: internal node i holds cent[i][4][d] and child[i][4]; a child reference c >= 0 is an
// internal node, c <= -2 the leaf -c - 2, -1 no child.  Leaf l covers perm[leaf_begin[l],
// leaf_end[l]).
#include <algorithm>
#include <climits>
#include <vector>

#include "pts_internal.cuh"

namespace pts {
namespace {

constexpr int kTreeK = 4;
constexpr int kTreeThreads = 256;  // >= kTreeK * kMaxD

// window n's coordinate j: the exact search stores -2 y_n window-major
__device__ __forceinline__ float tree_coord(const float *rows, int da, int n, int j) {
    return -0.5f * rows[(size_t)n * da + j];
}

__global__ void __launch_bounds__(kTreeThreads)
    k_tree_split(const int *__restrict__ nodes, const int2 *__restrict__ range, int *__restrict__ perm,
                 int *__restrict__ tmp, unsigned char *__restrict__ label, const float *__restrict__ rows, int da,
                 int d, int iters, float *__restrict__ cent, int2 *__restrict__ child_range) {
    __shared__ float c[kTreeK * kMaxD];
    __shared__ float s[kTreeK * kMaxD];
    __shared__ int cnt[kTreeK];
    const int node = nodes[blockIdx.x];
    const int2 rg = range[blockIdx.x];
    const int b = rg.x, size = rg.y - rg.x;
    const int t = threadIdx.x;
    if (t < kTreeK * d) {
        const int k = t / d, j = t - k * d;
        c[t] = tree_coord(rows, da, perm[b + (int)(((long)size * (2 * k + 1)) / (2 * kTreeK))], j);
    }
    __syncthreads();
    auto assign = [&]() {
        for (int p = t; p < size; p += blockDim.x) {
            const int n = perm[b + p];
            float best = INFINITY;
            int bk = 0;
            for (int k = 0; k < kTreeK; ++k) {
                float acc = 0.0f;
                for (int j = 0; j < d; ++j) {
                    const float diff = tree_coord(rows, da, n, j) - c[k * d + j];
                    acc = fmaf(diff, diff, acc);
                }
                if (acc < best) {
                    best = acc;
                    bk = k;
                }
            }
            label[b + p] = (unsigned char)bk;
        }
        __syncthreads();
    };
    for (int it = 0; it < iters; ++it) {
        assign();
        if (t < kTreeK * d) {  // thread (k, j): the coordinate-j sum of cluster k, in window order
            const int k = t / d, j = t - k * d;
            float acc = 0.0f;
            int m = 0;
            for (int p = 0; p < size; ++p)
                if (label[b + p] == k) {
                    acc += tree_coord(rows, da, perm[b + p], j);
                    ++m;
                }
            s[t] = acc;
            if (j == 0) cnt[k] = m;
        }
        __syncthreads();
        if (t < kTreeK * d && cnt[t / d] > 0) c[t] = s[t] / (float)cnt[t / d];
        __syncthreads();
    }
    assign();
    if (t < kTreeK * d) cent[(size_t)node * kTreeK * d + t] = c[t];
    if (t == 0) {  // stable partition of the range by cluster
        int off[kTreeK + 1] = {0, 0, 0, 0, 0};
        for (int p = 0; p < size; ++p) ++off[label[b + p] + 1];
        for (int k = 0; k < kTreeK; ++k) off[k + 1] += off[k];
        for (int k = 0; k < kTreeK; ++k) child_range[(size_t)blockIdx.x * kTreeK + k] = make_int2(b + off[k], b + off[k + 1]);
        int pos[kTreeK] = {off[0], off[1], off[2], off[3]};
        for (int p = 0; p < size; ++p) tmp[b + pos[label[b + p]]++] = perm[b + p];
        for (int p = 0; p < size; ++p) perm[b + p] = tmp[b + p];
    }
}

__global__ void k_iota(int *p, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

// One thread per query: greedy descent from the root (the nearest existing child centroid, the
// smaller index on ties), then the leaf's windows (at most 32) as candidates with bound 0.
__global__ void __launch_bounds__(256)
    k_tree_search(const float *__restrict__ qcoord, int da_q, int Q, int d, const float *__restrict__ cent,
                  const int *__restrict__ child, const int *__restrict__ leaf_begin, const int *__restrict__ leaf_end,
                  const int *__restrict__ perm, int max_depth, int *__restrict__ cand_idx,
                  float *__restrict__ cand_lb, int *__restrict__ leaf_out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    const float *y = qcoord + (size_t)q * da_q;
    int node = 0, leaf = -1;
    for (int depth = 0; depth <= max_depth && leaf < 0; ++depth) {
        float best = INFINITY;
        int bc = -1;
        for (int k = 0; k < kTreeK; ++k) {
            const int ch = child[node * kTreeK + k];
            if (ch == -1) continue;
            const float *ck = cent + ((size_t)node * kTreeK + k) * d;
            float acc = 0.0f;
            for (int j = 0; j < d; ++j) {
                const float diff = y[j] - ck[j];
                acc = fmaf(diff, diff, acc);
            }
            if (acc < best) {
                best = acc;
                bc = ch;
            }
        }
        if (bc >= 0)
            node = bc;
        else
            leaf = bc <= -2 ? -bc - 2 : 0;
    }
    if (leaf < 0) leaf = 0;  // unreachable: every path ends in a leaf within the tree's depth
    const int b = leaf_begin[leaf], e = min(leaf_end[leaf], leaf_begin[leaf] + kTopK);
    for (int i = 0; i < kTopK; ++i) {
        const bool real = b + i < e;
        cand_idx[(size_t)q * kTopK + i] = real ? perm[b + i] : -1;
        cand_lb[(size_t)q * kTopK + i] = real ? 0.0f : INFINITY;
    }
    if (leaf_out) leaf_out[q] = leaf;
}

}  // namespace

pts_status build_kmtree(KmTree &tr, const float *rows, int N, int da, int d, int iters, cudaStream_t st) {
    if (d < 1 || d > kMaxD) return set_error(PTS_ERR_INVALID_ARG, "pts_build_kmeans_tree: index d outside 1..64");
    PTS_TRY(tr.perm.ensure(N, "tree permutation"));
    PTS_TRY(tr.tmp.ensure(N, "tree scratch"));
    PTS_TRY(tr.label.ensure(N, "tree labels"));
    count_launches(1);
    k_iota<<<152 * 4, 256, 0, st>>>(tr.perm.ptr, N);
    std::vector<int> child, leaf_b, leaf_e;
    std::vector<int> level;          // internal nodes to split now
    std::vector<int2> level_range;   // their ranges
    int n_internal = 0;
    if (N >= kTreeK) {
        level.push_back(n_internal++);
        level_range.push_back(make_int2(0, N));
        child.assign(kTreeK, -1);
    } else {  // the whole exemplar is one leaf under a root with one child
        child.assign(kTreeK, -1);
        child[0] = -2;
        leaf_b.push_back(0);
        leaf_e.push_back(N);
        n_internal = 1;
    }
    // internal nodes partition their parent's windows, so there are fewer than N of them
    PTS_TRY(tr.cent.ensure((size_t)std::max(N, 1) * kTreeK * d, "tree centroids"));
    PTS_CUDA_TRY(cudaMemsetAsync(tr.cent.ptr, 0, sizeof(float) * (size_t)std::max(N, 1) * kTreeK * d, st));
    DevBuf<int> d_nodes;
    DevBuf<int2> d_range, d_child_range;
    int depth = 0;
    while (!level.empty()) {
        const int L = (int)level.size();
        PTS_TRY(d_nodes.ensure(L, "tree level"));
        PTS_TRY(d_range.ensure(L, "tree level"));
        PTS_TRY(d_child_range.ensure((size_t)L * kTreeK, "tree level"));
        PTS_CUDA_TRY(cudaMemcpyAsync(d_nodes.ptr, level.data(), sizeof(int) * L, cudaMemcpyHostToDevice, st));
        PTS_CUDA_TRY(cudaMemcpyAsync(d_range.ptr, level_range.data(), sizeof(int2) * L, cudaMemcpyHostToDevice, st));
        count_launches(1);
        k_tree_split<<<L, kTreeThreads, 0, st>>>(d_nodes.ptr, d_range.ptr, tr.perm.ptr, tr.tmp.ptr, tr.label.ptr, rows,
                                                 da, d, iters, tr.cent.ptr, d_child_range.ptr);
        std::vector<int2> cr((size_t)L * kTreeK);
        PTS_CUDA_TRY(cudaMemcpyAsync(cr.data(), d_child_range.ptr, sizeof(int2) * L * kTreeK, cudaMemcpyDeviceToHost,
                                     st));
        PTS_CUDA_TRY(cudaStreamSynchronize(st));
        PTS_CUDA_TRY(cudaGetLastError());
        std::vector<int> next;
        std::vector<int2> next_range;
        for (int i = 0; i < L; ++i) {
            const int parent_size = level_range[i].y - level_range[i].x;
            for (int k = 0; k < kTreeK; ++k) {
                const int2 r = cr[(size_t)i * kTreeK + k];
                const int size = r.y - r.x;
                int ref = -1;
                if (size >= kTreeK && size < parent_size) {
                    ref = n_internal++;
                    child.resize((size_t)n_internal * kTreeK, -1);
                    next.push_back(ref);
                    next_range.push_back(r);
                } else if (size > 0) {
                    ref = -2 - (int)leaf_b.size();
                    leaf_b.push_back(r.x);
                    leaf_e.push_back(r.y);
                }
                child[(size_t)level[i] * kTreeK + k] = ref;
            }
        }
        level.swap(next);
        level_range.swap(next_range);
        ++depth;
    }
    d_nodes.release();
    d_range.release();
    d_child_range.release();
    PTS_TRY(tr.child.ensure(child.size(), "tree children"));
    PTS_TRY(tr.leaf_begin.ensure(std::max<size_t>(leaf_b.size(), 1), "tree leaves"));
    PTS_TRY(tr.leaf_end.ensure(std::max<size_t>(leaf_e.size(), 1), "tree leaves"));
    PTS_CUDA_TRY(cudaMemcpyAsync(tr.child.ptr, child.data(), sizeof(int) * child.size(), cudaMemcpyHostToDevice, st));
    PTS_CUDA_TRY(cudaMemcpyAsync(tr.leaf_begin.ptr, leaf_b.data(), sizeof(int) * leaf_b.size(), cudaMemcpyHostToDevice,
                                 st));
    PTS_CUDA_TRY(cudaMemcpyAsync(tr.leaf_end.ptr, leaf_e.data(), sizeof(int) * leaf_e.size(), cudaMemcpyHostToDevice,
                                 st));
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    tr.n_internal = n_internal;
    tr.n_leaves = (int)leaf_b.size();
    tr.depth = depth;
    tr.d = d;
    tr.N = N;
    tr.ready = 1;
    return PTS_OK;
}

void launch_tree_search(const KmTree &tr, const float *qcoord, int da_q, int Q, int *cand_idx, float *cand_lb,
                        int *leaf_out, cudaStream_t st) {
    if (Q <= 0) return;
    ProfScope ps(kProfProbe, st, 1);
    k_tree_search<<<ceil_div(Q, 256), 256, 0, st>>>(qcoord, da_q, Q, tr.d, tr.cent.ptr, tr.child.ptr,
                                                     tr.leaf_begin.ptr, tr.leaf_end.ptr, tr.perm.ptr, tr.depth,
                                                     cand_idx, cand_lb, leaf_out);
}

}  // namespace pts
