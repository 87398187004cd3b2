// pts_internal.cuh -- shared declarations of the CUDA library (not part of the
// public ABI, which is include/pts.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pts.h"

namespace pts {

// ---------------------------------------------------------------------------
// tile shapes of the FP32 SIMT search (see search_f32.cu)
// ---------------------------------------------------------------------------
constexpr int kBN = 128;   // exemplar windows per tile (32 lanes x 4)
constexpr int kBQ = 64;    // queries per CTA (8 warps x 8 rows)
constexpr int kTcQueryRows = 128;  // queries per tensor-core query tile (the FP16 search's M)
constexpr int kTopK = 32;  // candidates kept per query (one per lane)
constexpr int kMaxAdaptiveParts = 32;    // exemplar parts of an adaptive full-dimension pass
constexpr int kAdaptiveGrid = 2 * 152;   // its CTAs (two per SM), each taking items in turn
constexpr int kPartRows = 1 << 17;       // its part records (of 32 candidates) at most
constexpr int kMaxDA = 68;     // exact search: d <= 64 coordinates + residual, padded to 4
constexpr int kMaxD = 64;      // PCA dimensions of the exact search
constexpr int kMaxDPca = 128;  // PCA dimensions an index may keep (fast modes use up to kMaxDFast)
constexpr int kMaxDFast = 124;  // tensor-core / proposal search: d + residual + 3 norm slots <= 128
constexpr int kMaxDAFast = 128;

// device status word bits (OR-ed by kernels, read at synchronising calls)
constexpr int kDevErrBounds = 1;   // an index read from an input was out of range
constexpr int kDevErrTimeout = 2;  // a bounded wait gave up
constexpr int kDevErrNumeric = 4;  // a factorisation met a non-positive pivot
constexpr int kDevErrCapacity = 8; // a list overflowed (handled, informational)

// ---------------------------------------------------------------------------
// host-side error reporting
// ---------------------------------------------------------------------------
pts_status set_error(pts_status s, const std::string &msg);
pts_status cuda_error(cudaError_t e, const char *where);

#define PTS_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return ::pts::cuda_error(_e, #expr); \
    } while (0)

#define PTS_TRY(expr)                          \
    do {                                       \
        pts_status _s = (expr);                \
        if (_s != PTS_OK) return _s;           \
    } while (0)

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// device memory owned by the library
// ---------------------------------------------------------------------------
// Every library allocation goes through these two: cudaMalloc / cudaFree, or the allocator a
// caller registered with pts_set_allocator (capi.cu).  dev_free synchronises the device before
// it hands memory to a registered allocator, as cudaFree does, so no queued kernel can still
// be reading it when the allocator gives it out again.
pts_status dev_alloc(void **p, size_t bytes, const char *what);
void dev_free(void *p);
// Called when the device buffer object at `buf` gets new memory: if the object lies inside a
// live index, that index's generation advances (a captured batch graph that holds the old
// pointer is then refused).  capi.cu keeps the registry of live indices.
void note_buffer_moved(const void *buf);

// A buffer frees itself when it goes out of scope (so scratch buffers are returned on every
// path, early error returns included); it cannot be copied, so no two owners share a pointer.
template <typename T>
struct DevBuf {
    T *ptr = nullptr;
    size_t count = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    pts_status ensure(size_t n, const char *what) {
        if (n <= count && ptr) return PTS_OK;
        if (ptr) dev_free(ptr);
        ptr = nullptr;
        count = 0;
        note_buffer_moved(this);
        if (n == 0) n = 1;
        void *p = nullptr;
        PTS_TRY(dev_alloc(&p, n * sizeof(T), what));
        ptr = static_cast<T *>(p);
        count = n;
        return PTS_OK;
    }
    void release() {
        if (ptr) {
            dev_free(ptr);
            note_buffer_moved(this);
        }
        ptr = nullptr;
        count = 0;
    }
};

struct Workspace {
    int q_cap = 0;
    DevBuf<float> qcoord;      // [Qpad][da] query search vectors (y, r, 0...)
    DevBuf<float> qnorm;       // [Qpad] ||u_q||^2
    DevBuf<float> tau;         // [Qpad] rounding slack of the bound
    DevBuf<int> cand_idx;      // [Q][32]
    DevBuf<float> cand_lb;     // [Q][32]
    DevBuf<int> fail_list;     // [Q] queries not certified by the PCA pass
    DevBuf<int> fail2_list;    // [Q] queries not certified by the full-dimension pass
    DevBuf<float> qfull;       // [Qpad/64][Dp][64] centred full vectors of failing queries
    DevBuf<float> full_pdist;  // [splits][Q][ntiles*128] partial sums of a split full pass
    DevBuf<unsigned long long> best64;  // [Q] packed (d2 bits, n)
    DevBuf<float> thr0;        // [Q][2] warm-start bounds (one per column half of a tile)
    DevBuf<float> pca_thr;     // [Q] warm-start bound of the exact PCA pass
    DevBuf<unsigned int> hist; // [2][3][256] channel histograms (image, exemplar)
    DevBuf<int> nn_prev;       // [Q] the previous search's windows (stopping rule)
    DevBuf<unsigned int> diff; // [1] how many windows changed
    DevBuf<__half> qtile;      // [ceil(Q/128)][128 x Ktc] FP16 query operand tiles
    DevBuf<uint8_t> qtile8;    // [ceil(Q/128)][128 x Kf8] FP8 query operand tiles
    DevBuf<float> qscale;      // [Q] FP8 query row scales
    DevBuf<__half> qtile16;    // [ceil(Q/128)][128 x tcf_k(D)] FP16 full-dimension query tiles
    DevBuf<float> tau_tc;      // [Q] slack of the full-dimension FP16 scores
    DevBuf<float> proj_part;   // per-slice partial sums of a split projection
    DevBuf<unsigned char> kept;  // kept groups of the tensor-core search, one record per (row, half)
    DevBuf<float> part_v;      // [Q][parts][32] per-part candidate lists of the tensor-core search
    DevBuf<int> part_i;
    int warm_q = -1, warm_ho = -1, warm_wo = -1, warm_stride = -1;  // geometry of cand_idx
    DevBuf<unsigned int> counters;  // [4]: fail, fail2, brute, spare
    DevBuf<int> nn;            // [Q] (synthesize_level)
    DevBuf<float> d2;          // [Q]
    DevBuf<float> wts;         // [Q]
    DevBuf<double> energy;     // [iters+1]
    DevBuf<double> partial;    // reduction partials
    DevBuf<unsigned int> ticket;
};

// ---------------------------------------------------------------------------
// learned proposal state (kmeans.cu, mlp.cu, probe.cu)
// ---------------------------------------------------------------------------
constexpr int kMlpH = 256;       // hidden width of the proposal network
constexpr int kMlpChunk = 65536; // queries per inference chunk

struct MlpState {
    int C = 0, bmax = 0;
    DevBuf<float> params, grads, adam_m, adam_v;  // FP32 master weights, packed
    DevBuf<__nv_bfloat16> wb, wt;                 // BF16 weights and their transposes
    DevBuf<__nv_bfloat16> xb, xt, h1b, h1t, h2b, h2t, dzb, dzt, dab, dat;
    DevBuf<float> a1, a2, z, dh, loss;
    DevBuf<int> labels;
    pts_status ensure(int C_, int Bmax, cudaStream_t st);
};

struct MlpInfer {  // packed weights of the fused inference kernel (mlp_infer.cu)
    int ready = 0, nchunk = 0;
    DevBuf<__nv_bfloat16> wp1, wp2, wp3;
    DevBuf<float> b3p;
    const float *b1 = nullptr, *b2 = nullptr;
};

// the paper's hierarchical k-means tree (k = 4), kmtree.cu
struct KmTree {
    DevBuf<float> cent;          // [internal][4][d] child centroids
    DevBuf<int> child;           // [internal][4]: >= 0 internal, <= -2 leaf -c - 2, -1 none
    DevBuf<int> leaf_begin, leaf_end;  // ranges in perm
    DevBuf<int> perm;            // windows in leaf order
    DevBuf<int> tmp;             // build scratch
    DevBuf<unsigned char> label; // build scratch
    DevBuf<int> leaf_of_query;   // [Q] the leaf each query reached (last search)
    int n_internal = 0, n_leaves = 0, depth = 0, d = 0, N = 0, ready = 0;
};

struct ProposalState {
    int ready = 0, C = 0;
    float factor = 1.2f;
    DevBuf<float> centroids;  // [C][d]
    DevBuf<int> assign;       // [N] cluster of each exemplar window
    DevBuf<int> counts;       // [C]
    DevBuf<int> off;          // [C+1] CSR offsets
    DevBuf<int> members;      // [N] windows in cluster order
    DevBuf<float> median;     // [C] median nearest-neighbour distance of the cluster's pairs
    DevBuf<int> top;          // [Q][4] probed clusters
    DevBuf<__half> etc_ivf;   // FP16 exemplar tiles with the windows in cluster order (members)
    DevBuf<int> ivf_cnt, ivf_poff, ivf_cursor, ivf_nblk, pair_q, pair_r;
    DevBuf<int4> ivf_blk;
    DevBuf<__half> ivf_qtile;
    DevBuf<float> ivf_part_v;
    DevBuf<int> ivf_part_i;
    DevBuf<unsigned char> ivf_kept;
    MlpState mlp;
    MlpInfer infer;
};

}  // namespace pts

struct pts_index_s {
    int device = 0;
    int C = 3;  // channels per pixel: 3 (RGB) or 4 (RGB + the scale map, section 1)
    int He = 0, We = 0, w = 0, D = 0, N = 0, d = 0, da = 0;
    int d_fast = 0, da_fast = 0;  // PCA dimensions / vector length of the fast modes
    int ny = 0, nx = 0;  // exemplar window grid
    int ntiles = 0;      // ceil(N / kBN)
    double var_retained = 0.0, eig_top = 0.0;
    int eig_iters = 0;
    float unorm2_max = 0.0f;
    pts::DevBuf<float> exemplar;  // He*We*3
    pts::DevBuf<float4> exemplar4; // He*We pixels as (r, g, b, 0): one 16-byte load per pixel
    pts::DevBuf<float> mu;        // D
    pts::DevBuf<float> basis;     // d*D
    pts::DevBuf<float> basisT;    // [D][128]: the basis transposed, 0 past the computed components
    pts::DevBuf<double> eig;      // d
    pts::DevBuf<float> et;        // [ntiles][da][kBN] = -2 * (y_n, r_n, 0...)
    pts::DevBuf<float> et_rows;   // [N][da], the same vectors window-major (warm-start bound)
    pts::DevBuf<float> enorm;     // [ntiles*kBN] ||u_n||^2, +inf for padding
    pts::DevBuf<float> efull;     // [ntiles][Dp][kBN] = -2 u_n (full dimension)
    pts::DevBuf<float> et_fast;   // [ntiles][da_fast][kBN] = -2 (y_n, r_n, 0...) with d_fast coordinates
    pts::DevBuf<float> et_fast_rows;  // [N][da_fast], the same vectors window-major (warm-start bound)
    double var_fast = 0.0;        // variance fraction the d_fast components keep
    int exact_fast = 0;           // exact bound: 0 d then d_fast, 1 d_fast only, 2 d only
    int last_cascade = 0;         // the last exact search ran the second (d_fast) bound on its listed queries
    pts::DevBuf<__half> etc;      // [tc_tiles(N)][tc_tile_rows() x Ktc] FP16 MMA operand tiles
    pts::DevBuf<uint8_t> etc8;    // [tc_tiles(N)][tc_tile_rows() x Kf8] FP8 E4M3 operand tiles
    pts::DevBuf<float> f8scale;   // [d_fast + 1] per-dimension scales of the FP8 tiles
    int kf8 = 0;                  // K of the FP8 search
    int ktc = 0;                  // K of the tensor-core search
    pts::DevBuf<unsigned char> basis16;  // the transposed basis' first d_fast rows as FP16 hi/lo tiles (project_tc.cu)
    bool basis16_ready = false;
    pts::DevBuf<__half> efull16;  // [tcf_tiles(N)][256 x tcf_k(D)] FP16 full-dimension tiles (PTS_EXACT_TC)
    int tcf_state = 0;            // those tiles: 0 not built, 1 ready, -1 unusable (a value out of FP16 range)
    pts::DevBuf<float> umax;      // [1]
    pts::DevBuf<int> status;      // [1] device status word
    pts::Workspace ws;
    pts_search_stats last{};
    int last_mode = 0;
    int tc_parts_override = 0;  // exemplar split of the tensor-core search chosen by the autotuner
    pts::ProposalState prop;
    pts::KmTree tree;
    unsigned long long generation = 0;  // advances whenever one of the index's buffers moves
};

namespace pts {
// Registry of live indices (capi.cu): register right after construction, unregister before the
// buffers are released.  index_generation returns false for an index that is not live.
void register_index(pts_index idx);
void unregister_index(pts_index idx);
bool index_generation(pts_index idx, unsigned long long *gen);
}  // namespace pts

namespace pts {

// ---------------------------------------------------------------------------
// launchers implemented in the .cu files
// ---------------------------------------------------------------------------
// pca.cu
pts_status nn_search_impl(pts_index idx, const float *X, int Ho, int Wo, int stride, int mode, int32_t *nn_out,
                          float *d2_out, cudaStream_t st);
pts_status ensure_workspace(pts_index idx, int Q);
pts_status check_grid_public(int H, int W, int w, int stride, const char *what);
void prof_suspend(bool on);
pts_status pca_fit_device(const float *exemplar, int He, int We, int C, int w, int d, double var_frac,
                          int max_iters, float *mean_out, float *basis_out, double *eig_out,
                          int *d_used, double *var_retained, double *eig_top, int *iters_used,
                          double *trace_out, int *status, cudaStream_t st);
// project.cu
void launch_project(const float *img, int H, int W, int C, int w, int stride, const float *mu,
                    const float *basisT, int d, int da, int layout, float *out_coord,
                    float *out_norm, float *out_tau, float tau_scale, const float *umax,
                    cudaStream_t st, DevBuf<float> *scratch = nullptr);
// The FP16 search's query operand straight from the image: each window's d coordinates, its
// residual and three ones, rounded to FP16, in the tensor-core query tiles (tc_query_blocks(Q) x
// kTcQueryRows rows of K), rows past the last query zero; ||u||^2 and tau as launch_project.
void launch_project_tile16(const float *img, int H, int W, int C, int w, int stride, const float *mu,
                           const float *basisT, int d, int K, __half *qtile, float *out_norm, float *out_tau,
                           float tau_scale, const float *umax, cudaStream_t st, DevBuf<float> *scratch = nullptr);
// project_tc.cu: the same outputs on the tensor cores (FP16 hi/lo split operands, FP32
// accumulation; d <= 124, K <= 128), the basis prepacked once per index by launch_pack_basis16
// (basis16_bytes(D) bytes)
void launch_project_tc16(const float *img, int H, int W, int C, int w, int stride, const float *mu,
                         const unsigned char *basis16, int d, int K, __half *qtile, float *out_norm, float *out_tau,
                         float tau_scale, const float *umax, int *status, cudaStream_t st,
                         DevBuf<float> *scratch = nullptr);
size_t basis16_bytes(int D);
bool project_tc16_fits(int H, int W, int C);  // image offsets within the kernel's 32-bit range
// the FP16 query tiles (Q rows of K, core-matrix layout) as row-major rows
void launch_tile16_rows(const __half *qtile, int Q, int K, __half *rows, cudaStream_t st);
void launch_pack_basis16(const float *basisT, int D, int d, unsigned char *basis16, cudaStream_t st);
void launch_basis_transpose(const float *basis, int dcount, int D, float *basisT, cudaStream_t st);
void launch_exemplar_pad(float *et, float *enorm, int N, int ntiles, int da, cudaStream_t st);
void launch_norm_max(const float *norm, int n, float *out, cudaStream_t st);
// search_f32.cu
// da: the stride of a search vector; dk <= da: its components that are not zero padding
void launch_search_topk(const float *qcoord, const float *qnorm, int Q, int da, int dk, const float *et,
                        const float *enorm, int ntiles, int *cand_idx, float *cand_lb, int *status,
                        cudaStream_t st, int nparts = 1,
                        float *part_v = nullptr, int *part_i = nullptr,
                        const float *thr_init = nullptr);
// The listed queries' rows of `rows` (da floats each, the first dk not zero padding) searched
// against tiles [ntiles][Dp][128] with the full pass's GEMM + top-32 (Dp a multiple of 32; qtiles
// holds [F/64][Dp][64]; part_v / part_i hold full_part_capacity(Q) entries).
void launch_search_rows(const float *rows, int da, int dk, const int *list, const unsigned int *count, int Q,
                        int Dp, float *qtiles, const float *etiles, const float *enorm, int ntiles, const float *qnorm,
                        int *cand_idx, float *cand_lb, float *part_v, int *part_i, int *status,
                        cudaStream_t st);
int launch_search_full(const float *X, int Wo, int C, int w, int stride, int qx, const float *mu,
                        const int *fail_list, const unsigned int *fail_count, int Q,
                        float *qfull, const float *efull, const float *enorm, int ntiles,
                        const float *qnorm, int *cand_idx, float *cand_lb, float *part_v, int *part_i,
                        int *status, cudaStream_t st, int N,
                        DevBuf<float> *pdist);
// entries of each part list the full-dimension passes need for Q queries
size_t full_part_capacity(int Q);
int pca_parts(int Q, int ntiles);
void launch_tiles_to_rows(const float *et, int N, int da, float *rows, cudaStream_t st);
void launch_warm_pca(const int *prev_idx, const float *qcoord, int da, const float *et_rows, const float *enorm, int Q,
                     int N, float *thr, cudaStream_t st);
void launch_exemplar_full(const float *Z, int We, int C, int w, int ex, int N, const float *mu,
                          float *efull, int ntiles, cudaStream_t st);
// search_tc.cu
int tc_padded_k(int d);
int tc_query_blocks(int Q);
int tc_tiles(int N);
int tc_tile_rows();
int tc_parts(int Q, int ntiles);
void launch_pack_queries(const float *qcoord, int Q, int d, int da, int K, __half *qtile, cudaStream_t st,
                         const int *qlist = nullptr, const unsigned int *qcount = nullptr);
void launch_pack_exemplar(const float *et, const float *enorm, int N, int d, int da, int K, __half *out,
                          cudaStream_t st, const int *perm = nullptr);
// learned proposal probe on the tensor cores (cluster-ordered exemplar tiles)
struct IvfBuffers {
    int *cnt, *poff, *cursor, *nblk, *pair_q, *pair_r;
    int4 *blk;
    __half *qtile;
    float *part_v;
    int *part_i;
    void *kept;
};
int ivf_max_blocks(int Q, int C);
void tc_tail_plan(int Q, int ntiles, int *tail_from, int *tail_parts);
size_t tc_kept_bytes_search(int Q, int ntiles, int nparts);
size_t tc_kept_bytes(int Q, int nparts);
void launch_ivf_probe(const int *top, int Q, int C, const int *moff, const float *qcoord, const float *qnorm, int d,
                      int da, int K, const __half *etile_ivf, int ntiles, int N, const int *members, IvfBuffers &b,
                      int *cand_idx, float *cand_lb, int *status, cudaStream_t st);
void launch_warm_threshold(const int *prev_idx, const __half *qtile, const float *qnorm, const __half *etile,
                           const float *umax, int Q, int K, int N, float eps_scale, float *thr0, cudaStream_t st);
void launch_search_tc(const void *qtile, const float *qnorm, int Q, int K, const void *etile, int ntiles,
                      int nparts, const float *thr0, int *cand_idx, float *cand_lb, float *part_v, int *part_i,
                      int *status, cudaStream_t st, const int *qlist, const unsigned int *qcount, int fp8,
                      const float *qscale, const float *enorm, int N, void *kept_buf);
int tc_padded_k8(int d);
void launch_fp8_tables(const float *et, int N, int d, int da, int K, float *scale, uint8_t *out, cudaStream_t st);
void launch_pack_queries_f8(const float *qcoord, int Q, int d, int da, int K, const float *scale, uint8_t *qtile,
                            float *qscale, cudaStream_t st, const int *qlist = nullptr,
                            const unsigned int *qcount = nullptr);
pts_status tc_selftest(int N, int K, int f16, double *max_abs_err, double *max_abs_ref);
// kmeans.cu
pts_status kmeans_device(const float *Y, int n, int d, int k, const double *u, int iters, float *C, int *assign,
                         float *cost, int *counts, int *off, int *members, int *iters_used, cudaStream_t st);
void launch_extract_y(const float *et, int N, int da, int d, float *Y, cudaStream_t st);
pts_status cluster_medians(const int *nn, const float *d2, int n, const int *assign, int N, int C, int *lab,
                           float *dist, float *median, cudaStream_t st);
// mlp_infer.cu
pts_status mlp_pack_infer(MlpState &s, MlpInfer &f, cudaStream_t st);
void launch_mlp_top4(const MlpInfer &f, const float *qcoord, int Q, int d, int ldq, int *top, int *status,
                     cudaStream_t st);
// probe.cu
void launch_top4(const float *logits, int Q, int C, int *top, cudaStream_t st);
void launch_fallback(const int *nn, const float *d2, int Q, const int *assign, const float *median, float factor,
                     int N, int *list, unsigned int *count, cudaStream_t st);
// mlp.cu / gemm_tc.cu
long mlp_param_count(int C);
void mlp_refresh_bf16(MlpState &s, cudaStream_t st);
void mlp_forward(MlpState &s, int B, int train, int *status, cudaStream_t st);
void mlp_backward(MlpState &s, int B, const int *labels, int *status, cudaStream_t st);
void mlp_adamw(MlpState &s, float lr, float wd, int step, cudaStream_t st);
void mlp_gather(MlpState &s, const float *Y, int d, int ldy, const int *perm, int off, int B, const int *lab_all,
                cudaStream_t st);
pts_status gemm_selftest(int M, int N, int K, double *max_rel_err);
// full-dimension vectors are padded with zero rows to a multiple of 32
inline int padded_dim(int D) { return (D + 31) / 32 * 32; }
// rerank.cu
struct RerankArgs {
    const float *X;
    int Ho, Wo, stride, qx;
    const float *Z;
    int We, w, ex, N;
    int Q;
    int C;  // channels per pixel of both images (3: RGB, 4: RGB + scale)
    const float4 *Z4;  // the exemplar as one (r, g, b, scale or 0) float4 per pixel
};
// qlist/qcount == NULL: all Q queries; else the listed ones (count on the device)
void launch_list_all(int *list, unsigned int *count, int Q, cudaStream_t st);
void launch_rerank(const RerankArgs &a, const int *qlist, const unsigned int *qcount,
                   const int *cand_idx, const float *cand_lb, const float *tau, int certify,
                   int *nn_out, float *d2_out, int *fail_list, unsigned int *fail_count,
                   unsigned long long *best64, int *status, cudaStream_t st);
void launch_brute_fallback(const RerankArgs &a, const int *fail_list,
                           const unsigned int *fail_count, unsigned int *brute_count,
                           unsigned long long *best64, int *status, cudaStream_t st);
void launch_resolve(const int *fail_list, const unsigned int *fail_count,
                    const unsigned long long *best64, int Q, int *nn_out, float *d2_out,
                    cudaStream_t st);
// search_tcf.cu: the full-dimension FP16 tensor-core search (PTS_EXACT_TC)
int tcf_k(int D);             // K of its operands: D rounded up to 64
int tcf_tiles(int N);         // 256-window tiles
int tcf_query_blocks(int Q);  // 128-query blocks
// s (z - mu) of every exemplar window in FP16 tiles; *over is set when a value leaves the FP16 range
void launch_pack_exemplar_full16(const float *Z, int We, int C, int w, int nx, int N, const float *mu,
                                 __half *etile, int *over, cudaStream_t st);
// Every query window (all Q of the grid) packed for the full-dimension GEMM, with ||u_q||^2, exact
// mode's slack tau (tau_scale per unit) and the GEMM's tau_tc (tc_scale per unit, +inf for a query
// with a value past the FP16 range) from the same pass; then the GEMM and the top-32 of every query.
void launch_pack_queries_full16(const float *X, int Wo, int C, int w, int stride, int qx, int Q, const float *mu,
                                __half *qtile, float *qnorm, float *tau, float tau_scale, float *tau_tc, float tc_scale,
                                const float *umax, cudaStream_t st);
void launch_gemm_tcf(const __half *qtile, int Q, int C, int w, const __half *etile, int N, const float *enorm,
                     const float *qnorm, float *score, int *cand_idx, float *cand_lb, int *status, cudaStream_t st);
// the 32 smallest of the sum over splits of score[split][f][n] (n < N) for queries q0 + f, f < nq
// (search_f32.cu)
void launch_full_select_range(const float *score, int nsplit, int npad, int N, int q0, int nq, int Q,
                              const float *qnorm, int *cand_idx, float *cand_lb, int *status, cudaStream_t st);
// profile.cu: launch counting and event timing of kernel classes
enum ProfClass { kProfSearchTopk = 0, kProfSearchFull, kProfRerank, kProfProject, kProfMStep,
                 kProfSearchTc, kProfMlp, kProfProbe, kProfBrute, kProfIrls, kProfSearchTcList, kProfSearchTcf,
                 kProfClasses };
void count_launches(int n);
// Raises a kernel's dynamic shared-memory limit on the current device (once per kernel, device
// and size; thread-safe).
void set_smem_attr(const void *kernel, int bytes);
void prof_begin(int cls, cudaStream_t st, void **token);
void prof_end(int cls, cudaStream_t st, void *token);
struct ProfScope {
    int cls;
    cudaStream_t st;
    void *tok;
    ProfScope(int c, cudaStream_t s, int nlaunch) : cls(c), st(s), tok(nullptr) {
        count_launches(nlaunch);
        prof_begin(c, s, &tok);
    }
    ~ProfScope() { prof_end(cls, st, tok); }
};
// mstep.cu
void launch_rgba(const float *Z, long npix, int C, float4 *out, cudaStream_t st);
void launch_count_diff(const int *a, const int *b, int n, unsigned int *count, cudaStream_t st);
// kmtree.cu (section 2.2's k-means tree)
pts_status build_kmtree(KmTree &tr, const float *rows, int N, int da, int d, int iters, cudaStream_t st);
void launch_tree_search(const KmTree &tr, const float *qcoord, int da_q, int Q, int *cand_idx, float *cand_lb,
                        int *leaf_out, cudaStream_t st);
// histogram.cu (section 3, Eq. 9)
constexpr int kMaxHistBins = 256;
// bin of a channel value: clamped to [0, 1], times nbins in FP32, floored, capped at the last bin
__device__ __forceinline__ int hist_bin(float v, int nbins) {
    const float c = fminf(fmaxf(v, 0.0f), 1.0f);
    return min((int)floorf(c * (float)nbins), nbins - 1);
}
void launch_hist3(const float *img, long npix, int nbins, unsigned int *counts, cudaStream_t st);
void launch_hist_match(float *img, long npix, int nbins, const unsigned int *cx, long nx, const unsigned int *cz,
                       long nz, cudaStream_t st);
void launch_m_step_hist(const int *nn, const float *wts, const float4 *Z4, int We, int ex, int N, int w, int Ho, int Wo,
                        int stride, int nbins, const unsigned int *cx, long nx, const unsigned int *cz, long nz,
                        float *out, int *status, cudaStream_t st);
void launch_m_step(const int *nn, const float *wts, const float4 *Z4, int We, int ex, int N, int C, int w,
                   int Ho, int Wo, int stride, float *out, int *status, cudaStream_t st);
void launch_irls(const float *d2, int Q, float r, float delta, float *wts, double *energy_out,
                 double *partial, unsigned int *ticket, cudaStream_t st);
void launch_downsample2(const float *in, int H, int W, float *out, cudaStream_t st);
void launch_upsample2(const float *in, int H, int W, float *out, cudaStream_t st);
constexpr int kIrlsGrid = 152;

}  // namespace pts

// ---------------------------------------------------------------------------
// device helpers: mbarrier + bulk copies with bounded waits
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace pts {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with the given parity to complete.  Gives up after
// ~1 s of wall time (or 2^26 polls), sets kDevErrTimeout and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t i = 0; i < (1u << 26); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && global_timer_ns() - t0 > 1000000000ull) break;
    }
    atomicOr(status, kDevErrTimeout);
    return false;
}

// 1-D bulk copy global -> shared completing on an mbarrier (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ unsigned long long pack_dist_idx(float d2, int n) {
    return (static_cast<unsigned long long>(__float_as_uint(d2)) << 32) |
           static_cast<unsigned int>(n);
}

}  // namespace pts
#endif
