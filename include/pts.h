/*
 * pts.h -- C ABI of the GB300 (sm_103a) library for perspective texture
 * synthesis by energy optimisation (Bashir & Ghouri, arXiv:2006.11851).
 *
 * The library implements the hot path of the method's optimisation stage:
 *   - the search phase (E-step, section 2.1 and Eq. 4): every output
 *     neighbourhood on the 2x2-patch grid (section 2.2) is matched to its
 *     nearest exemplar neighbourhood, searched after PCA reduction
 *     (section 2.2);
 *   - the optimization phase (M-step, Eq. 8 minimised over x): output pixels
 *     become the weighted mean of the matched windows that cover them, with
 *     IRLS weights W_p = ||x_p - z_p||^(r-2) (Eqs. 5-7);
 *   - the coarse-to-fine driver (section 2.1).
 *
 * Conventions used by every entry point:
 *   images     float32, H x W x C, row-major, channel fastest (HWC), DEVICE
 *              memory owned by the caller; C = 3 (RGB), or C = 4 (RGBS: RGB
 *              and the scale map of section 1 as a fourth channel) for the
 *              images an RGBS index searches and updates;
 *   window     the w x w block whose top-left pixel is (y0, x0); vector
 *              element (dy, dx, c) is number (dy*w + dx)*C + c; D = C w^2;
 *   exemplar   windows at every stride-1 origin inside the exemplar:
 *              N = (He-w+1)(We-w+1), index n = y*(We-w+1) + x;
 *   queries    output windows whose origins lie on the stride grid
 *              y0 in {0, s, ..., Ho-w}: Q = ((Ho-w)/s+1)((Wo-w)/s+1),
 *              index q = (y0/s)*((Wo-w)/s+1) + x0/s.  (Ho-w) and (Wo-w) must
 *              be multiples of s, and w a multiple of s, so that every pixel
 *              is covered and all pixels of an s x s patch share one covering
 *              set;
 *   streams    every call is asynchronous on `stream` (a cudaStream_t, NULL =
 *              legacy default stream) unless its comment says it synchronises;
 *   errors     a call returns PTS_OK or a negative pts_status.  Argument
 *              errors are detected on the host before anything is launched.
 *              Device-side checks (index bounds, bounded waits) set a status
 *              word in the index; synchronising calls return it as
 *              PTS_ERR_DEVICE / PTS_ERR_TIMEOUT, and pts_index_device_status
 *              reads it.  pts_last_error() gives a thread-local message.
 *   threading  an index must not be used by two host threads at once.
 */
#ifndef PTS_H
#define PTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PTS_OK = 0,
    PTS_ERR_INVALID_ARG = -1, /* bad size, pointer, mode or grid */
    PTS_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    PTS_ERR_OOM = -3,         /* device allocation failed */
    PTS_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    PTS_ERR_UNSUPPORTED = -6, /* valid request the library does not support */
    PTS_ERR_DEVICE = -7       /* a device-side check failed (see message) */
} pts_status;

/* Search modes of the E-step.
 *   PTS_EXACT_F32     the full-dimension nearest neighbour of Eq. 4.  PCA
 *                     coordinates plus the residual norm give a lower bound
 *                     on every full-dimension distance; the 32 best bounds
 *                     are re-ranked in full dimension and certified (the
 *                     best distance lies below the 32nd bound by a slack
 *                     tau_q = 8 sqrt(D) 2^-24 (||u_q||^2 + max_n ||u_n||^2)
 *                     that models FP32 rounding; it is not a worst-case
 *                     bound).  Queries the first d components leave
 *                     uncertified get the same bound with the index's d_fast
 *                     components, then a full-dimension GEMM pass (top-32
 *                     again, re-ranked, certified the same way), and what
 *                     still fails a direct scan.  FP32 SIMT, no tensor cores.
 *   PTS_F16_RERANK    PCA-space bounds (d_fast coordinates + residual) as an
 *                     FP16 tensor-core GEMM (FP32 accumulate), top-32 by
 *                     bound, exact FP32 full-dimension re-rank.  Not
 *                     certified: a window whose FP16-rounded bound misses the
 *                     32 best is lost.
 *   PTS_FP8_RERANK    as F16 with FP8-E4M3 operands (kind::f8f6f4): the exemplar
 *                     side holds -2 y / s_j with per-dimension scales s_j =
 *                     max_n |2 y_nj| / 448, the query y s_j / t_q with a per-row
 *                     scale t_q; the epilogue forms ||u_n||^2 + t_q acc in FP32.
 *                     Not certified; every candidate is re-ranked in FP32.
 *   PTS_PROPOSAL      learned cluster proposal: the network ranks k-means
 *                     clusters, the 4 best are probed on the FP16 tensor cores,
 *                     the candidates re-ranked in exact FP32; queries whose
 *                     result fails the distance test (pts_train_proposal) are
 *                     searched as in PTS_F16_RERANK.
 *   PTS_KMTREE        the paper's own search (section 2.2): greedy descent of a
 *                     k = 4 hierarchical k-means tree over the PCA coordinates
 *                     (pts_build_kmeans_tree) to a leaf, whose windows are
 *                     re-ranked in exact FP32.  Approximate.
 *   PTS_EXACT_TC      the nearest windows of PTS_EXACT_F32 through the tensor
 *                     cores: full-dimension scores ||u_n||^2 - 2 u_q . u_n from
 *                     an FP16 GEMM of 2^12 u (FP32 accumulate) over all D
 *                     components, the 32 best re-ranked in FP32 and certified
 *                     with tau_q = ((2^-9 + (D + 2) 2^-22)(1 + 2^-10) +
 *                     8 sqrt(D) 2^-24)(||u_q||^2 + max_n ||u_n||^2): the FP16
 *                     rounding of both operands and an FP32 accumulation
 *                     allowed 2^-22 relative error per addition, bounded in
 *                     the worst case, plus the FP32 model of PTS_EXACT_F32.
 *                     Uncertified queries (and queries with a value |x - mu|
 *                     >= 16, past the FP16 range) take PTS_EXACT_F32's
 *                     full-dimension pass.  The results are those of
 *                     PTS_EXACT_F32.  For levels whose PCA keeps too little
 *                     variance for a useful PCA bound (the coarse levels).
 *                     The scores of all pairs go through device memory, so the
 *                     mode runs PTS_EXACT_F32 instead when they would take
 *                     more than 256 MB (Q times N rounded up to 256, 4 bytes
 *                     each), where moving them costs more than the FP32
 *                     route's bounds save.  The index builds its FP16 tiles
 *                     (2 D bytes per window) on the first such search.  The
 *                     mode also runs PTS_EXACT_F32 when an exemplar value lies
 *                     past the FP16 range or max_n ||u_n||^2 < D 2^-21 (a nearly
 *                     constant exemplar, where FP16 underflow would not be
 *                     covered). */
typedef enum {
    PTS_EXACT_F32 = 0,
    PTS_F16_RERANK = 1,
    PTS_FP8_RERANK = 2,
    PTS_PROPOSAL = 3,
    PTS_KMTREE = 4,
    PTS_EXACT_TC = 5
} pts_mode;

typedef struct pts_index_s *pts_index; /* opaque, owned by the library */

typedef struct {
    int d;           /* PCA dimensions, 1..64; <= 0: smallest d whose retained
                        variance reaches var_frac (section 2.2 keeps 95%),
                        capped at 64 */
    double var_frac; /* used when d <= 0 */
    int max_iters;   /* eigen-solver iteration cap (0 = 200) */
    int d_fast;      /* PCA dimensions of the tensor-core and proposal searches, 1..124
                        (0 = 124; capped by the covariance rank min(D, N - 1)) */
    int channels;    /* 0 or 3: RGB images; 4: RGBS images (sections 2.2 and 3: the scale
                        map as a fourth channel; D = 4 w^2).  With 4, the exemplar and every
                        image searched or updated have 4 channels, the M-step updates R, G
                        and B and leaves the fourth channel as it is, and the histogram
                        entry points are refused */
} pts_index_params;

typedef struct {
    int He, We, w, D, N, d;
    int da;                  /* search vector length: d coordinates + residual, padded to 4 */
    int d_fast;              /* PCA dimensions of the tensor-core and proposal searches */
    double var_retained;     /* sum of the d eigenvalues / trace of the covariance */
    double eig_top;          /* largest eigenvalue */
    int eig_iters;           /* subspace iterations used */
    float unorm2_max;        /* max_n ||v_n - mu||^2 over exemplar windows */
    int channels;            /* channels per pixel of the images: 3 (RGB) or 4 (RGBS) */
    int exact_dims;          /* PCA components of the exact search's lower bound */
    double exact_var;        /* the variance fraction they keep (below 0.85 the exact search
                                skips its PCA pass and scans every window in full dimension) */
} pts_index_info;

typedef struct {
    long long queries;        /* queries of the last nn_search */
    long long certified;      /* exact mode: certified from the 32 best bounds of the first PCA bound */
    long long range_queries;  /* exact mode: queries the first bound did not certify (sent to the
                                 second bound when it runs, else to the full-dimension pass) */
    long long range_pairs;    /* exact mode: queries the full-dimension pass did not certify */
    long long brute_queries;  /* exact mode: queries that needed a direct scan */
    long long fallback_queries; /* proposal mode: queries sent to the exact search */
    long long full_splits;    /* exact mode: pieces the full-dimension pass cut the window
                                 vectors into (partial sums added in fixed order); 1 = not
                                 cut, 0 = no full-dimension pass ran */
    long long second_certified; /* exact mode: queries the second bound (the index's d_fast
                                 components, run on the first bound's uncertified queries)
                                 certified */
    long long full_queries;   /* exact mode: queries the full-dimension pass searched */
    long long second_queries; /* exact mode: queries the second bound searched (0 when it did not run) */
} pts_search_stats;

/* Parameters of the learned cluster proposal (pts_train_proposal). */
typedef struct {
    int n_clusters;        /* k-means clusters over the exemplar's PCA vectors, 4..1024 */
    int kmeans_iters;      /* Lloyd iteration cap (0 = 25) */
    int epochs;            /* training epochs (0 = 8) */
    int batch;             /* minibatch size, a multiple of 8 (0 = 4096) */
    float lr;              /* peak AdamW learning rate, cosine decay to 0 (0 = 1e-3) */
    float weight_decay;    /* AdamW decoupled weight decay (0 = 1e-4) */
    float fallback_factor; /* exact fallback when the re-ranked distance exceeds this many
                              times the median distance of the window's cluster (0 = 1.2) */
    unsigned long long seed; /* k-means++ uniforms, weight initialisation and batch order */
} pts_proposal_params;

/* Message describing the last error on this host thread ("" if none). */
const char *pts_last_error(void);

/* Library version string. */
const char *pts_version(void);

/*
 * Device memory (no counterpart in the paper).  Every buffer the library owns (index tables,
 * workspaces, scratch) is allocated through one pair of functions: cudaMalloc / cudaFree by
 * default, or the caller's, e.g. a framework's caching allocator.
 *   alloc(bytes, stream, user)  returns device memory of at least `bytes` bytes on the current
 *                               device, or NULL on failure (the library call then returns
 *                               PTS_ERR_OOM); `stream` is always NULL (the legacy stream);
 *   release(ptr, stream, user)  takes back a pointer alloc returned.  The library synchronises
 *                               the device first, as cudaFree does, so nothing it queued still
 *                               reads the memory.
 * pts_set_allocator installs both (alloc and release non-NULL) or restores cudaMalloc /
 * cudaFree (both NULL); one NULL is PTS_ERR_INVALID_ARG.  It may be called only while the
 * library holds no device memory (no index or batch alive): otherwise PTS_ERR_INVALID_ARG, so
 * no pointer is ever returned to an allocator that did not make it.  Not to be called
 * concurrently with other library calls.
 * pts_live_allocations counts the library's allocations not yet freed (every destroy call
 * brings it back to where it was before the matching create).
 */
typedef void *(*pts_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*pts_free_fn)(void *ptr, void *stream, void *user);
pts_status pts_set_allocator(pts_alloc_fn alloc, pts_free_fn release, void *user);
long long pts_live_allocations(void);

/*
 * pca_fit -- PCA of the exemplar's neighbourhood vectors (section 2.2: the
 * search runs on PCA-reduced vectors; the paper keeps 95% of the variance).
 * d may be up to 128 here; an index keeps up to max(d, d_fast) components.
 *   mu    = (1/N) sum_n v_n,  Sigma = (1/N) sum_n (v_n - mu)(v_n - mu)^T,
 * both accumulated in FP64 on the GPU; the top-d eigenpairs of Sigma come
 * from FP64 subspace iteration with Rayleigh-Ritz steps solved by Jacobi.
 * exemplar    device, He x We x 3 float32.
 * d           1..128, or <= 0 to choose the smallest d <= 64 reaching var_frac.
 * mean_out    device, D float32 (may be NULL).
 * basis_out   device, d x D float32, row j = unit eigenvector j (eigenvalues
 *             descending); must hold 64 x D floats when d <= 0.
 * eigvals_out device, d float64 (may be NULL).
 * d_out       host int receiving the d used (may be NULL).
 * Synchronises `stream`.  Errors: INVALID_ARG if w > He or We, d > min(D, N-1).
 */
pts_status pca_fit(const float *exemplar, int He, int We, int w, int d, double var_frac,
                   float *mean_out, float *basis_out, double *eigvals_out, int *d_out, void *stream);
/* pca_fit for images of C channels (3: RGB, 4: RGBS, the scale map as a fourth channel,
 * sections 2.2 and 3): exemplar device He x We x C float32, D = C w^2; otherwise as pca_fit. */
pts_status pca_fit_channels(const float *exemplar, int He, int We, int C, int w, int d, double var_frac,
                            float *mean_out, float *basis_out, double *eigvals_out, int *d_out, void *stream);

/*
 * build_exemplar_index -- everything the search needs about one exemplar and
 * window width: a device copy of the exemplar, the PCA (as pca_fit), and the
 * projected exemplar windows y_n = B^T(v_n - mu) with their residual norms
 * ||(I - B B^T)(v_n - mu)|| and squared norms ||v_n - mu||^2 (section 2.2).
 * exemplar is a device pointer to He x We x C float32 (C = params->channels:
 * 3, or 4 for an RGBS exemplar whose fourth channel is its scale map); the
 * index keeps its own copy, so the caller may free it afterwards.
 * Synchronises `stream`.  *out receives a new index (release it with
 * pts_index_destroy).
 */
pts_status build_exemplar_index(const float *exemplar, int He, int We, int w,
                                const pts_index_params *params, void *stream, pts_index *out);

/* Frees an index and all its device memory (NULL is ignored).  Synchronises
 * the device. */
void pts_index_destroy(pts_index index);

/* Fills *info (host) with the index's sizes and PCA summary. */
pts_status pts_index_get_info(pts_index index, pts_index_info *info);

/*
 * Index files (section 2.2's preprocessing run once per exemplar and window width).
 * pts_index_save writes everything a search needs -- the exemplar, the PCA (mean, basis,
 * eigenvalues), every search table, and, when present, the trained proposal (clusters,
 * cluster-ordered tiles, the network's FP32 weights) and the k-means tree -- to `path`
 * (written under a temporary name, then renamed).  Synchronises the device.
 * pts_index_load reads such a file into a new index on the current device, owned by the caller
 * (free it with pts_index_destroy).  Every search on it returns what the same search on the
 * saved index returns.  The file's header, its length and the integer tables the kernels
 * index with (cluster offsets, members and assignments; tree links, leaf ranges and window
 * order) are checked before anything is allocated: a file that is not an index file, was
 * written with another byte order or layout version, is truncated, whose tables disagree with
 * its header, or whose integer tables are out of range gives PTS_ERR_INVALID_ARG
 * (see pts_last_error).  Synchronises the device.  Files are in host byte order; the x86-64 and
 * AArch64 hosts of this library share it.
 */
pts_status pts_index_save(pts_index index, const char *path);
pts_status pts_index_load(const char *path, pts_index *out);

/* Sets how many CTAs split the exemplar tiles of one 128-query block in the
 * tensor-core searches (PTS_F16_RERANK, PTS_FP8_RERANK); 0 restores the
 * automatic choice, which fills the 152 SMs when the query blocks alone do not,
 * and otherwise splits only the query blocks of the last, partial wave (one CTA
 * per SM), each over up to 4 CTAs, when at least one full wave precedes them.
 * The candidates, hence the results, are the same for every split: each part
 * keeps its own best groups and the merge takes the best of their union.
 * A tuning knob only (pts_batch_create sets it from timings).  PTS_ERR_INVALID_ARG
 * for a NULL index or parts < 0; parts larger than the tile count act as the
 * tile count. */
pts_status pts_index_set_tc_parts(pts_index index, int parts);

/* The components of the exact search's PCA lower bound (section 2.2's PCA; no counterpart in
 * the paper, a tuning knob).  fast = 0 (the default): every query is bounded with the index's
 * first d components, and the queries that bound cannot certify are bounded again with its d_fast
 * components (when d_fast > d) before the full-dimension pass takes what is left.  fast = 1: one
 * bound, with the d_fast components (each bound costs about twice as much).  fast = 2: one bound,
 * with the first d components.  Results are the certified nearest windows of Eq. 4 whatever the
 * choice.  PTS_ERR_INVALID_ARG for a NULL index or other values. */
pts_status pts_index_set_exact_bound(pts_index index, int fast);

/*
 * pts_build_kmeans_tree -- builds the search tree of PTS_KMTREE (section 2.2): hierarchical
 * k-means with k = 4 over the index's d PCA coordinates, each node split until it holds fewer
 * than 4 windows (a split that leaves a child with all of its parent's windows makes that child
 * a leaf).  Each split seeds the centroids with the node's windows at 1/8, 3/8, 5/8 and 7/8 of its
 * range and runs `iters` Lloyd iterations (1..100); deterministic.  Synchronises `stream` once
 * per tree level.
 * pts_kmtree_info -- internal nodes, leaves and levels of the built tree (host ints, any may be
 * NULL); PTS_ERR_INVALID_ARG when no tree is built.
 * pts_kmtree_export -- copies the tree to HOST arrays (each may be NULL): child[4 * internal]
 * (>= 0 internal node, <= -2 leaf -c - 2, -1 none), leaf_begin/leaf_end[leaves] (ranges of
 * perm), perm[N] (windows in leaf order), cent[4 * internal * d] (child centroids).
 * Synchronises `stream`.
 * pts_kmtree_last_leaves -- the leaf each query reached in the last PTS_KMTREE search (HOST,
 * Q ints).  Synchronises `stream`.
 */
pts_status pts_build_kmeans_tree(pts_index index, int iters, void *stream);
pts_status pts_kmtree_info(pts_index index, int *n_internal, int *n_leaves, int *depth);
pts_status pts_kmtree_export(pts_index index, int *child, int *leaf_begin, int *leaf_end, int *perm, float *cent,
                             void *stream);
pts_status pts_kmtree_last_leaves(pts_index index, int *leaves, int Q, void *stream);

/* Reads and clears the index's device status word (synchronises `stream`).
 * Returns PTS_OK, PTS_ERR_DEVICE or PTS_ERR_TIMEOUT. */
pts_status pts_index_device_status(pts_index index, void *stream);

/*
 * nn_search -- the search phase (E-step, Eq. 4): for every query window of
 * `output` (device, Ho x Wo x C float32, C the index's channels) on the stride grid, the index n of
 * its nearest exemplar window and the squared full-dimension distance
 * ||x_p - z_n||^2 computed in FP32 from the pixels.
 * nn_out     device, Q int32.   dist2_out  device, Q float32.
 * Ties within FP32 rounding may resolve to either window; exact ties go to
 * the smallest n.  Asynchronous; uses workspace owned by the index.
 */
pts_status nn_search(pts_index index, const float *output, int Ho, int Wo, int stride, int mode,
                     int32_t *nn_out, float *dist2_out, void *stream);

/*
 * pts_project_queries -- PCA coordinates y_q = B^T (x_q - mu) (section 2.2) of every query
 * window of `output` (device Ho x Wo x C), written to y_out (device Q x d float32, row-major).
 * Used to collect training pairs for the proposal.  Asynchronous.
 */
pts_status pts_project_queries(pts_index index, const float *output, int Ho, int Wo, int stride, float *y_out,
                               void *stream);

/*
 * pts_index_pca -- the index's PCA (section 2.2): mean_out (device, D float32) = mu, basis_out
 * (device, d_fast x D float32, row-major) = the first d_fast unit eigenvectors, the basis every
 * projection of the index uses.  Asynchronous; PTS_ERR_INVALID_ARG on a null argument.
 */
pts_status pts_index_pca(pts_index index, float *mean_out, float *basis_out, void *stream);

/*
 * pts_query_rows_f16 -- the rows the FP16 search (PTS_F16_RERANK) multiplies, for every query
 * window of `output` (device Ho x Wo x C): row q = (y_q, r_q, 1, 1, 1, 0, ...) rounded to FP16,
 * y_q = B^T (x_q - mu) the d_fast PCA coordinates, r_q = sqrt(max(0, ||u_q||^2 - ||y_q||^2)) the
 * residual norm (section 2.2), the three ones against the exemplar's norm slots.
 * tensor_cores  1: the projection the search runs (tcgen05, FP16 hi/lo split operands, FP32
 *               accumulation); 0: the FP32 SIMT projection, for comparison.
 * rows_out      device, Q x K FP16 values (IEEE binary16 bit patterns), row-major,
 *               K = 16 * ceil((d_fast + 4) / 16).
 * norm_out      device, Q float32: ||u_q||^2 = ||x_q - mu||^2.
 * Asynchronous; uses workspace owned by the index.  PTS_ERR_INVALID_ARG on a null pointer or a
 * grid the stride does not fit (as nn_search).
 */
pts_status pts_query_rows_f16(pts_index index, const float *output, int Ho, int Wo, int stride, int tensor_cores,
                              uint16_t *rows_out, float *norm_out, void *stream);

/*
 * pts_train_proposal -- builds the learned cluster proposal of PTS_PROPOSAL, which takes
 * the place of the paper's k-means search tree (section 2.2):
 *   1. k-means (k-means++ seeding, Lloyd) over the exemplar windows' PCA coordinates;
 *   2. labels: the cluster of each training pair's exact nearest window; per-cluster median
 *      of the pairs' nearest-neighbour distances (global median for clusters with < 5 pairs);
 *   3. trains the network 64 -> 256 -> 256 -> n_clusters (GELU) with softmax cross-entropy and
 *      AdamW on BF16 tensor-core GEMMs with FP32 master weights.
 * y       device n x d float32: query PCA coordinates (pts_project_queries);
 * nn, d2  device n int32 / float32: their exact nearest windows and squared distances
 *         (nn_search in PTS_EXACT_F32).
 * loss_out host array of `epochs` doubles (mean loss of each epoch's last batch), may be NULL.
 * Synchronises `stream`.
 */
pts_status pts_train_proposal(pts_index index, const float *y, const int32_t *nn, const float *d2, int n,
                              const pts_proposal_params *params, double *loss_out, void *stream);

/* The 4 clusters the trained network ranks first for each query of `output` (test support,
 * no counterpart in the paper): fused != 0 runs the fused inference kernel the search uses,
 * fused == 0 the training-side GEMM path plus a separate top-4 (the two must agree).
 * top_out device, Q x 4 int32.  Asynchronous. */
pts_status pts_proposal_top4(pts_index index, const float *output, int Ho, int Wo, int stride, int fused,
                             int32_t *top_out, void *stream);

/* Inspection of a trained proposal (test support, no counterpart in the paper): the number of
 * clusters, and optionally their sizes (host, n_clusters ints) and the cluster of every exemplar
 * window (host, N ints).  Synchronises the device.  INVALID_ARG when no proposal is trained. */
pts_status pts_proposal_info(pts_index index, int *n_clusters, int *sizes_out, int *assign_out);

/* Standalone k-means (test support, no counterpart in the paper): points device n x d float32,
 * u host k doubles in [0, 1) (k-means++ uniforms), centroids_out device k x d float32,
 * assign_out device n int32.  Returns the Lloyd iterations run in *iters_out (host, may be
 * NULL).  Synchronises the stream. */
pts_status pts_kmeans(const float *points, int n, int d, int k, const double *u, int iters,
                      float *centroids_out, int32_t *assign_out, int *iters_out, void *stream);

/* One forward/backward pass of the proposal network (test support): params device float32
 * packed [W1 256x64, b1 256, W2 256x256, b2 256, W3 Cx256, b3 C] (row-major [out][in]), X device
 * B x 64 float32 (rounded to BF16 here, as in training), labels device B int32; writes the
 * gradients of the mean cross-entropy (same packing) to grads_out and the loss to *loss_out
 * (host).  Synchronises the stream. */
pts_status pts_mlp_grad(int C, const float *params, const float *X, const int32_t *labels, int B,
                        float *grads_out, double *loss_out, void *stream);

/* Self-test of the BF16 tensor-core GEMM (test support): C = A B^T + bias, GELU, on seeded
 * data against an FP64 host product; writes the largest relative error.  Synchronises. */
pts_status pts_gemm_selftest(int M, int N, int K, double *max_rel_err);

/* Statistics of the last nn_search on this index (synchronises `stream`). */
pts_status pts_index_search_stats(pts_index index, pts_search_stats *stats, void *stream);

/*
 * irls_weights -- IRLS weights and energy (Eqs. 5-8): with d_p = sqrt(dist2_p),
 *   W_p = max(d_p, delta)^(r-2)      (Eq. 7; delta > 0 keeps W finite at d_p = 0)
 *   energy = sum_p d_p^r             (Eq. 5; Eq. 4 when r = 2)
 * dist2 device Q float32; weights_out device Q float32 (may be NULL);
 * energy_out device, one float64 (may be NULL).  The sum is deterministic
 * (fixed grid, fixed reduction order).  Asynchronous.
 */
pts_status irls_weights(const float *dist2, int Q, float r, float delta, float *weights_out,
                        double *energy_out, void *stream);

/*
 * irls_weights_noalloc -- irls_weights for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a deployment aid.  Some
 * callers must not call cudaMalloc or cudaFree while they run: a host
 * framework that owns the whole device memory budget through its own pool,
 * or a pipeline that cannot afford the device-wide synchronisation a
 * cudaFree implies.  irls_weights allocates (and frees) its reduction scratch
 * on every call; this variant allocates nothing and keeps that scratch (one
 * double per 2048 distances plus a completion counter, 32 KB in all) in a
 * fixed array compiled into the library, which every GPU that loads the
 * library holds until the process exits.
 * Same weights and energy as irls_weights (the energy may differ in the last
 * bits: the partial sums are grouped differently).  Limits and behaviour:
 *   Q           at most 8,388,608; larger Q returns PTS_ERR_INVALID_ARG;
 *   first call  in each CUDA context (each device's primary context, or a
 *               context the caller made current) looks up the array's
 *               device address (cudaGetSymbolAddress) and caches it under
 *               that context's id, so a device reset or a second context
 *               gets a fresh lookup; make that first call before any stream
 *               capture;
 *   sharing     all calls share the one array, which keeps the previous
 *               call's contents; each call clears the counter it needs, but
 *               calls that overlap on the GPU (for example on two streams)
 *               race on the array and must be serialised by the caller;
 *   energy_out  device pointer to one float64 (may be NULL);
 *   asynchronous on `stream` (unlike irls_weights, it does not synchronise).
 */
pts_status irls_weights_noalloc(const float *dist2, int Q, float r, float delta, float *weights_out,
                                double *energy_out, void *stream);

/*
 * m_step -- the optimization phase (Eq. 8 minimised over x): every pixel of
 * `output` becomes
 *   x_i = sum_{p covers i} W_p z_{nn(p)}[i - p] / sum_{p covers i} W_p,
 * computed once per s x s patch (section 2.2) by gathering from the index's
 * exemplar copy, in increasing query order, without atomics.
 * nn device Q int32 (values in [0, N)); weights device Q float32 or NULL
 * (all 1); output device Ho x Wo x C float32 (C the index's channels): R, G
 * and B overwritten (not read); with C = 4 the fourth channel is left as it
 * is (the output's scale map stays fixed, section 3).
 * Out-of-range nn values are clamped and flagged in the device status word.
 */
pts_status m_step(pts_index index, const int32_t *nn, const float *weights, int Ho, int Wo,
                  int stride, float *output, void *stream);

/*
 * synthesize_level -- `iters` EM iterations of the energy optimisation
 * (section 2.1) on one level: search phase (nn_search in `mode`), IRLS
 * weights (r, delta), optimization phase (m_step), repeated; then one last
 * search phase so that energy_out[iters] is the energy of the result.
 * output      device Ho x Wo x C (C the index's channels): in = initial image,
 *             out = result.
 * energy_out  HOST, iters + 1 float64: energy_out[t] is the energy of the
 *             iterate entering iteration t (Eq. 4 / Eq. 5).
 * Synchronises `stream` once at the end and returns the device status.
 */
pts_status synthesize_level(pts_index index, float *output, int Ho, int Wo, int stride, int iters,
                            float r, float delta, int mode, double *energy_out, void *stream);

/*
 * synthesize_level_async -- synthesize_level without its closing synchronisation, so that a
 * caller can queue several levels (or jobs) back to back: the energies go to energy_dev
 * (DEVICE, iters + 1 float64) and an error a kernel raises stays in the index's device status
 * word until pts_index_device_status reads it.  Host-side argument errors return at once.  The
 * first call on a new grid size may still synchronise (it sizes the workspace).
 */
pts_status synthesize_level_async(pts_index index, float *output, int Ho, int Wo, int stride, int iters,
                                  float r, float delta, int mode, double *energy_dev, void *stream);

/*
 * Histogram matching (section 3, Eq. 9; the last step of the synthesis
 * procedure, section 4).  Histograms: one per colour channel, nbins equal bins
 * over [0, 1] (2 <= nbins <= 256), as fractions of the image's pixels; a value's
 * bin is clamp(v, 0, 1) * nbins in FP32, floored, capped at nbins - 1.
 *
 * m_step_hist -- m_step with the weights of Eq. 9: the contribution of window
 * p to pixel i is weighted
 *   W_p,i = w_p / (1 + sum_j max[0, H_x,j(b_j(c)) - H_z,j(b_j(c))]),
 * c = z_{nn(p)}[i - p] the exemplar pixel it brings, j over the three channels,
 * H_x the histograms of `current` (the image the search phase matched, device
 * Ho x Wo x 3), H_z those of the index's exemplar; each pixel is divided by its
 * own sum of weights.  `output` may be `current` (its histograms are taken
 * first).  Other arguments and errors as m_step; PTS_ERR_INVALID_ARG for nbins
 * outside 2..256.  The energy is no longer guaranteed not to rise.
 *
 * pts_histogram_match -- each channel of `image` (device H x W x 3, in place)
 * mapped onto the exemplar's distribution, v -> F_z^-1(F_x(v)), with both CDFs
 * piecewise linear inside the bins (F(v) = C[b] + (v nbins - b) h[b] for v in
 * bin b; F_z^-1(u) = (m + (u - C_z[m]) / h_z[m]) / nbins for the non-empty bin
 * m with C_z[m] <= u < C_z[m+1], 1 beyond).  Asynchronous.
 *
 * synthesize_level_hist -- synthesize_level with the M-step of m_step_hist
 * (H_x re-taken before every M-step).  nbins must be in 2..256.
 */
pts_status m_step_hist(pts_index index, const int32_t *nn, const float *weights, int Ho, int Wo, int stride,
                       int nbins, const float *current, float *output, void *stream);
pts_status pts_histogram_match(pts_index index, float *image, int H, int W, int nbins, void *stream);
pts_status synthesize_level_hist(pts_index index, float *output, int Ho, int Wo, int stride, int iters, float r,
                                 float delta, int mode, int nbins, double *energy_out, void *stream);

/*
 * synthesize_level_converge -- the EM loop of synthesize_level with section
 * 2.1's stopping rule: iterate until the search phase returns, for every
 * query, the window it returned the iteration before (the set {z_p} no longer
 * changes), or until max_iters M-steps have run (max_iters >= 0).  nbins 0
 * takes the plain M-step, 2..256 that of m_step_hist.  The paper prefers the
 * robust r = 0.8 (delta as in synthesize_level).
 * energy_out  HOST, max_iters + 1 float64, of which iters_out + 1 are written:
 *             energy_out[t] is the energy of the iterate entering iteration t,
 *             energy_out[iters_out] that of the result.
 * iters_out   HOST, one int: the M-steps run.
 * Synchronises `stream` once per iteration (the rule reads a device count).
 */
pts_status synthesize_level_converge(pts_index index, float *output, int Ho, int Wo, int stride, int max_iters,
                                     float r, float delta, int mode, int nbins, double *energy_out, int *iters_out,
                                     void *stream);

/*
 * The scale map (Methodology section 1, Eqs. 1-3) and its use in synthesis (section 3).
 * Maps are DEVICE float64 arrays, row 0 at the top.  Readings: the image-plane origin is the
 * bottom-left pixel (row r has p(y) = h - 1 - r) and w/2, h/2 are real halves; Eq. 3's leading
 * term, printed as Y_max, is read as S_max, so S = S_max - (p(Y_proj) - Y_min) S_delta / Y_delta
 * runs from S_max (near pixel (1, 1)) to S_min (the top-right pixel) and is 1 everywhere for a
 * fronto-parallel plane.  Every value is FP64 with each operation rounded on its own, in the
 * order written (no fused multiply-add): bit-reproducible.
 *
 * pts_scale_map        Eqs. 1-3 for an h x w image: S_max = 1/cos(slant), S_min = cos(slant)
 *                      (Eq. 1); Y_max = (w-1-w/2) sin(tilt) + (h-1-h/2) cos(tilt), Y_min =
 *                      -Y_max (Eq. 2); S_out device h x w.  slant in [0, 90), tilt in [0, 90]
 *                      degrees; Y_delta = 0 is refused.  Asynchronous.
 * pts_scale_resample   section 3 step 2: S (He x We) resampled bilinearly, corner-aligned, to
 *                      Ho x Wo (all sides >= 2).  Asynchronous.
 * pts_scale_guided_init section 3 step 3: the initial output (out: device Ho x Wo x 3 float32)
 *                      filled from exemplar pixels of the same scale.  The exemplar map's range
 *                      [lo, hi] is cut into nbins (1..1024) equal bins, bin(s) = floor((s - lo) /
 *                      (hi - lo) nbins) clamped; output pixel o, in the bin of S_x[o], copies
 *                      exemplar pixel floor(u[o] m) of that bin's m pixels in raster order; an
 *                      empty bin borrows the nearest filled bin (the lower one on a tie).
 *                      exemplar device He x We x 3, S_z device He x We, S_x and u (uniforms in
 *                      [0, 1)) device Ho x Wo float64; src_out device Ho x Wo int32 (may be
 *                      NULL): the raster index of the exemplar pixel copied.  Synchronises
 *                      `stream` (its scratch is released before it returns).
 * pts_rgbs             the RGBS image of sections 2.2 and 3: out (device H x W x 4, 16-byte
 *                      aligned) = (R, G, B, lam S) from rgb (H x W x 3) and S (H x W float64),
 *                      the fourth value lam S rounded to float32.  Asynchronous.
 * pts_rgb_of           the colour channels of an RGBS image (16-byte aligned) into H x W x 3.
 */
pts_status pts_scale_map(int h, int w, double slant_deg, double tilt_deg, double *S_out, void *stream);
pts_status pts_scale_resample(const double *S, int He, int We, int Ho, int Wo, double *S_out, void *stream);
pts_status pts_scale_guided_init(const float *exemplar, const double *S_z, int He, int We, const double *S_x,
                                 const double *u, int Ho, int Wo, int nbins, float *out, int32_t *src_out,
                                 void *stream);
pts_status pts_rgbs(const float *rgb, const double *S, double lam, int H, int W, float *out, void *stream);
pts_status pts_rgb_of(const float *rgbs, int H, int W, float *rgb_out, void *stream);

/*
 * Pyramid filters for coarse-to-fine synthesis (section 2.1: a coarse result
 * is up-sampled by interpolation to initialise the next level).  The paper
 * names no filter; the library uses
 *   pts_downsample2: separable binomial [1 4 6 4 1]/16, mirrored border
 *                    (index -1 -> 1, H -> H-2), even samples kept:
 *                    out is ((H+1)/2) x ((W+1)/2) x 3;
 *   pts_upsample2:   bilinear x2, half-pixel centres, clamped: out is 2H x 2W x 3.
 * Device pointers; asynchronous.
 */
pts_status pts_downsample2(const float *in, int H, int W, float *out, void *stream);
pts_status pts_upsample2(const float *in, int H, int W, float *out, void *stream);

/*
 * Measurement support (no counterpart in the paper).  The library counts
 * every kernel it launches, and while profiling is on it brackets each launch
 * of the named kernel classes with CUDA events recorded on the launch stream.
 *   pts_launch_count     kernels launched by this process so far.
 *   pts_profile_enable   on != 0 starts recording (and clears old records).
 *   pts_profile_read     total device milliseconds and launch count of one
 *                        kernel class ("search_topk", "search_full",
 *                        "rerank", "project", "m_step", "brute", "irls",
 *                        "search_tc", "search_tc_list" (tensor-core
 *                        searches of a device query list), "mlp",
 *                        "probe"); synchronises on the
 *                        recorded events.  Returns INVALID_ARG for an unknown
 *                        name.
 */
long long pts_launch_count(void);

/*
 * Batched synthesis (no counterpart in the paper; the batched form of the EM loop of section 2.1
 * for many independent jobs of uneven sizes).  A job is one level: `iters` EM iterations on its
 * own index and output, then the final search phase.  Jobs can be chained into pyramids
 * (section 2.1's coarse to fine): a job whose `parent` is an earlier job of the batch starts each
 * run from that job's result up-sampled by 2 (pts_upsample2), after the parent has finished.
 */
typedef struct {
    pts_index index;  /* the job's exemplar index; no two jobs of a batch may share one */
    float *output;    /* device Ho x Wo x C float32 (C the index's channels); in: initial image,
                         out: result */
    int Ho, Wo, stride;
    int mode;         /* PTS_EXACT_F32, PTS_F16_RERANK, PTS_FP8_RERANK, PTS_PROPOSAL (the index
                         has a trained proposal) or PTS_KMTREE (the index has a built tree) */
    double *energy;   /* device, iters + 1 doubles: energy entering each iteration, then the final */
    int parent;       /* -1: the run starts from `output` as the caller left it; k >= 0 (an
                         earlier job, RGB indices, the parent's output exactly half this job's
                         Ho and Wo): the run starts from job k's result up-sampled by 2 */
} pts_job;

typedef struct pts_batch_s *pts_batch; /* opaque, owned by the library */

/* Builds a batch: runs one search per job (sizing every workspace), with tune != 0 picks the
 * tensor-core search's exemplar split per job shape by timing the candidates (cached per
 * process), then captures all jobs' iterations into one CUDA graph, jobs spread round-robin
 * over n_streams (1..64) forked streams.  The job structs are copied; outputs and energy arrays
 * stay the caller's.  Synchronises `stream`.  Jobs' outputs are searched (not modified) here.
 * Each index's own exemplar split (pts_index_set_tc_parts) is left as the caller had it.
 * Lifetime: the graph holds raw device pointers into every job's index (its tables and the
 * workspace its searches use), its output and its energy array.  Keep them all alive and do not
 * move them while the batch may run: a search on a job's index that needs larger or other
 * buffers (a bigger output, another mode, a trained proposal) reallocates them, and after that,
 * or after pts_index_destroy of a job's index, pts_batch_run returns PTS_ERR_INVALID_ARG; create
 * the batch again.  Outputs and energy arrays are the caller's to keep in place. */
pts_status pts_batch_create(const pts_job *jobs, int n_jobs, int iters, float r, float delta, int n_streams,
                            int tune, void *stream, pts_batch *out);
/* Replays the batch's graph on `stream` (asynchronous): every job runs from its current output.
 * PTS_ERR_INVALID_ARG, with nothing launched, if a job's index was destroyed or had buffers
 * reallocated since pts_batch_create (see above). */
pts_status pts_batch_run(pts_batch batch, void *stream);
/* The one-call form: pts_batch_create (8 streams at most, autotuned), one pts_batch_run,
 * pts_batch_destroy.  Synchronises `stream`; returns the first error of the three, else the
 * first job whose index reports a device-side error (PTS_ERR_DEVICE / PTS_ERR_TIMEOUT).  For
 * repeated runs of the same jobs keep the batch instead: building it costs a sizing search per
 * job and a graph capture. */
pts_status synthesize_batched(const pts_job *jobs, int n_jobs, int iters, float r, float delta, void *stream);
/* Kernel launches one run issues, and (parts_out, n_jobs ints, may be NULL) each job's exemplar
 * split chosen by the autotuner (0 for exact jobs). */
pts_status pts_batch_info(pts_batch batch, long long *launches_per_run, int *parts_out);
void pts_batch_destroy(pts_batch batch);

/* Self-test of the tensor-core operand layout (no counterpart in the paper):
 * one 128 x N x K tcgen05 MMA (f16 == 3: FP8 E4M3, kind::f8f6f4, K a multiple of 32;
 * f16 == 2: FP16 with the A operand read from tensor memory; f16 == 1: FP16 with both
 * operands in shared memory, as in the search; f16 == 0: BF16 as in the proposal
 * network) through the same shared-memory
 * and instruction descriptors the kernels use, on seeded data generated here,
 * compared with an FP64 host product.  N, K multiples of 16 (N <= 256,
 * K <= 128).  Writes the largest absolute error and the largest |reference|.
 * Synchronises the device. */
pts_status pts_tc_selftest(int N, int K, int f16, double *max_abs_err, double *max_abs_ref);

/* Self-test of the bounded device waits (no counterpart in the paper).  One thread waits on a
 * new mbarrier phase with the library's bounded wait (abortable != 0: the variant that also
 * raises an abort flag for the kernel's other roles).  With arrive != 0 the phase completes:
 * PTS_OK and *completed_out = 1.  With arrive == 0 nothing completes it: the wait gives up after
 * about one second, the kernel returns, and the call returns PTS_ERR_TIMEOUT with
 * *completed_out = 0 (PTS_ERR_DEVICE if the abortable wait did not raise its flag).  The context
 * stays usable.  Synchronises the device. */
pts_status pts_wait_selftest(int arrive, int abortable, int *completed_out);
void pts_profile_enable(int on);
pts_status pts_profile_read(const char *kernel, double *total_ms, long long *launches);

/* FP32 FMA throughput of this GPU (no counterpart in the paper; the denominator of the
 * exact-mode rooflines, whose kernels run on the FP32 SIMT pipe).  A grid of 2 CTAs x 1024
 * threads per SM, each thread running 8 independent FMA chains for `iters` x 128 FMAs
 * (iters in 1..10^6), is timed with CUDA events on `stream` `reps` times (1..100); writes the
 * best rate in TFLOP/s (2 flops per FMA) and its milliseconds.  Synchronises `stream`. */
pts_status pts_fp32_fma_peak(int iters, int reps, void *stream, double *tflops, double *best_ms);

#ifdef __cplusplus
}
#endif

#endif /* PTS_H */
