// search_f32.cu -- exact-mode search phase (E-step, Eq. 4) on FP32 SIMT cores.
//
// Pass 1 (k_search_pca), PCA space.  Every exemplar window n carries
// e_n = (y_n, r_n) (PCA coordinates and residual norm, section 2.2) and
// ||u_n||^2 = ||v_n - mu||^2; every query q carries a_q = (y_q, r_q) and
// ||u_q||^2.  For an orthonormal basis
//   LB(q, n) = ||y_q - y_n||^2 + (r_q - r_n)^2
//            = ||u_q||^2 + ||u_n||^2 - 2 a_q . e_n  <=  ||x_q - z_n||^2,
// a lower bound on the full-dimension distance of Eq. 4.  The exemplar side
// is stored pre-multiplied by -2, so one FMA chain from ||u_n||^2 gives
// p(q, n) = LB(q, n) - ||u_q||^2.
//
// Pass 2 (k_search_full), full dimension, only for the queries whose pass-1
// result could not be certified: the same GEMM + top-32 on the centred
// window vectors u themselves (D = 3 w^2 terms), i.e. the expanded form of
// ||u_q - u_n||^2, fed K-chunk by K-chunk through a 4-stage ring (D padded
// with zero rows to Dp, a multiple of the 32-row chunk).
//
// Both passes: exemplar data in tiles of kBN = 128 windows whose K rows are
// contiguous ([tile][K][128]), copied to shared memory by 1-D bulk copies
// completing on mbarriers.  A CTA owns kBQ = 64 queries (8 warps x 8 rows);
// each lane computes 8 rows x 4 consecutive windows.  Per query a warp keeps
// the 32 smallest (p, n) in lexicographic order, one sorted entry per lane;
// a value enters only when it beats the current 32nd, found with warp
// ballots, so after the first tiles insertions are rare.
#include <float.h>

#include <algorithm>
#include <climits>

#include "pts_internal.cuh"
#include "tc_common.cuh"
#include "warp_keys.cuh"

namespace pts {
namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

// Per-warp top-32 state for 8 query rows (lane L holds entry L, ascending).
struct TopK8 {
    float ld[8];
    int li[8];
    float thr[8];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            ld[i] = INFINITY;
            li[i] = -1;
            thr[i] = INFINITY;
        }
    }
    // offer the 8x4 values of this lane (rows i, windows nbase + j)
    __device__ __forceinline__ void offer(const float (&p)[8][4], int tile_base, int lane) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float m = fminf(fminf(p[i][0], p[i][1]), fminf(p[i][2], p[i][3]));
            if (!__any_sync(kFull, m < thr[i])) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                unsigned fl = __ballot_sync(kFull, p[i][j] < thr[i]);
                while (fl) {
                    const int src = __ffs(fl) - 1;
                    const float cd = __shfl_sync(kFull, p[i][j], src);
                    const int ci = tile_base + src * 4 + j;
                    const bool before = (ld[i] < cd) || (ld[i] == cd && li[i] < ci);
                    const int pos = __popc(__ballot_sync(kFull, before));
                    const float ud = __shfl_up_sync(kFull, ld[i], 1);
                    const int ui = __shfl_up_sync(kFull, li[i], 1);
                    if (lane > pos) {
                        ld[i] = ud;
                        li[i] = ui;
                    } else if (lane == pos) {
                        ld[i] = cd;
                        li[i] = ci;
                    }
                    thr[i] = fminf(thr[i], __shfl_sync(kFull, ld[i], 31));
                    fl &= ~(1u << src);
                    fl &= __ballot_sync(kFull, p[i][j] < thr[i]);
                }
            }
        }
    }
};

// ---------------------------------------------------------------------------
// pass 1: PCA-space lower bounds
// ---------------------------------------------------------------------------
// DAM: the longest search vector the layout holds (68: d <= 64 coordinates + residual; 128:
// the d_fast <= 124 coordinates of the index's larger PCA + residual)
template <int DAM>
struct PcaSmem {
    float a[DAM][kBQ];     // query vectors, transposed
    float e[2][DAM][kBN];  // exemplar tiles (double buffer)
    float en[2][kBN];         // exemplar norms
    uint64_t bar[2];          // tile of buffer b landed
    uint64_t empty[2];        // all 8 warps are done with buffer b
    int abort_flag;
};

template <int DAM>
__global__ void __launch_bounds__(kThreads, DAM <= kMaxDA ? 2 : 1)
    k_search_pca(const float *__restrict__ qcoord, const float *__restrict__ qnorm, int Q, int da, int dk,
                 const float *__restrict__ et, const float *__restrict__ enorm, int ntiles, int tiles_per_part,
                 int *__restrict__ cand_idx, float *__restrict__ cand_lb, float *__restrict__ part_v,
                 int *__restrict__ part_i, int *__restrict__ status, const float *__restrict__ thr_init) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PcaSmem<DAM> &sm = *reinterpret_cast<PcaSmem<DAM> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int qbase = blockIdx.x * kBQ;
    for (int i = tid; i < kBQ * da; i += kThreads) {
        const int r = i / da, k = i - r * da;
        const int q = qbase + r;
        sm.a[k][r] = q < Q ? qcoord[(size_t)q * da + k] : 0.0f;
    }
    const int row0 = warp * 8;
    TopK8 top;
    top.init();
    if (thr_init)  // warm start: a value enters only below the bound (which caps the 32nd best)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int q = qbase + row0 + i;
            top.thr[i] = q < Q ? thr_init[q] : INFINITY;
        }
    const uint32_t tile_floats = static_cast<uint32_t>(da) * kBN;
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        mbar_init(&sm.empty[0], kThreads / 32);
        mbar_init(&sm.empty[1], kThreads / 32);
        fence_mbar_init();
        sm.abort_flag = 0;
    }
    __syncthreads();
    auto issue = [&](int t, int buf) {
        mbar_expect_tx(&sm.bar[buf], tile_floats * 4u + kBN * 4u);
        bulk_g2s(&sm.e[buf][0][0], et + (size_t)t * tile_floats, tile_floats * 4u, &sm.bar[buf]);
        bulk_g2s(&sm.en[buf][0], enorm + (size_t)t * kBN, kBN * 4u, &sm.bar[buf]);
    };
    // this CTA's exemplar tiles (blockIdx.y splits them; the parts' lists are merged afterwards)
    const int t_begin = blockIdx.y * tiles_per_part;
    const int t_end = min(ntiles, t_begin + tiles_per_part);
    const int nt = max(0, t_end - t_begin);
    // No block-wide barrier in the loop: every warp waits for the tile's copy itself and releases
    // the buffer with one arrival; lane 0 of warp 0 refills a buffer once all 8 warps released it.
    // Every wait is bounded; a failed wait aborts the whole CTA (warp-uniform breaks), and thread 0
    // then waits for the last copy issued into each buffer before the CTA exits.
    int last_issued[2] = {-1, -1};  // tile slot i last copied into each buffer (thread 0)
    if (tid == 0) {
        if (nt > 0) {
            issue(t_begin, 0);
            last_issued[0] = 0;
        }
        if (nt > 1) {
            issue(t_begin + 1, 1);
            last_issued[1] = 1;
        }
    }
    for (int i = 0; i < nt; ++i) {
        const int t = t_begin + i;
        const int buf = i & 1;
        const uint32_t par = (uint32_t)((i >> 1) & 1);
        const bool ok = mbar_wait_or_abort(&sm.bar[buf], par, status, &sm.abort_flag);
        if (!__all_sync(kFull, ok)) {
            sm.abort_flag = 1;
            break;
        }
        float acc[8][4];
        const float4 nv = *reinterpret_cast<const float4 *>(&sm.en[buf][lane * 4]);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            acc[i][0] = nv.x;
            acc[i][1] = nv.y;
            acc[i][2] = nv.z;
            acc[i][3] = nv.w;
        }
        const float *eb = &sm.e[buf][0][lane * 4];
#pragma unroll 8
        for (int k = 0; k < dk; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&sm.a[k][row0]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&sm.a[k][row0 + 4]);
            const float4 b = *reinterpret_cast<const float4 *>(eb + k * kBN);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.empty[buf]);  // this warp's last read of `buf` is done
        top.offer(acc, t * kBN, lane);
        if (warp == 0 && i + 2 < nt) {
            bool refilled = false;
            if (lane == 0 && mbar_wait_or_abort(&sm.empty[buf], par, status, &sm.abort_flag)) {
                issue(t + 2, buf);
                last_issued[buf] = i + 2;
                refilled = true;
            }
            if (!__shfl_sync(kFull, refilled, 0)) {
                sm.abort_flag = 1;
                break;
            }
        }
    }
    __syncthreads();
    if (sm.abort_flag) {
        if (tid == 0)
            for (int b = 0; b < 2; ++b)
                if (last_issued[b] >= 0) mbar_wait_bounded(&sm.bar[b], (uint32_t)((last_issued[b] >> 1) & 1), status);
        return;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int q = qbase + row0 + i;
        if (q < Q) {
            if (gridDim.y > 1) {
                const size_t o = ((size_t)q * gridDim.y + blockIdx.y) * kTopK + lane;
                part_v[o] = top.ld[i];
                part_i[o] = top.li[i];
            } else {
                cand_idx[(size_t)q * kTopK + lane] = top.li[i];
                cand_lb[(size_t)q * kTopK + lane] = top.ld[i] + qnorm[q];
            }
        }
    }
}

// Warm start of the exact PCA pass: the previous search's 32 distinct windows of each query scored
// with the current query vector by the pass's own arithmetic (||u_n||^2, then one FMA per
// coordinate in coordinate order, so each value equals the pass's bit for bit).  Their largest is
// at least the 32nd smallest over all windows; with a 2^-20 relative margin it bounds the values
// that can enter the top-32 (the list still fills, ties included).  +inf when a lane has no
// window.  One warp per query.
__global__ void __launch_bounds__(256) k_warm_pca(const int *__restrict__ prev_idx, const float *__restrict__ qcoord,
                                                  int da, const float *__restrict__ et_rows,
                                                  const float *__restrict__ enorm, int Q, int N,
                                                  float *__restrict__ thr) {
    const int lane = threadIdx.x & 31;
    const long q = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    const int n = prev_idx[q * kTopK + lane];
    const bool valid = n >= 0 && n < N;
    float p = INFINITY;
    if (valid) {
        const float *a = qcoord + q * da;
        const float *e = et_rows + (size_t)n * da;
        p = enorm[n];
        for (int k = 0; k < da; k += 4) {  // da is a multiple of 4
            const float4 av = __ldg(reinterpret_cast<const float4 *>(a + k));
            const float4 ev = __ldg(reinterpret_cast<const float4 *>(e + k));
            p = fmaf(av.x, ev.x, p);
            p = fmaf(av.y, ev.y, p);
            p = fmaf(av.z, ev.z, p);
            p = fmaf(av.w, ev.w, p);
        }
    }
    float m = p;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, s));
    if (lane == 0) thr[q] = isinf(m) ? INFINITY : m + fmaxf(fabsf(m), 1e-30f) * 9.5367431640625e-7f;
}

// [ntiles][da][128] -> [N][da]
__global__ void k_tiles_to_rows(const float *__restrict__ et, int N, int da, float *__restrict__ rows) {
    const long total = (long)N * da;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int n = (int)(i / da), k = (int)(i - (long)n * da);
        rows[i] = et[((size_t)(n / kBN) * da + k) * kBN + n % kBN];
    }
}

// One warp per query: the 32 smallest (p, n) of its nparts sorted part lists (missing entries
// are (+inf, -1) and sort last), + ||u_q||^2.
__global__ void __launch_bounds__(256) k_merge_pca_parts(const float *__restrict__ part_v,
                                                         const int *__restrict__ part_i, int nparts, int Q,
                                                         const float *__restrict__ qnorm, int *__restrict__ cand_idx,
                                                         float *__restrict__ cand_lb) {
    const int lane = threadIdx.x & 31;
    const long q = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    const size_t base = (size_t)q * nparts * kTopK;
    unsigned long long k = pack_key(part_v[base + lane], part_i[base + lane]);
    for (int p = 1; p < nparts; ++p)
        warp_merge_keys(k, pack_key(part_v[base + (size_t)p * kTopK + lane], part_i[base + (size_t)p * kTopK + lane]),
                        lane);
    const float v = key_value(k);
    cand_idx[(size_t)q * kTopK + lane] = v < INFINITY ? key_index(k) : -1;
    cand_lb[(size_t)q * kTopK + lane] = v + qnorm[q];
}

// ---------------------------------------------------------------------------
// pass 2: full dimension for the uncertified queries
// ---------------------------------------------------------------------------
constexpr int kKC = 32;     // K rows per chunk
constexpr int kStages = 4;  // ring depth

constexpr int kItemOverheadTiles = 4;

// Exemplar parts of an adaptive full pass with nf listed queries: the part count p (at most
// kMaxAdaptiveParts, parts of at least 4 tiles, nf * p part records at most kPartRows) whose
// (query block, part) items finish soonest on the fixed grid of kAdaptiveGrid CTAs, counted as
// rounds of the grid times the tiles of a part plus kItemOverheadTiles for the item's own costs
// (its query tile, the ring's fill, its records and their merge); the smaller p on a tie.  The pass and its merge
// take the same value from the same device count.
__device__ __forceinline__ int adaptive_parts(int nf, int ntiles) {
    const int nqb = (nf + kBQ - 1) / kBQ;
    if (nqb <= 0) return 1;
    const int pmax = max(1, min(min(kMaxAdaptiveParts, ntiles / 4), kPartRows / max(nf, 1)));
    int best = 1;
    long best_cost = LONG_MAX;
    for (int p = 1; p <= pmax; ++p) {
        const int tpp = (ntiles + p - 1) / p;
        const int np = (ntiles + tpp - 1) / tpp;
        const long cost = ((long)nqb * np + kAdaptiveGrid - 1) / kAdaptiveGrid * (tpp + kItemOverheadTiles);
        if (cost < best_cost) {
            best_cost = cost;
            best = np;
        }
    }
    return best;
}

struct FullSmem {
    float a[kStages][kKC][kBQ];
    float e[kStages][kKC][kBN];
    uint64_t bar[kStages];    // chunk of stage s landed
    uint64_t empty[kStages];  // all 8 warps are done with stage s
    int abort_flag;
};

__global__ void __launch_bounds__(kThreads, 2)
    k_search_full(const float *__restrict__ qfull,  // [F/64][D][64]: u_q of failing queries
                  const int *__restrict__ fail_list, const unsigned int *__restrict__ fail_count,
                  int Q, int Dp, const float *__restrict__ efull,  // [ntiles][Dp][128] = -2 u_n
                  const float *__restrict__ enorm, int ntiles, int tiles_per_part,
                  const float *__restrict__ qnorm, int *__restrict__ cand_idx, float *__restrict__ cand_lb,
                  float *__restrict__ part_v, int *__restrict__ part_i, int *__restrict__ status,
                  int kc_split, float *__restrict__ pdist, int adaptive, int kvalid) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FullSmem &sm = *reinterpret_cast<FullSmem *>(smem_raw);
    const int nf = static_cast<int>(*fail_count);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row0 = warp * 8;
    // Work items (query block, exemplar part).  Fixed grids: blockIdx.x is the block, blockIdx.y
    // the part.  Adaptive grids (a fixed number of CTAs, whatever the device-side count of listed
    // queries): the part count follows that count (adaptive_parts), and each CTA takes items
    // blockIdx.x, blockIdx.x + gridDim.x, ...
    int nparts = gridDim.y, tpp = tiles_per_part;
    int item = 0, nitems = 1, step = 1;
    if (adaptive) {
        nparts = adaptive_parts(nf, ntiles);
        tpp = (ntiles + nparts - 1) / nparts;
        nitems = (nf + kBQ - 1) / kBQ * nparts;
        item = blockIdx.x;
        step = gridDim.x;
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sm.bar[s], 1);
            mbar_init(&sm.empty[s], kThreads / 32);
        }
        fence_mbar_init();
        sm.abort_flag = 0;
    }
    __syncthreads();
    // Stages and barrier phases follow one running chunk count g0 + it over all of this CTA's
    // items, so the barriers are initialised once.  Every copy of an item is consumed before its
    // closing block barrier, so the next item fills its first stages without waiting.
    long g0 = 0;
    for (; item < nitems; item += step) {
    const int qb = adaptive ? item / nparts : (int)blockIdx.x;
    const int part = adaptive ? item % nparts : (int)blockIdx.y;
    const int fbase = qb * kBQ;
    if (fbase >= nf) return;  // uniform for the CTA
    // this item's exemplar tiles (parts are merged afterwards) and chunks of the vector
    // (blockIdx.z splits them when pdist is given: partial sums, summed afterwards)
    const int c0 = blockIdx.z * kc_split, c1 = min(Dp / kKC, c0 + kc_split);
    const int nchunks = c1 - c0;
    const int t_begin = part * tpp;
    const int nt = max(0, min(ntiles, t_begin + tpp) - t_begin);
    const long total = (long)nt * nchunks;
    const float *qa = qfull + (size_t)qb * Dp * kBQ;
    TopK8 top;
    top.init();
    auto issue = [&](int s, int t, int c) {
        mbar_expect_tx(&sm.bar[s], (uint32_t)(kKC * (kBQ + kBN) * 4));
        bulk_g2s(&sm.a[s][0][0], qa + (size_t)c * kKC * kBQ, kKC * kBQ * 4u, &sm.bar[s]);
        bulk_g2s(&sm.e[s][0][0], efull + ((size_t)(t_begin + t) * Dp + (size_t)c * kKC) * kBN, kKC * kBN * 4u,
                 &sm.bar[s]);
    };
    // As in k_search_pca: no block-wide barrier in the loop; every warp waits for a chunk itself
    // and releases its stage with one arrival, lane 0 of warp 0 refills a stage once all 8 warps
    // released it; bounded waits, warp-uniform aborts, and on abort thread 0 waits for the last
    // copy issued into each stage before the CTA exits.
    long last_issued[kStages];
#pragma unroll
    for (int s = 0; s < kStages; ++s) last_issued[s] = -1;
    if (tid == 0)
        for (long it = 0; it < kStages && it < total; ++it) {
            const int t = (int)(it / nchunks);
            issue((int)((g0 + it) % kStages), t, c0 + (int)(it - (long)t * nchunks));
            last_issued[(g0 + it) % kStages] = g0 + it;
        }
    // stage, phase, tile and chunk of the current chunk and of the next one to copy, advanced
    // one chunk at a time (no division in the loop)
    int s = (int)(g0 % kStages), t = 0, c = c0;
    uint32_t par = (uint32_t)((g0 / kStages) & 1);
    int nx_t = kStages / nchunks, nx_c = c0 + kStages % nchunks;
    float acc[8][4];
    for (long it = 0; it < total; ++it) {
        if (c == c0) {
            const float4 nv = blockIdx.z == 0
                                  ? __ldg(reinterpret_cast<const float4 *>(enorm + (t_begin + t) * kBN + lane * 4))
                                  : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc[i][0] = nv.x;
                acc[i][1] = nv.y;
                acc[i][2] = nv.z;
                acc[i][3] = nv.w;
            }
        }
        const bool ok = mbar_wait_or_abort(&sm.bar[s], par, status, &sm.abort_flag);
        if (!__all_sync(kFull, ok)) {
            sm.abort_flag = 1;
            break;
        }
        const float *eb = &sm.e[s][0][lane * 4];
        auto step = [&](int k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&sm.a[s][k][row0]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&sm.a[s][k][row0 + 4]);
            const float4 b = *reinterpret_cast<const float4 *>(eb + k * kBN);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        };
        // the rows past the vector's kvalid components are zero on both sides and are skipped
        // (adding 0 x 0 leaves every sum as it is)
        const int klen = min(kKC, kvalid - c * kKC);
        if (klen == kKC) {
#pragma unroll 4
            for (int k = 0; k < kKC; ++k) step(k);
        } else {
#pragma unroll 4
            for (int k = 0; k < klen; ++k) step(k);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.empty[s]);  // this warp's last read of stage s is done
        if (c == c1 - 1) {
            if (pdist) {  // partial sums of this chunk range: [z][f][tile * 128 + window]
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int f = fbase + row0 + i;
                    if (f < nf)
                        *reinterpret_cast<float4 *>(pdist + ((size_t)blockIdx.z * Q + f) * ((size_t)ntiles * kBN) +
                                                    (size_t)(t_begin + t) * kBN + lane * 4) =
                            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                }
            } else {
                top.offer(acc, (int)(t_begin + t) * kBN, lane);
            }
        }
        if (warp == 0 && it + kStages < total) {
            bool refilled = false;
            if (lane == 0 && mbar_wait_or_abort(&sm.empty[s], par, status, &sm.abort_flag)) {
                issue(s, nx_t, nx_c);
                last_issued[s] = g0 + it + kStages;
                refilled = true;
            }
            if (!__shfl_sync(kFull, refilled, 0)) {
                sm.abort_flag = 1;
                break;
            }
            if (++nx_c == c1) {
                nx_c = c0;
                ++nx_t;
            }
        }
        if (++c == c1) {
            c = c0;
            ++t;
        }
        if (++s == kStages) {
            s = 0;
            par ^= 1u;
        }
    }
    __syncthreads();
    if (sm.abort_flag) {
        if (tid == 0)
            for (int b = 0; b < kStages; ++b)
                if (last_issued[b] >= 0)
                    mbar_wait_bounded(&sm.bar[b], (uint32_t)((last_issued[b] / kStages) & 1), status);
        return;
    }
    if (pdist) return;
    g0 += total;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int f = fbase + row0 + i;
        if (f < nf) {
            if (nparts > 1) {
                const size_t o = ((size_t)f * nparts + part) * kTopK + lane;
                part_v[o] = top.ld[i];
                part_i[o] = top.li[i];
                continue;
            }
            const int q = fail_list[f];
            if (q >= 0 && q < Q) {
                cand_idx[(size_t)q * kTopK + lane] = top.li[i];
                cand_lb[(size_t)q * kTopK + lane] = top.ld[i] + qnorm[q];
            } else if (lane == 0) {
                atomicOr(status, kDevErrBounds);
            }
        }
    }
    __syncthreads();  // every warp is done with the stages before the next item re-arms them
    }
}

// (a, ia) < (b, ib) lexicographically; window -1 (no window) only ever pairs with +inf
__device__ __forceinline__ bool lex_less_f(float a, int ia, float b, int ib) {
    return (a < b) || (a == b && ia < ib);
}

// One warp per listed query: the 32 smallest (p, n) over the parts' sorted lists (the elementwise
// minimum of a list and another reversed is bitonic; five stages sort it).
__global__ void k_merge_fail_parts(const float *__restrict__ part_v, const int *__restrict__ part_i, int ntiles,
                                   const int *__restrict__ fail_list, const unsigned int *__restrict__ fail_count,
                                   int Q, const float *__restrict__ qnorm, int *__restrict__ cand_idx,
                                   float *__restrict__ cand_lb, int *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nf = (int)*fail_count;
    if (f >= nf) return;
    const int nparts = adaptive_parts(nf, ntiles);
    if (nparts == 1) return;  // the pass wrote the candidates itself
    const size_t base = (size_t)f * nparts * kTopK;
    float v = part_v[base + lane];
    int i = part_i[base + lane];
    for (int p = 1; p < nparts; ++p) {
        const float w = __shfl_sync(kFull, part_v[base + (size_t)p * kTopK + lane], 31 - lane);
        const int j = __shfl_sync(kFull, part_i[base + (size_t)p * kTopK + lane], 31 - lane);
        if (lex_less_f(w, j, v, i)) {
            v = w;
            i = j;
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            const float ov = __shfl_xor_sync(kFull, v, s);
            const int oi = __shfl_xor_sync(kFull, i, s);
            const bool take = ((lane & s) == 0) ? lex_less_f(ov, oi, v, i) : lex_less_f(v, i, ov, oi);
            if (take) {
                v = ov;
                i = oi;
            }
        }
    }
    const int q = fail_list[f];
    if (q >= 0 && q < Q) {
        cand_idx[(size_t)q * kTopK + lane] = i;
        cand_lb[(size_t)q * kTopK + lane] = v + qnorm[q];
    } else if (lane == 0) {
        atomicOr(status, kDevErrBounds);
    }
}

// One warp per listed query of a pass split along the vector: the nsplit partial sums of each
// window added in split order, then the 32 smallest (p, n) kept by sorting each 32 windows and
// merging them into the running list (skipped when none beats its 32nd).  Padding windows
// (n >= N, p = +inf) never enter.
constexpr int kSelCap = 128;  // keys a warp collects at or below its threshold (full_select_row)

// The 32 smallest (score, window) pairs of one query, one warp: score n = sum over the splits of
// row[split * split_stride + n] for n < N (NaN and +inf skipped), sorted; to the candidate lists
// with ||u_q||^2 added.  Lane l reads windows 4l .. 4l + 3, 4l + 128 ... (npad is a multiple of
// 128 and the rows 16-byte aligned).  A first
// pass keeps each lane's two smallest scores; the 32nd smallest T of those 64 values bounds the
// 32nd smallest score from above (at least 32 scores are <= T), so a second pass collects the
// scores <= T into buf (kSelCap keys of this warp) and sorts only those.  When more than kSelCap
// scores lie at or below T (many ties), the warp sorts every score chunk by chunk instead.  The
// result is the same either way: the 32 smallest (score, window) keys.
__device__ __forceinline__ void full_select_row(const float *__restrict__ row, size_t split_stride, int nsplit,
                                                int npad, int N, int q, int Q, const float *__restrict__ qnorm,
                                                int *__restrict__ cand_idx, float *__restrict__ cand_lb,
                                                int *__restrict__ status, int lane, unsigned long long *buf) {
    const unsigned long long kNone = pack_key(INFINITY, INT_MAX);
    auto score = [&](int n) -> float {
        float v = 0.0f;
        for (int sp = 0; sp < nsplit; ++sp) v += row[(size_t)sp * split_stride + n];
        return (n < N && v < INFINITY) ? v : INFINITY;  // NaN fails the test too
    };
    // four consecutive scores per lane and load (npad is a multiple of 128, rows 16-byte aligned)
    auto score4 = [&](int n) -> float4 {
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int sp = 0; sp < nsplit; ++sp) {
            const float4 t = *reinterpret_cast<const float4 *>(row + (size_t)sp * split_stride + n);
            v.x += t.x;
            v.y += t.y;
            v.z += t.z;
            v.w += t.w;
        }
        v.x = (n < N && v.x < INFINITY) ? v.x : INFINITY;
        v.y = (n + 1 < N && v.y < INFINITY) ? v.y : INFINITY;
        v.z = (n + 2 < N && v.z < INFINITY) ? v.z : INFINITY;
        v.w = (n + 3 < N && v.w < INFINITY) ? v.w : INFINITY;
        return v;
    };
    float m1 = INFINITY, m2 = INFINITY;
    for (int n0 = 0; n0 < npad; n0 += 128) {
        const float4 v4 = score4(n0 + 4 * lane);
        const float vs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            m2 = fminf(m2, fmaxf(m1, vs[c]));
            m1 = fminf(m1, vs[c]);
        }
    }
    unsigned long long a = pack_key(m1, lane), b = pack_key(m2, 32 + lane);
    warp_sort_keys(a, lane);
    warp_sort_keys(b, lane);
    warp_merge_keys(a, b, lane);
    const float T = key_value(__shfl_sync(kFull, a, 31));
    int cnt = 0;  // warp-uniform
    for (int n0 = 0; n0 < npad; n0 += 128) {
        const float4 v4 = score4(n0 + 4 * lane);
        const float vs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const bool take = vs[c] < INFINITY && vs[c] <= T;
            const unsigned m = __ballot_sync(kFull, take);
            const int pos = cnt + __popc(m & ((1u << lane) - 1u));
            if (take && pos < kSelCap) buf[pos] = pack_key(vs[c], n0 + 4 * lane + c);
            cnt += __popc(m);
        }
    }
    __syncwarp();
    unsigned long long best = kNone;
    if (cnt <= kSelCap) {
        for (int g = 0; g < cnt; g += 32) {
            unsigned long long k = g + lane < cnt ? buf[g + lane] : kNone;
            warp_sort_keys(k, lane);
            if (g == 0)
                best = k;
            else
                warp_merge_keys(best, k, lane);
        }
    } else {
        for (int n0 = 0; n0 < npad; n0 += 32) {
            const float v = score(n0 + lane);
            unsigned long long k = v < INFINITY ? pack_key(v, n0 + lane) : kNone;
            if (!__any_sync(kFull, k < __shfl_sync(kFull, best, 31))) continue;
            warp_sort_keys(k, lane);
            warp_merge_keys(best, k, lane);
        }
    }
    __syncwarp();
    const int i = key_index(best);
    const bool real = i != INT_MAX;
    if (q >= 0 && q < Q) {
        cand_idx[(size_t)q * kTopK + lane] = real ? i : -1;
        cand_lb[(size_t)q * kTopK + lane] = real ? key_value(best) + qnorm[q] : INFINITY;
    } else if (lane == 0) {
        atomicOr(status, kDevErrBounds);
    }
}

// listed queries: row f of pdist [split][Q][npad] belongs to query fail_list[f]
__global__ void __launch_bounds__(256) k_full_select(const float *__restrict__ pdist, int nsplit, int npad, int N,
                                                     const int *__restrict__ fail_list,
                                                     const unsigned int *__restrict__ fail_count, int Q,
                                                     const float *__restrict__ qnorm, int *__restrict__ cand_idx,
                                                     float *__restrict__ cand_lb, int *__restrict__ status) {
    __shared__ unsigned long long buf[256 / 32][kSelCap];
    const int lane = threadIdx.x & 31;
    const long f = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (f >= (long)*fail_count) return;
    full_select_row(pdist + (size_t)f * npad, (size_t)Q * npad, nsplit, npad, N, fail_list[f], Q, qnorm, cand_idx,
                    cand_lb, status, lane, buf[threadIdx.x >> 5]);
}

// a range of queries: row f of score [nsplit][nq][npad] belongs to query q0 + f
__global__ void __launch_bounds__(256) k_full_select_range(const float *__restrict__ score, int nsplit, int npad,
                                                           int N, int q0, int nq, int Q,
                                                           const float *__restrict__ qnorm,
                                                           int *__restrict__ cand_idx, float *__restrict__ cand_lb,
                                                           int *__restrict__ status) {
    __shared__ unsigned long long buf[256 / 32][kSelCap];
    const int lane = threadIdx.x & 31;
    const long f = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (f >= nq) return;
    full_select_row(score + (size_t)f * npad, (size_t)nq * npad, nsplit, npad, N, q0 + (int)f, Q, qnorm, cand_idx,
                    cand_lb, status, lane, buf[threadIdx.x >> 5]);
}

// u_q = x_q - mu of the failing queries, tiled [F/64][Dp][64], zero rows k >= D
__global__ void k_gather_full(const float *__restrict__ X, int Wo, int C, int w, int stride, int qx,
                              const float *__restrict__ mu, const int *__restrict__ fail_list,
                              const unsigned int *__restrict__ fail_count, int Q, int Dp,
                              float *__restrict__ qfull) {
    const int row = C * w, D = row * w;
    const long n = (long)(*fail_count) * Dp;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int f = (int)(i / Dp), k = (int)(i - (long)f * Dp);
        float v = 0.0f;
        if (k < D) {
            int q = fail_list[f];
            q = q < 0 ? 0 : (q >= Q ? Q - 1 : q);
            const int y0 = (q / qx) * stride, x0 = (q % qx) * stride;
            const int dy = k / row, e = k - dy * row;
            v = X[((size_t)(y0 + dy) * Wo + x0) * C + e] - mu[k];
        }
        qfull[((size_t)(f / kBQ) * Dp + k) * kBQ + (f % kBQ)] = v;
    }
}

// -2 u_n of every exemplar window, tiled [ntiles][Dp][128] (the caller zeroes
// the buffer first, so padding rows and columns stay 0)
__global__ void k_exemplar_full(const float *__restrict__ Z, int We, int C, int w, int ex, int N, int Dp,
                                const float *__restrict__ mu, float *__restrict__ efull) {
    const int row = C * w, D = row * w;
    const long n = (long)N * D;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int win = (int)(i / D), k = (int)(i - (long)win * D);
        const int ey = win / ex, exx = win - ey * ex;
        const int dy = k / row, e = k - dy * row;
        efull[((size_t)(win / kBN) * Dp + k) * kBN + (win % kBN)] =
            -2.0f * (Z[((size_t)(ey + dy) * We + exx) * C + e] - mu[k]);
    }
}

// Rows of listed queries (row q of rows, da floats) as the pass's query tiles [F/64][Dp][64],
// zero past da: the second, larger PCA bound of the exact search runs through k_search_full on
// these instead of full window vectors.
__global__ void k_gather_rows(const float *__restrict__ rows, int da, const int *__restrict__ list,
                              const unsigned int *__restrict__ count, int Q, int Dp, float *__restrict__ out) {
    const long n = (long)(*count) * Dp;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int f = (int)(i / Dp), k = (int)(i - (long)f * Dp);
        float v = 0.0f;
        if (k < da) {
            int q = list[f];
            q = q < 0 ? 0 : (q >= Q ? Q - 1 : q);
            v = rows[(size_t)q * da + k];
        }
        out[((size_t)(f / kBQ) * Dp + k) * kBQ + (f % kBQ)] = v;
    }
}

}  // namespace

void launch_tiles_to_rows(const float *et, int N, int da, float *rows, cudaStream_t st) {
    count_launches(1);
    k_tiles_to_rows<<<152 * 4, 256, 0, st>>>(et, N, da, rows);
}

void launch_warm_pca(const int *prev_idx, const float *qcoord, int da, const float *et_rows, const float *enorm, int Q,
                     int N, float *thr, cudaStream_t st) {
    if (Q <= 0) return;
    count_launches(1);
    k_warm_pca<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(prev_idx, qcoord, da, et_rows, enorm, Q, N, thr);
}

// Exemplar parts of the PCA pass: only a grid of fewer query blocks than SMs is split (to about
// two CTAs per SM, at least 8 tiles a part).  Larger grids stay whole: every part restarts its
// top-32 from empty, and on the 64,009-query fine level a 3-way split measured slower.
int pca_parts(int Q, int ntiles) {
    const long nqb = ceil_div(Q, kBQ);
    if (nqb >= 152) return 1;
    int p = (int)std::min<long>(8, ceil_div(2L * 152, std::max(nqb, 1L)));
    while (p > 1 && ntiles / p < 8) --p;
    return p;
}

void launch_search_topk(const float *qcoord, const float *qnorm, int Q, int da, int dk, const float *et,
                        const float *enorm, int ntiles, int *cand_idx, float *cand_lb, int *status,
                        cudaStream_t st, int nparts, float *part_v, int *part_i, const float *thr_init) {
    const bool wide = da > kMaxDA;
    const size_t smem = wide ? sizeof(PcaSmem<kMaxDAFast>) : sizeof(PcaSmem<kMaxDA>);
    set_smem_attr(reinterpret_cast<const void *>(k_search_pca<kMaxDA>), (int)sizeof(PcaSmem<kMaxDA>));
    set_smem_attr(reinterpret_cast<const void *>(k_search_pca<kMaxDAFast>), (int)sizeof(PcaSmem<kMaxDAFast>));
    const int grid = ceil_div(Q, kBQ);
    if (grid == 0) return;
    if (!part_v || !part_i) nparts = 1;
    const int tpp = ceil_div(ntiles, std::max(nparts, 1));
    const int np = ceil_div(ntiles, tpp);
    ProfScope ps(kProfSearchTopk, st, np > 1 ? 2 : 1);
    if (wide)
        k_search_pca<kMaxDAFast><<<dim3(grid, np), kThreads, smem, st>>>(
            qcoord, qnorm, Q, da, dk, et, enorm, ntiles, tpp, cand_idx, cand_lb, part_v, part_i, status, thr_init);
    else
        k_search_pca<kMaxDA><<<dim3(grid, np), kThreads, smem, st>>>(
            qcoord, qnorm, Q, da, dk, et, enorm, ntiles, tpp, cand_idx, cand_lb, part_v, part_i, status, thr_init);
    if (np > 1)
        k_merge_pca_parts<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(part_v, part_i, np, Q, qnorm, cand_idx,
                                                                       cand_lb);
}

// The full-dimension pass over the listed queries (count on the device): a fixed grid of two
// CTAs per SM takes the (query block, exemplar part) items, the part count set on the device from
// the count (adaptive_parts), then the part lists are merged (the merge returns at once when
// there is one part).  part_v / part_i hold full_part_capacity(Q) entries.
static void launch_full_adaptive(const float *qtiles, const int *list, const unsigned int *count, int Q, int Dp,
                                 int kvalid, const float *etiles, const float *enorm, int ntiles, const float *qnorm,
                                 int *cand_idx, float *cand_lb, float *part_v, int *part_i, int *status,
                                 cudaStream_t st) {
    if (Q <= 0) return;
    const int grid = (int)std::min<long>((long)ceil_div((long)Q, kBQ) * kMaxAdaptiveParts, kAdaptiveGrid);
    k_search_full<<<grid, kThreads, sizeof(FullSmem), st>>>(qtiles, list, count, Q, Dp, etiles, enorm, ntiles, 0,
                                                            qnorm, cand_idx, cand_lb, part_v, part_i, status,
                                                            Dp / kKC, nullptr, 1, kvalid);
    k_merge_fail_parts<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(
        part_v, part_i, ntiles, list, count, Q, qnorm, cand_idx, cand_lb, status);
}

int launch_search_full(const float *X, int Wo, int C, int w, int stride, int qx, const float *mu,
                        const int *fail_list, const unsigned int *fail_count, int Q,
                        float *qfull, const float *efull, const float *enorm, int ntiles,
                        const float *qnorm, int *cand_idx, float *cand_lb, float *part_v, int *part_i,
                        int *status, cudaStream_t st, int N, DevBuf<float> *pdist) {
    const size_t smem = sizeof(FullSmem);
    set_smem_attr(reinterpret_cast<const void *>(k_search_full), (int)smem);
    const int Dp = padded_dim(C * w * w);
    count_launches(1);
    k_gather_full<<<152 * 4, 256, 0, st>>>(X, Wo, C, w, stride, qx, mu, fail_list, fail_count, Q, Dp,
                                           qfull);
    // A grid of few (query block, tile) pairs with long vectors (the coarse levels, where every
    // query takes this pass) is split along the vector as well, for about four CTAs per slot,
    // each split at least four chunks long and the partial sums at most 256 MB.
    const int nqb = ceil_div(Q, kBQ), nchunks = Dp / kKC;
    const size_t npad = (size_t)ntiles * kBN;
    int nsplit = 1;
    if (pdist && (long)nqb * ntiles < 4L * 2 * 152) {
        nsplit = std::min<long>(nchunks / 4, ceil_div(4L * 2 * 152, (long)nqb * ntiles));
        while (nsplit > 1 && (size_t)nsplit * Q * npad * sizeof(float) > (256u << 20)) --nsplit;
        if (nsplit > 1 && pdist->ensure((size_t)nsplit * Q * npad, "full-pass partial sums") != PTS_OK) nsplit = 1;
    }
    if (nsplit > 1) {
        const int kcs = ceil_div(nchunks, nsplit);
        nsplit = ceil_div(nchunks, kcs);
        ProfScope ps(kProfSearchFull, st, 2);
        k_search_full<<<dim3(nqb, ntiles, nsplit), kThreads, smem, st>>>(
            qfull, fail_list, fail_count, Q, Dp, efull, enorm, ntiles, 1, qnorm, cand_idx, cand_lb, part_v, part_i,
            status, kcs, pdist->ptr, 0, C * w * w);
        k_full_select<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(pdist->ptr, nsplit, (int)npad, N, fail_list,
                                                                    fail_count, Q, qnorm, cand_idx, cand_lb, status);
        return nsplit;
    }
    ProfScope ps(kProfSearchFull, st, 2);
    launch_full_adaptive(qfull, fail_list, fail_count, Q, Dp, C * w * w, efull, enorm, ntiles, qnorm, cand_idx, cand_lb, part_v,
                         part_i, status, st);
    return 1;
}

void launch_search_rows(const float *rows, int da, int dk, const int *list, const unsigned int *count, int Q,
                        int Dp, float *qtiles, const float *etiles, const float *enorm, int ntiles, const float *qnorm,
                        int *cand_idx, float *cand_lb, float *part_v, int *part_i, int *status,
                        cudaStream_t st) {
    const size_t smem = sizeof(FullSmem);
    set_smem_attr(reinterpret_cast<const void *>(k_search_full), (int)smem);
    count_launches(1);
    k_gather_rows<<<152 * 4, 256, 0, st>>>(rows, da, list, count, Q, Dp, qtiles);
    ProfScope ps(kProfSearchTopk, st, 2);
    launch_full_adaptive(qtiles, list, count, Q, Dp, dk, etiles, enorm, ntiles, qnorm, cand_idx, cand_lb, part_v, part_i,
                         status, st);
}

void launch_full_select_range(const float *score, int nsplit, int npad, int N, int q0, int nq, int Q,
                              const float *qnorm, int *cand_idx, float *cand_lb, int *status, cudaStream_t st) {
    if (nq <= 0) return;
    count_launches(1);
    k_full_select_range<<<ceil_div((long)nq * 32, 256), 256, 0, st>>>(score, nsplit, npad, N, q0, nq, Q, qnorm,
                                                                      cand_idx, cand_lb, status);
}

size_t full_part_capacity(int Q) {
    return std::min<size_t>((size_t)std::max(Q, 1) * kMaxAdaptiveParts, (size_t)kPartRows) * kTopK;
}

void launch_exemplar_full(const float *Z, int We, int C, int w, int ex, int N, const float *mu,
                          float *efull, int ntiles, cudaStream_t st) {
    const int Dp = padded_dim(C * w * w);
    cudaMemsetAsync(efull, 0, sizeof(float) * (size_t)ntiles * Dp * kBN, st);
    count_launches(1);
    k_exemplar_full<<<152 * 8, 256, 0, st>>>(Z, We, C, w, ex, N, Dp, mu, efull);
}

}  // namespace pts
