// search_tc.cu -- PCA-space search phase (E-step) on the tcgen05 tensor cores: FP16 operands,
// FP32 accumulation in tensor memory, a per-query top-32 in the epilogue.
//
// Score of query q against exemplar window n (section 2.2: PCA coordinates plus the residual
// norm bound the full-dimension distance from below):
//   p(q, n) = ||u_n||^2 - 2 (y_q . y_n + r_q r_n),   LB(q, n) = p(q, n) + ||u_q||^2.
// K carries d coordinates, the residual and three slots holding ||u_n||^2 split FP16
// hi/mid/lo against query-side ones, so the accumulator is p with no epilogue add.
//
// GEMM layout: M = 128 queries per CTA (TMEM lane = query), N = 256 windows per exemplar tile
// (TMEM columns), both operands K-major in the no-swizzle core-matrix layout, staged by 1-D bulk
// copies of pre-packed tiles: the query tile once, the exemplar tiles through a 2-stage ring.
// Two accumulator stages of 256 columns fill TMEM's 512.
//
// Warps (10): 0-7 epilogue (TMEM lane quarter = warp % 4, column half = warp / 4), 8 producer,
// 9 MMA issuer and TMEM owner.  Selection works on groups of 8 consecutive windows; a tile's
// 32 groups are split 16/16 between its column halves.  An epilogue thread owns one (query, half)
// and keeps, in registers, the 8 groups of its half with the smallest minimum score seen so
// far, sorted by (minimum, group); the 8 scores of each kept group sit in a shared-memory slot
// that moves with the group, as FP16 offsets from the group minimum.  Per tile the thread loads
// its 128 accumulators (two 64-column tcgen05.ld), reduces each group of 8 to its minimum and,
// only for a group whose minimum beats the 8th kept one, shifts it into the register list and
// stores its offsets into the slot of the evicted group.  Every window among the query's 8 best
// of a half lies in one of that half's 8 best groups, and each list is exactly those 8 groups
// whatever the scan order (ties go to the smaller group, which comes first).  At the end each
// warp takes queries one at a time, rebuilds the 2 x 64 kept scores (minimum + offset, 4 per
// lane) and keeps the 32 smallest (score, window) pairs by bitonic sort and merge.  Padding
// windows score NaN: a group minimum ignores them and they are dropped.
//
// The exemplar tiles of a query block may be split across blockIdx.y; each part keeps the 8 best
// groups of its own tiles and k_select_parts takes the 8 best of their union per half, so the
// result does not depend on the split.  Optional per-query, per-half bounds thr0 (warm
// start, an upper bound on the 8th best group minimum of each half) seed the group lists with
// sentinels (thr0, none): only groups whose minimum is below the bound are kept, and since at
// least 8 are, the kept groups are the same as without the bound.  All waits are bounded; on a
// timeout the kernel flags the status word, drains its copies and frees TMEM.
#include <algorithm>
#include <climits>
#include <cmath>
#include <type_traits>
#include <vector>

#include "tc_common.cuh"
#include "warp_keys.cuh"

namespace pts {
namespace {

constexpr int kQM = kTcQueryRows;   // queries per CTA (MMA M)
constexpr int kTN = 256;            // exemplar windows per tile (MMA N)
constexpr int kAcc = 2;             // accumulator stages of kTN columns
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = kEpiThreads + 64;
constexpr int kMaxKt = 128;         // K of the search vectors
constexpr int kRing = 128 * 1024;   // bytes of exemplar-tile ring
constexpr int kMaxStages = 8;
constexpr int kG = 8;               // windows per group
constexpr int kKeep = 8;            // groups kept per (query, column half)
constexpr int kPayStride = kKeep + 1;  // 16-byte units per thread of kept offsets (one per slot, odd)
constexpr unsigned kFull = 0xffffffffu;
constexpr int kNoWindow = INT_MAX;
constexpr int kNoGroup = 0x7FFFFFF;  // group field of a sentinel (27 bits)

struct TcSmem {
    alignas(1024) unsigned char q[kQM * kMaxKt * 2];
    alignas(1024) unsigned char e[kRing];
    uint4 pay[kEpiThreads * kPayStride];   // per thread, per slot: a kept group's 8 FP16 offsets
    uint64_t full[kMaxStages], empty[kMaxStages], acc_full[kAcc], acc_empty[kAcc], q_full, done;
    uint32_t tmem_base;
    int abort_flag;
};
static_assert(kAcc == 2, "the MMA issuer alternates two accumulators");
static_assert(sizeof(TcSmem) + 1024 <= 227 * 1024, "tensor-core search tile set exceeds shared memory");

// Sorted register list of the kept groups: value gv[k] (group minimum) and gs[k] = group << 4 |
// slot, ascending in (value, group).
struct GroupList {
    float gv[kKeep];
    int gs[kKeep];
};

// Shifts (x, group) into the list (the caller checked x < gv[kKeep - 1]), reusing the evicted
// entry's slot, and returns that slot.  Groups arrive in increasing order, so a strict value test
// places ties after the groups already kept.
__device__ __forceinline__ int group_insert(GroupList &L, float x, int group) {
    const int slot = L.gs[kKeep - 1] & 15;  // kKeep <= 16
    const int packed = (group << 4) | slot;
#pragma unroll
    for (int k = kKeep - 1; k > 0; --k) {
        const bool before_prev = x < L.gv[k - 1];
        const bool here = x < L.gv[k];
        L.gv[k] = before_prev ? L.gv[k - 1] : (here ? x : L.gv[k]);
        L.gs[k] = before_prev ? L.gs[k - 1] : (here ? packed : L.gs[k]);
    }
    if (x < L.gv[0]) {
        L.gv[0] = x;
        L.gs[0] = packed;
    }
    return slot;
}

// minimum of three (a NaN operand is ignored, as by fminf)
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// 64 columns (8 groups) of a tile for the calling thread's query.
__device__ __forceinline__ void scan64(const float (&v)[64], int group0, GroupList &L, uint4 *pay_row) {
    float m[8];
#pragma unroll
    for (int g = 0; g < 8; ++g)
        m[g] = min3f(min3f(v[8 * g], v[8 * g + 1], v[8 * g + 2]), min3f(v[8 * g + 3], v[8 * g + 4], v[8 * g + 5]),
                     fminf(v[8 * g + 6], v[8 * g + 7]));
    const float mm = min3f(min3f(m[0], m[1], m[2]), min3f(m[3], m[4], m[5]), fminf(m[6], m[7]));
    if (!__any_sync(kFull, mm < L.gv[kKeep - 1])) return;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        if (m[g] < L.gv[kKeep - 1]) {
            const int slot = group_insert(L, m[g], group0 + g);
            // offsets from the minimum (NaN stays NaN): FP16 keeps them to 2^-11 relative
            uint4 pk;
            __half2 h;
            h = __floats2half2_rn(v[8 * g] - m[g], v[8 * g + 1] - m[g]);
            pk.x = *reinterpret_cast<uint32_t *>(&h);
            h = __floats2half2_rn(v[8 * g + 2] - m[g], v[8 * g + 3] - m[g]);
            pk.y = *reinterpret_cast<uint32_t *>(&h);
            h = __floats2half2_rn(v[8 * g + 4] - m[g], v[8 * g + 5] - m[g]);
            pk.z = *reinterpret_cast<uint32_t *>(&h);
            h = __floats2half2_rn(v[8 * g + 6] - m[g], v[8 * g + 7] - m[g]);
            pk.w = *reinterpret_cast<uint32_t *>(&h);
            pay_row[slot] = pk;
        }
    }
}

// FP8 scores: p = ||u_n||^2 + t_q acc for 64 consecutive windows from col0 (NaN past N).  The
// norms are the same for every lane of a warp (one broadcast load each).
__device__ __forceinline__ void fp8_finish(float (&v)[64], float tq, const float *__restrict__ enorm, int col0,
                                           int N) {
#pragma unroll
    for (int j4 = 0; j4 < 16; ++j4) {
        const int c = col0 + 4 * j4;
        float4 e;
        if (c + 3 < N) {
            e = __ldg(reinterpret_cast<const float4 *>(enorm + c));
        } else {
            e.x = c < N ? __ldg(enorm + c) : NAN;
            e.y = c + 1 < N ? __ldg(enorm + c + 1) : NAN;
            e.z = c + 2 < N ? __ldg(enorm + c + 2) : NAN;
            e.w = c + 3 < N ? __ldg(enorm + c + 3) : NAN;
        }
        v[4 * j4] = fmaf(tq, v[4 * j4], e.x);
        v[4 * j4 + 1] = fmaf(tq, v[4 * j4 + 1], e.y);
        v[4 * j4 + 2] = fmaf(tq, v[4 * j4 + 2], e.z);
        v[4 * j4 + 3] = fmaf(tq, v[4 * j4 + 3], e.w);
    }
}

// Cluster-restricted blocks (the learned proposal's probe): block b covers rows f0 .. f0+nrows-1
// of the (query, probed cluster) pair list and the exemplar tiles t_begin .. t_begin+nt-1 of its
// cluster (exemplar tiles in cluster order); a row's 32 best go to part slot pair_r of pair_q.
// What an epilogue thread keeps for its (output row, column half): the 8 groups' minima and
// indices, and each group's 8 scores as FP16 offsets from its minimum (slot order).
struct KeptGroups {
    float gmin[kKeep];
    int gmap[kKeep];
    uint4 pay[kKeep];
};

struct IvfArgs {
    const int4 *blk;         // [nblk] (f0, nrows, t_begin, nt)
    const int *nblk;         // device count of blocks
    const int *pair_q, *pair_r;
};

// EB = operand bytes: 2 for FP16 (kind::f16, the norms ride in K), 1 for FP8 E4M3
// (kind::f8f6f4, per-dimension scales; the epilogue forms p = ||u_n||^2 + t_q acc).
template <int EB>
__global__ void __launch_bounds__(kThreads, 1)
    k_search_tc(const void *__restrict__ qtile, const float *__restrict__ qnorm, int Q, int K,
                const void *__restrict__ etile, int ntiles, int tiles_per_part, int nstages,
                const float *__restrict__ qscale, const float *__restrict__ enorm, int N,
                const float *__restrict__ thr0, const int *__restrict__ qlist,
                const unsigned int *__restrict__ qcount, IvfArgs ivf, KeptGroups *__restrict__ kept,
                int *__restrict__ status, int tail_from, int tail_parts) {
    // with a query list, tile row f holds query qlist[f] (f < *qcount); blocks past the list exit
    const int nrows = qlist ? (int)min((unsigned int)Q, *qcount) : Q;
    // Query block, exemplar part and the part count of this block.  With tail_parts > 1 (a 1-D
    // grid), the blocks before tail_from run unsplit and each later query block is split over
    // tail_parts CTAs of tiles_per_part tiles: only the last, partial wave is cut finer.  Their
    // records go to a second region after the unsplit blocks' ones.
    int qb = blockIdx.x, part = blockIdx.y, nsplit = gridDim.y, tpp = tiles_per_part;
    KeptGroups *kbase = kept;
    int qoff = 0;
    if (tail_parts > 1) {
        if ((int)blockIdx.x < tail_from) {
            part = 0;
            nsplit = 1;
            tpp = ntiles;
        } else {
            const int j = (int)blockIdx.x - tail_from;
            qb = tail_from + j / tail_parts;
            part = j % tail_parts;
            nsplit = tail_parts;
            kbase = kept + (size_t)tail_from * kQM * 2;
            qoff = tail_from * kQM;
        }
    }
    int4 blk = make_int4(0, 0, 0, 0);
    if (ivf.blk) {
        if ((int)blockIdx.x >= *ivf.nblk) return;
        blk = ivf.blk[blockIdx.x];
    } else if (qb * kQM >= nrows) {
        return;
    }
    // tile row r -> query (and, for cluster-restricted blocks, its part slot); -1 when empty
    auto row_query = [&](int r, int *slot) -> int {
        if (ivf.blk) {
            if (r >= blk.y) return -1;
            *slot = ivf.pair_r[blk.x + r];
            return ivf.pair_q[blk.x + r];
        }
        const int f = qb * kQM + r;
        *slot = part;
        return f < nrows ? (qlist ? qlist[f] : f) : -1;
    };
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    volatile int *abort_flag = &sm.abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nparts = ivf.blk ? 4 : nsplit;
    const int t_begin = ivf.blk ? blk.z : part * tpp;
    const int nt = ivf.blk ? blk.w : max(0, min(ntiles, t_begin + tpp) - t_begin);
    const uint32_t stage_bytes = (uint32_t)(kTN * K * EB);
    const uint32_t q_bytes = (uint32_t)(kQM * K * EB);
    const unsigned char *qtile_b = static_cast<const unsigned char *>(qtile);
    const unsigned char *etile_b = static_cast<const unsigned char *>(etile);

    if (warp == kEpiWarps + 1) {
        tmem_alloc(&sm.tmem_base, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < nstages; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        for (int a = 0; a < kAcc; ++a) {
            mbar_init(&sm.acc_full[a], 1);
            mbar_init(&sm.acc_empty[a], kEpiWarps);
        }
        mbar_init(&sm.q_full, 1);
        mbar_init(&sm.done, 1);
        fence_mbar_init();
        sm.abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    if (warp == kEpiWarps) {
        // ---------------- producer ----------------
        if (lane == 0) {
            mbar_expect_tx(&sm.q_full, q_bytes);
            bulk_g2s(sm.q, qtile_b + (size_t)(ivf.blk ? blockIdx.x : qb) * q_bytes, q_bytes, &sm.q_full);
            int issued = 0;
            for (int i = 0; i < nt; ++i) {
                const int s = i % nstages;
                if (i >= nstages &&
                    !mbar_wait_or_abort(&sm.empty[s], (uint32_t)(((i / nstages) - 1) & 1), status, abort_flag))
                    break;
                mbar_expect_tx(&sm.full[s], stage_bytes);
                bulk_g2s(sm.e + (size_t)s * stage_bytes, etile_b + (size_t)(t_begin + i) * stage_bytes, stage_bytes,
                         &sm.full[s]);
                issued = i + 1;
            }
            // every copy this thread issued has landed before the CTA may exit
            mbar_wait_bounded(&sm.q_full, 0, status);
            for (int i = max(0, issued - nstages); i < issued; ++i)
                mbar_wait_bounded(&sm.full[i % nstages], (uint32_t)((i / nstages) & 1), status);
        }
    } else if (warp == kEpiWarps + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = EB == 2 ? idesc_f16(kQM, kTN) : idesc_e4m3(kQM, kTN);
            const uint32_t lbo_q = (uint32_t)(kQM / 8) * 128u, lbo_e = (uint32_t)(kTN / 8) * 128u;
            const uint32_t qaddr = smem_u32(sm.q);
            bool ok = mbar_wait_or_abort(&sm.q_full, 0, status, abort_flag);
            // descriptors built once: the address field (bits 0-13, 16-byte units) of every later
            // operand is the base's plus an offset, all inside shared memory
            const uint64_t adesc0 = smem_desc(qaddr, lbo_q, 128u);
            const uint64_t bdesc0 = smem_desc(smem_u32(sm.e), lbo_e, 128u);
            const uint64_t a_step = (2u * lbo_q) >> 4, b_step = (2u * lbo_e) >> 4, b_stage = stage_bytes >> 4;
            const int nks = K * EB / 32;
            int s = 0;
            uint32_t full_par = 0;
            for (int i = 0; i < nt && ok; ++i) {
                const int a = i & 1;  // kAcc == 2
                if (i >= kAcc &&
                    !mbar_wait_or_abort(&sm.acc_empty[a], (uint32_t)(((i >> 1) - 1) & 1), status, abort_flag))
                    break;
                if (!mbar_wait_or_abort(&sm.full[s], full_par, status, abort_flag)) break;
                tc_fence_after();
                const uint64_t bd = bdesc0 + (uint64_t)s * b_stage;
                const uint32_t dcol = tmem + (uint32_t)(a * kTN);
                // one instruction per 32 bytes of K (16 FP16 or 32 FP8 values): two core-matrix columns
                for (int ks = 0; ks < nks; ++ks) {
                    if constexpr (EB == 2)
                        mma_bf16(dcol, adesc0 + ks * a_step, bd + ks * b_step, idesc, ks > 0 ? 1u : 0u);
                    else
                        mma_f8(dcol, adesc0 + ks * a_step, bd + ks * b_step, idesc, ks > 0 ? 1u : 0u);
                }
                mma_commit(&sm.empty[s]);
                mma_commit(&sm.acc_full[a]);
                if (++s == nstages) {
                    s = 0;
                    full_par ^= 1u;
                }
            }
            // all MMAs issued by this thread have completed once `done` fires
            mma_commit(&sm.done);
            mbar_wait_bounded(&sm.done, 0, status);
        }
    } else {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3, half = warp >> 2;
        const int row = quarter * 32 + lane;
        int slot_unused = 0;
        const int q = row_query(row, &slot_unused);
        GroupList L;
        {
            const float t = q >= 0 ? (thr0 ? thr0[2 * (size_t)q + half] : INFINITY) : -INFINITY;
#pragma unroll
            for (int k = 0; k < kKeep; ++k) {
                L.gv[k] = t;
                L.gs[k] = (kNoGroup << 4) | k;
            }
        }
        uint4 *pay_row = &sm.pay[tid * kPayStride];
        const float tq = (EB == 1 && q >= 0) ? qscale[q] : 0.0f;
        const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * (kTN / 2));
        for (int i = 0; i < nt; ++i) {
            const int a = i % kAcc;
            const bool ok = mbar_wait_or_abort(&sm.acc_full[a], (uint32_t)((i / kAcc) & 1), status, abort_flag);
            if (!__all_sync(kFull, ok)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int group0 = (t_begin + i) * (kTN / kG) + half * (kTN / kG / 2);
            const int col0 = group0 * kG;
            // both 64-column halves in one load: one wait, and the accumulator is released
            // before the scan
            float v[128];
            tmem_ld128(lane_addr + (uint32_t)(a * kTN), v);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.acc_empty[a]);
            float (&v0)[64] = *reinterpret_cast<float (*)[64]>(&v[0]);
            float (&v1)[64] = *reinterpret_cast<float (*)[64]>(&v[64]);
            if constexpr (EB == 1) fp8_finish(v0, tq, enorm, col0, N);
            scan64(v0, group0, L, pay_row);
            if constexpr (EB == 1) fp8_finish(v1, tq, enorm, col0 + 64, N);
            scan64(v1, group0 + 8, L, pay_row);
        }
        // hand the kept groups to k_select (one record per output row and column half)
        if (!*abort_flag && q >= 0) {
            int slot = 0;
            row_query(row, &slot);
            KeptGroups *rec = kbase + (((size_t)(q - qoff) * nparts + slot) * 2 + half);
#pragma unroll
            for (int k = 0; k < kKeep; ++k) {
                const int sl = L.gs[k] & 15;
                rec->gmin[sl] = L.gv[k];
                rec->gmap[sl] = L.gs[k] >> 4;
                rec->pay[sl] = pay_row[sl];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kEpiWarps + 1) {
        __syncwarp();
        tmem_dealloc(tmem, 512);
    }
}

// One warp per output row (query x part): the 32 smallest (score, window) pairs among the 2 x 8
// kept groups of its two column halves, sorted; to the candidate lists (+ ||u_q||^2) when the
// row is the query's only part, else to the part lists.  Windows are indexed through perm when
// the tiles hold them in another order.
__global__ void __launch_bounds__(256) k_select(const KeptGroups *__restrict__ kept, int Q, int nparts,
                                                const float *__restrict__ qnorm, const int *__restrict__ perm, int N,
                                                int *__restrict__ cand_idx, float *__restrict__ cand_lb,
                                                float *__restrict__ part_v, int *__restrict__ part_i) {
    const int lane = threadIdx.x & 31;
    const long o = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (o >= (long)Q * nparts) return;
    const unsigned long long kNone = pack_key(INFINITY, kNoWindow);
    unsigned long long key[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const KeptGroups &rec = kept[o * 2 + (c >> 1)];
        const int k = lane + 32 * (c & 1);  // slot k / 8, element k % 8
        const int grp = rec.gmap[k / kG];
        const __half off = reinterpret_cast<const __half *>(&rec.pay[k / kG])[k % kG];
        const float x = rec.gmin[k / kG] + __half2float(off);
        key[c] = (grp != kNoGroup && !isnan(x)) ? pack_key(x, grp * kG + (k % kG)) : kNone;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) warp_sort_keys(key[c], lane);
    warp_merge_keys(key[0], key[1], lane);
    warp_merge_keys(key[2], key[3], lane);
    warp_merge_keys(key[0], key[2], lane);
    const float v = key_value(key[0]);
    const int i = key_index(key[0]);
    if (nparts == 1) {
        bool real = i != kNoWindow;
        int n = i;
        if (real && perm) {
            real = n >= 0 && n < N;
            n = real ? perm[n] : -1;
        }
        cand_idx[o * kTopK + lane] = real ? n : -1;
        cand_lb[o * kTopK + lane] = real ? v + qnorm[o] : INFINITY;
    } else {
        part_v[o * kTopK + lane] = v;
        part_i[o * kTopK + lane] = i;
    }
}

// Query q of a search whose tiles were split into nparts parts of tpp tiles, one warp.  Each
// part kept the 8 best groups of its own tiles per column half, so their union holds the 8 best
// of the whole half: first those, by (minimum, group), then the 32 smallest (score, window) pairs
// of the 2 x 8 groups.  The result is the single-part one, whatever the split or a warm bound.
__device__ __forceinline__ void select_parts_row(const KeptGroups *__restrict__ kept, long q, int nparts, int tpp,
                                                 const float *__restrict__ qnorm, int *__restrict__ cand_idx,
                                                 float *__restrict__ cand_lb, int lane) {
    const unsigned long long kNone = pack_key(INFINITY, kNoWindow);
    unsigned long long best[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        best[h] = kNone;
        for (int p0 = 0; p0 < nparts; p0 += 32 / kKeep) {
            const int p = p0 + lane / kKeep, s = lane % kKeep;
            unsigned long long g = kNone;
            if (p < nparts) {
                const KeptGroups &rec = kept[(q * nparts + p) * 2 + h];
                const int grp = rec.gmap[s];
                const float m = rec.gmin[s];
                if (grp != kNoGroup && !isnan(m)) g = pack_key(m, grp);
            }
            warp_sort_keys(g, lane);
            if (p0 == 0)
                best[h] = g;
            else
                warp_merge_keys(best[h], g, lane);
        }
    }
    // lanes 0..7 of best[h]: the 8 best groups of half h, ascending
    unsigned long long key[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int h = c >> 1;
        const int k = lane + 32 * (c & 1);  // rank k / 8 in half h, element k % 8
        const unsigned long long g = __shfl_sync(kFull, best[h], k / kG);
        key[c] = kNone;
        if (g != kNone) {
            const int grp = key_index(g);
            const int p = grp / (kTN / kG) / tpp;
            const KeptGroups &rec = kept[(q * nparts + p) * 2 + h];
            int j = 0;
#pragma unroll
            for (int s = 1; s < kKeep; ++s) j = rec.gmap[s] == grp ? s : j;
            const __half off = reinterpret_cast<const __half *>(&rec.pay[j])[k % kG];
            const float x = rec.gmin[j] + __half2float(off);
            if (!isnan(x)) key[c] = pack_key(x, grp * kG + (k % kG));
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) warp_sort_keys(key[c], lane);
    warp_merge_keys(key[0], key[1], lane);
    warp_merge_keys(key[2], key[3], lane);
    warp_merge_keys(key[0], key[2], lane);
    const int i = key_index(key[0]);
    const bool real = i != kNoWindow;
    cand_idx[q * kTopK + lane] = real ? i : -1;
    cand_lb[q * kTopK + lane] = real ? key_value(key[0]) + qnorm[q] : INFINITY;
}

// select_parts_row for every query, one warp each
__global__ void __launch_bounds__(256) k_select_parts(const KeptGroups *__restrict__ kept, int Q, int nparts, int tpp,
                                                      const float *__restrict__ qnorm, int *__restrict__ cand_idx,
                                                      float *__restrict__ cand_lb) {
    const long q = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    select_parts_row(kept, q, nparts, tpp, qnorm, cand_idx, cand_lb, threadIdx.x & 31);
}

// k_select for a device-side query list (one part per query)
__global__ void __launch_bounds__(256) k_select_list(const KeptGroups *__restrict__ kept, const int *__restrict__ qlist,
                                                     const unsigned int *__restrict__ qcount, int Q,
                                                     const float *__restrict__ qnorm, int *__restrict__ cand_idx,
                                                     float *__restrict__ cand_lb) {
    const long f = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (f >= (long)min((unsigned int)Q, *qcount)) return;
    const int q = qlist[f];
    if (q < 0 || q >= Q) return;
    // same as k_select for row q with one part
    const int lane = threadIdx.x & 31;
    const unsigned long long kNone = pack_key(INFINITY, kNoWindow);
    unsigned long long key[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const KeptGroups &rec = kept[(long)q * 2 + (c >> 1)];
        const int k = lane + 32 * (c & 1);
        const int grp = rec.gmap[k / kG];
        const __half off = reinterpret_cast<const __half *>(&rec.pay[k / kG])[k % kG];
        const float x = rec.gmin[k / kG] + __half2float(off);
        key[c] = (grp != kNoGroup && !isnan(x)) ? pack_key(x, grp * kG + (k % kG)) : kNone;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) warp_sort_keys(key[c], lane);
    warp_merge_keys(key[0], key[1], lane);
    warp_merge_keys(key[2], key[3], lane);
    warp_merge_keys(key[0], key[2], lane);
    const int i = key_index(key[0]);
    const bool real = i != kNoWindow;
    cand_idx[(size_t)q * kTopK + lane] = real ? i : -1;
    cand_lb[(size_t)q * kTopK + lane] = real ? key_value(key[0]) + qnorm[q] : INFINITY;
}

// One warp per query: merges the sorted part lists into the final candidate list.
__global__ void k_merge_parts(const float *__restrict__ part_v, const int *__restrict__ part_i, int Q, int nparts,
                              const float *__restrict__ qnorm, int *__restrict__ cand_idx,
                              float *__restrict__ cand_lb, const int *__restrict__ perm, int nperm) {
    const int lane = threadIdx.x & 31;
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    const size_t base = (size_t)q * nparts * kTopK;
    unsigned long long k = pack_key(part_v[base + lane], part_i[base + lane]);
    for (int p = 1; p < nparts; ++p)
        warp_merge_keys(k, pack_key(part_v[base + (size_t)p * kTopK + lane], part_i[base + (size_t)p * kTopK + lane]),
                        lane);
    int i = key_index(k);
    bool real = i != kNoWindow;
    if (real && perm) {  // cluster-ordered positions -> window indices
        real = i >= 0 && i < nperm;
        i = real ? perm[i] : kNoWindow;
    }
    cand_idx[(size_t)q * kTopK + lane] = real ? i : -1;
    cand_lb[(size_t)q * kTopK + lane] = real ? key_value(k) + qnorm[q] : INFINITY;
}

// Query vectors as FP16 MMA operand tiles: rows = queries, K = (y, r, 1, 1, 1, 0...); rows past Q
// are zero.  One tile of 128 queries is contiguous.
__global__ void k_pack_queries(const float *__restrict__ qcoord, int Q, int d, int da, int K, int nblocks,
                               const int *__restrict__ qlist, const unsigned int *__restrict__ qcount,
                               __half *__restrict__ out) {
    const int nrows = qlist ? (int)min((unsigned int)Q, *qcount) : Q;
    const long total = (long)min(nblocks, (nrows + kQM - 1) / kQM) * kQM * K;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int b = (int)(i / (kQM * K));
        const int rem = (int)(i - (long)b * kQM * K);
        const int r = rem / K, k = rem - r * K;
        const int f = b * kQM + r;
        const int q = f < nrows ? (qlist ? qlist[f] : f) : -1;
        float v = 0.0f;
        if (q >= 0 && q < Q) {
            if (k <= d)
                v = qcoord[(size_t)q * da + k];
            else if (k <= d + 3)
                v = 1.0f;
        }
        *reinterpret_cast<__half *>(reinterpret_cast<unsigned char *>(out + (size_t)b * kQM * K) +
                                    core_offset(r, k, kQM)) = __float2half_rn(v);
    }
}

// Exemplar vectors as FP16 MMA operand tiles: rows = windows, K = (-2 y, -2 r, norm hi/mid/lo,
// 0...).  Padding windows carry +inf and -inf in the hi and mid slots, so their score is NaN and
// fails every comparison.
__global__ void k_pack_exemplar(const float *__restrict__ et, const float *__restrict__ enorm, int N, int ntiles,
                                int d, int da, int K, const int *__restrict__ perm, __half *__restrict__ out) {
    const long total = (long)ntiles * kTN * K;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int t = (int)(i / (kTN * K));
        const int rem = (int)(i - (long)t * kTN * K);
        const int m = rem / K, k = rem - m * K;
        const long p = (long)t * kTN + m;
        const bool pad = p >= N;
        const long n = pad ? 0 : (perm ? perm[p] : p);  // row p holds window perm[p]
        const float nrm = pad ? 0.0f : enorm[n];
        float v = 0.0f;
        if (k <= d) {
            v = pad ? 0.0f : et[((n / kBN) * da + k) * kBN + (n % kBN)];
        } else if (k <= d + 3) {
            if (pad) {
                v = (k == d + 1) ? INFINITY : (k == d + 2) ? -INFINITY : 0.0f;
            } else {
                const float hi = __half2float(__float2half_rn(nrm));
                const float r1 = nrm - hi;
                const float mid = __half2float(__float2half_rn(r1));
                v = (k == d + 1) ? hi : (k == d + 2) ? mid : (r1 - mid);
            }
        }
        *reinterpret_cast<__half *>(reinterpret_cast<unsigned char *>(out + (size_t)t * kTN * K) +
                                    core_offset(m, k, kTN)) = __float2half_rn(v);
    }
}

// FP8 operands (E4M3, saturating).  Per search dimension j (coordinates and the residual) the
// exemplar side stores -2 y_nj / s_j with s_j = max_n |2 y_nj| / 448; the query absorbs s_j and a
// per-row scale t_q = max_j |y_qj s_j| / 448, so acc = sum_j q_j e_j = -2 (y_q . y_n + r_q r_n) / t_q.
__global__ void k_fp8_dim_scale(const float *__restrict__ et, int N, int d, int da, float *__restrict__ scale) {
    const int j = blockIdx.x;  // 0..d (coordinates, then the residual)
    float m = 0.0f;
    for (int n = threadIdx.x; n < N; n += blockDim.x) m = fmaxf(m, fabsf(et[((size_t)(n / kBN) * da + j) * kBN + (n % kBN)]));
    __shared__ float red[256];
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) scale[j] = red[0] > 0.0f ? red[0] / 448.0f : 1.0f;
}

__global__ void k_pack_exemplar_f8(const float *__restrict__ et, int N, int ntiles, int d, int da, int K,
                                   const float *__restrict__ scale, uint8_t *__restrict__ out) {
    const long total = (long)ntiles * kTN * K;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int t = (int)(i / (kTN * K));
        const int rem = (int)(i - (long)t * kTN * K);
        const int m = rem / K, k = rem - m * K;
        const long n = (long)t * kTN + m;
        float v = 0.0f;
        if (n < N && k <= d) v = et[((n / kBN) * da + k) * kBN + (n % kBN)] / scale[k];
        const __nv_fp8_e4m3 h(v);
        out[(size_t)t * kTN * K + core_offset8(m, k, kTN)] = *reinterpret_cast<const uint8_t *>(&h);
    }
}

// one warp per query row of the FP8 query tiles (rows past the list or Q are zero)
__global__ void k_pack_queries_f8(const float *__restrict__ qcoord, int Q, int d, int da, int K, int nblocks,
                                  const float *__restrict__ scale, const int *__restrict__ qlist,
                                  const unsigned int *__restrict__ qcount, uint8_t *__restrict__ out,
                                  float *__restrict__ qscale) {
    const int nrows = qlist ? (int)min((unsigned int)Q, *qcount) : Q;
    const int lane = threadIdx.x & 31;
    const long f = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (f >= (long)nblocks * kQM) return;
    const int q = f < nrows ? (qlist ? qlist[f] : (int)f) : -1;
    const bool ok = q >= 0 && q < Q;
    float m = 0.0f;
    for (int k = lane; k <= d; k += 32) m = ok ? fmaxf(m, fabsf(qcoord[(size_t)q * da + k] * scale[k])) : m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    const float tq = m > 0.0f ? m / 448.0f : 1.0f;
    const int b = (int)(f / kQM), r = (int)(f % kQM);
    for (int k = lane; k < K; k += 32) {
        float v = 0.0f;
        if (ok && k <= d) v = qcoord[(size_t)q * da + k] * scale[k] / tq;
        const __nv_fp8_e4m3 h(v);
        out[(size_t)b * kQM * K + core_offset8(r, k, kQM)] = *reinterpret_cast<const uint8_t *>(&h);
    }
    if (ok && lane == 0) qscale[q] = tq;
}

// --- cluster-restricted probe planning (learned proposal) ---
// Pairs (query q, probe rank r, cluster top[4q + r]) grouped by cluster; each cluster's pairs are
// cut into blocks of <= 128 rows that scan the tiles holding the cluster's members.
// Pair counts per cluster: a shared-memory histogram per block (most pairs fall into a few
// large clusters, so global atomics per pair would serialise), one global add per bin.
constexpr int kIvfChunk = 8192;  // pairs per block of the count and scatter kernels

__global__ void __launch_bounds__(1024) k_ivf_count(const int *__restrict__ top, int Q, int C, int *__restrict__ cnt) {
    __shared__ int h[1024];
    for (int c = threadIdx.x; c < 1024; c += blockDim.x) h[c] = 0;
    __syncthreads();
    const long p0 = (long)blockIdx.x * kIvfChunk, p1 = min(4L * Q, p0 + kIvfChunk);
    for (long i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
        const int c = top[i];
        if (c >= 0 && c < C) atomicAdd(&h[c], 1);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x)
        if (h[c]) atomicAdd(&cnt[c], h[c]);
}

// one block: pair offsets, per-cluster fill cursors, and the block table (C <= 1024)
__global__ void __launch_bounds__(1024) k_ivf_plan(const int *__restrict__ cnt, const int *__restrict__ moff, int C,
                                                   int max_blocks, int *__restrict__ poff, int *__restrict__ cursor,
                                                   int4 *__restrict__ blk, int *__restrict__ nblk) {
    __shared__ int sp[1024], sb[1024];
    const int c = threadIdx.x;
    const int n = c < C ? cnt[c] : 0;
    const int nb = (n + kQM - 1) / kQM;
    sp[c] = n;
    sb[c] = nb;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scans
        const int a = c >= o ? sp[c - o] : 0, b = c >= o ? sb[c - o] : 0;
        __syncthreads();
        sp[c] += a;
        sb[c] += b;
        __syncthreads();
    }
    const int p0 = sp[c] - n, b0 = sb[c] - nb;
    if (c < C) {
        poff[c] = p0;
        cursor[c] = p0;
        const int lo = moff[c], hi = moff[c + 1];
        const int t0 = lo / kTN, t1 = hi > lo ? (hi - 1) / kTN : t0 - 1;
        for (int j = 0; j < nb && b0 + j < max_blocks; ++j)
            blk[b0 + j] = make_int4(p0 + j * kQM, min(kQM, n - j * kQM), t0, t1 - t0 + 1);
    }
    if (c == 1023) *nblk = min(sb[1023], max_blocks);
}

// Writes each pair into its cluster's range: positions within the block from a shared-memory
// histogram, one global reservation per (block, cluster).
__global__ void __launch_bounds__(1024) k_ivf_scatter(const int *__restrict__ top, int Q, int C, int *__restrict__ cursor,
                                                      int *__restrict__ pair_q, int *__restrict__ pair_r) {
    __shared__ int h[1024], base[1024];
    for (int c = threadIdx.x; c < 1024; c += blockDim.x) h[c] = 0;
    __syncthreads();
    const long p0 = (long)blockIdx.x * kIvfChunk, p1 = min(4L * Q, p0 + kIvfChunk);
    constexpr int kPer = kIvfChunk / 1024;
    int pos[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const long i = p0 + threadIdx.x + (long)k * 1024;
        pos[k] = -1;
        if (i < p1) {
            const int c = top[i];
            if (c >= 0 && c < C) pos[k] = atomicAdd(&h[c], 1);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) base[c] = h[c] ? atomicAdd(&cursor[c], h[c]) : 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const long i = p0 + threadIdx.x + (long)k * 1024;
        if (pos[k] < 0) continue;
        const int slot = base[top[i]] + pos[k];
        pair_q[slot] = (int)(i >> 2);
        pair_r[slot] = (int)(i & 3);
    }
}

// FP16 query tiles of the cluster-restricted blocks: block b, row r = pair f0 + r; a thread
// converts 8 consecutive values and stores them as one 16-byte core-matrix row.
__global__ void k_pack_queries_ivf(const float *__restrict__ qcoord, int d, int da, int K, const int4 *__restrict__ blk,
                                   const int *__restrict__ nblk, const int *__restrict__ pair_q,
                                   __half *__restrict__ out) {
    const int b = blockIdx.x;
    if (b >= *nblk) return;
    const int4 e = blk[b];
    const int k8n = K / 8;
    for (int i = threadIdx.x; i < kQM * k8n; i += blockDim.x) {
        const int r = i / k8n, k0 = (i - r * k8n) * 8;
        const int q = r < e.y ? pair_q[e.x + r] : -1;
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int k = k0 + t;
            v[t] = q < 0 ? 0.0f : (k <= d ? qcoord[(size_t)q * da + k] : (k <= d + 3 ? 1.0f : 0.0f));
        }
        uint4 pk;
        uint32_t *pw = reinterpret_cast<uint32_t *>(&pk);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const __half2 h2 = __floats2half2_rn(v[2 * t], v[2 * t + 1]);
            pw[t] = *reinterpret_cast<const uint32_t *>(&h2);
        }
        *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(out + (size_t)b * kQM * K) +
                                   core_offset(r, k0, kQM)) = pk;
    }
}

// Warm start: the previous search's 32 windows of each query, scored in FP32 from the same FP16
// operands the tensor cores multiply (16-byte rows of the operand layout, 8 values per load, the
// query's row read from its packed tile).  A window's score bounds its group's minimum from
// above, so with g_1 <= g_2 <= ... the smallest score of each distinct group of one column half
// among them, that half's 8th best group minimum is at most g_8; plus a margin for a different
// summation order, that is the half's bound (thr0[2 q + half]).  With fewer than 8 distinct
// groups in a half its bound is +inf.  One warp per query, two sorts of 64-bit keys: by (half,
// group, score), which puts each group's minimum first in its run, then the minima by (half,
// score) with every other entry after the minima of its half.
__global__ void k_warm_threshold(const int *__restrict__ prev_idx, const __half *__restrict__ qtile,
                                 const float *__restrict__ qnorm, const __half *__restrict__ etile,
                                 const float *__restrict__ umax, int Q, int K, int N, float eps_scale,
                                 float *__restrict__ thr0) {
    const int lane = threadIdx.x & 31;
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    const int n = prev_idx[(size_t)q * kTopK + lane];
    const bool valid = n >= 0 && n < N;
    float p = INFINITY;
    if (valid) {
        const unsigned char *e = reinterpret_cast<const unsigned char *>(etile + (size_t)(n / kTN) * kTN * K);
        const unsigned char *a = reinterpret_cast<const unsigned char *>(qtile + (size_t)(q / kQM) * kQM * K);
        const int m = n % kTN, r = q % kQM;
        p = 0.0f;
        for (int k8 = 0; k8 < K; k8 += 8) {
            const uint4 ev = __ldg(reinterpret_cast<const uint4 *>(e + core_offset(m, k8, kTN)));
            const uint4 av = __ldg(reinterpret_cast<const uint4 *>(a + core_offset(r, k8, kQM)));
            const __half2 *eh = reinterpret_cast<const __half2 *>(&ev);
            const __half2 *ah = reinterpret_cast<const __half2 *>(&av);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float2 af = __half22float2(ah[h]);
                const float2 ef = __half22float2(eh[h]);
                p = fmaf(af.x, ef.x, p);
                p = fmaf(af.y, ef.y, p);
            }
        }
    }
    constexpr unsigned long long kLast = ~0ull;
    const int grp = valid ? n / kG : 0;
    const unsigned half = valid ? (unsigned)((grp % (kTN / kG)) / (kTN / kG / 2)) : 0u;
    const unsigned score = (unsigned)(pack_key(p, 0) >> 32);  // order-preserving bits of p
    unsigned long long k1 = valid ? ((unsigned long long)((half << 27) | (unsigned)grp) << 32) | score : kLast;
    warp_sort_keys(k1, lane);
    const unsigned long long before = __shfl_up_sync(kFull, k1, 1);
    const bool first = k1 != kLast && (lane == 0 || (before >> 32) != (k1 >> 32));
    const unsigned h1 = (unsigned)(k1 >> 59);  // the half bit
    unsigned long long k2 = k1 == kLast ? kLast
                                        : ((unsigned long long)h1 << 32) | (first ? (k1 & 0xffffffffull) : 0xffffffffull);
    warp_sort_keys(k2, lane);
    const int n0 = __popc(__ballot_sync(kFull, (k2 >> 32) == 0));  // entries of half 0
    const unsigned long long s0 = __shfl_sync(kFull, k2, 7);
    const unsigned long long s1 = __shfl_sync(kFull, k2, min(n0 + 7, 31));
    if (lane == 0) {
        const float eps = eps_scale * (qnorm[q] + 2.0f * *umax);
        // |error| of an FP32 sum of K exact products <= K 2^-24 sum|terms|, sum|terms| <= qnorm + 2 umax
        float g0 = INFINITY, g1 = INFINITY;
        if (n0 > 7 && (unsigned)s0 != 0xffffffffu) g0 = key_value(s0 << 32);
        if (n0 + 7 < 32 && (s1 >> 32) == 1 && (unsigned)s1 != 0xffffffffu) g1 = key_value(s1 << 32);
        thr0[2 * (size_t)q] = isinf(g0) ? INFINITY : g0 + eps;
        thr0[2 * (size_t)q + 1] = isinf(g1) ? INFINITY : g1 + eps;
    }
}

// --- self-test: one 128 x N x K tile through the same descriptors, written back row-major.
// With TA the A operand goes through tensor memory (tcgen05.st, then an MMA reading [a_tmem]).
// The search keeps A in shared memory: its two 256-column accumulators fill all 512 columns of
// tensor memory, so A has no room there.
template <typename T, bool TA>
__global__ void __launch_bounds__(128) k_tc_selftest(const T *__restrict__ A, const T *__restrict__ B, int N, int K,
                                                     uint32_t idesc, float *__restrict__ D, int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char *sa = sm_raw;
    unsigned char *sb = sm_raw + kQM * K * 2;
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < kQM * K; i += 128) *reinterpret_cast<T *>(sa + core_offset(i / K, i % K, kQM)) = A[i];
    for (int i = tid; i < N * K; i += 128) *reinterpret_cast<T *>(sb + core_offset(i / K, i % K, N)) = B[i];
    fence_proxy_async_smem();
    if (warp == 0) {
        tmem_alloc(&tbase, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;
    constexpr uint32_t kACol = 256;  // A in columns 256.. (D uses at most 256)
    if (TA) {
        // row tid of A, K values packed two per column
        uint32_t r[64];
#pragma unroll
        for (int c = 0; c < 64; ++c) {
            const int k = 2 * c;
            const T lo = k < K ? A[(size_t)tid * K + k] : T(0.0f);
            const T hi = k + 1 < K ? A[(size_t)tid * K + k + 1] : T(0.0f);
            r[c] = (uint32_t)(*reinterpret_cast<const unsigned short *>(&lo)) |
                   ((uint32_t)(*reinterpret_cast<const unsigned short *>(&hi)) << 16);
        }
        tmem_st64(tmem + ((uint32_t)(warp * 32) << 16) + kACol, r);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        const uint32_t lbo_a = (uint32_t)(kQM / 8) * 128u, lbo_b = (uint32_t)(N / 8) * 128u;
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t bdesc = smem_desc(smem_u32(sb) + ks * 2u * lbo_b, lbo_b, 128u);
            if (TA)
                mma_f16_ta(tmem, tmem + kACol + (uint32_t)(ks * 8), bdesc, idesc, ks > 0 ? 1u : 0u);
            else
                mma_bf16(tmem, smem_desc(smem_u32(sa) + ks * 2u * lbo_a, lbo_a, 128u), bdesc, idesc,
                         ks > 0 ? 1u : 0u);
        }
        mma_commit(&bar);
    }
    __syncwarp();
    mbar_wait_bounded(&bar, 0, status);
    tc_fence_after();
    for (int c = 0; c < N; c += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        const int row = warp * 32 + (tid & 31);
#pragma unroll
        for (int j = 0; j < 16; ++j) D[(size_t)row * N + c + j] = v[j];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// FP8 (E4M3) variant of the self-test: bytes in the 8-bit core-matrix layout, K = 32 per MMA.
__global__ void __launch_bounds__(128) k_tc_selftest_f8(const uint8_t *__restrict__ A, const uint8_t *__restrict__ B,
                                                        int N, int K, float *__restrict__ D, int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char *sa = sm_raw;
    unsigned char *sb = sm_raw + kQM * K;
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < kQM * K; i += 128) sa[core_offset8(i / K, i % K, kQM)] = A[i];
    for (int i = tid; i < N * K; i += 128) sb[core_offset8(i / K, i % K, N)] = B[i];
    fence_proxy_async_smem();
    if (warp == 0) {
        tmem_alloc(&tbase, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;
    if (tid == 0) {
        const uint32_t lbo_a = (uint32_t)(kQM / 8) * 128u, lbo_b = (uint32_t)(N / 8) * 128u;
        for (int ks = 0; ks < K / 32; ++ks)
            mma_f8(tmem, smem_desc(smem_u32(sa) + ks * 2u * lbo_a, lbo_a, 128u),
                   smem_desc(smem_u32(sb) + ks * 2u * lbo_b, lbo_b, 128u), idesc_e4m3(kQM, N), ks > 0 ? 1u : 0u);
        mma_commit(&bar);
    }
    __syncwarp();
    mbar_wait_bounded(&bar, 0, status);
    tc_fence_after();
    for (int c = 0; c < N; c += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        const int row = warp * 32 + (tid & 31);
#pragma unroll
        for (int j = 0; j < 16; ++j) D[(size_t)row * N + c + j] = v[j];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

pts_status run_selftest_f8(int N, int K, double *max_abs_err, double *max_abs_ref) {
    std::vector<uint8_t> hA((size_t)kQM * K), hB((size_t)N * K);
    std::vector<float> fA(hA.size()), fB(hB.size());
    uint64_t z = 0x1234567ull;
    auto nextf = [&]() {
        z = z * 6364136223846793005ull + 1442695040888963407ull;
        return (float)((z >> 40) & 0xFFFF) / 8192.0f - 4.0f;
    };
    for (size_t i = 0; i < hA.size(); ++i) {
        const __nv_fp8_e4m3 v(nextf());
        hA[i] = *reinterpret_cast<const uint8_t *>(&v);
        fA[i] = (float)v;
    }
    for (size_t i = 0; i < hB.size(); ++i) {
        const __nv_fp8_e4m3 v(nextf());
        hB[i] = *reinterpret_cast<const uint8_t *>(&v);
        fB[i] = (float)v;
    }
    DevBuf<uint8_t> dA, dB;
    DevBuf<float> dD;
    DevBuf<int> dst;
    PTS_TRY(dA.ensure(hA.size(), "selftest A"));
    PTS_TRY(dB.ensure(hB.size(), "selftest B"));
    PTS_TRY(dD.ensure((size_t)kQM * N, "selftest D"));
    PTS_TRY(dst.ensure(1, "selftest status"));
    PTS_CUDA_TRY(cudaMemcpy(dA.ptr, hA.data(), hA.size(), cudaMemcpyHostToDevice));
    PTS_CUDA_TRY(cudaMemcpy(dB.ptr, hB.data(), hB.size(), cudaMemcpyHostToDevice));
    PTS_CUDA_TRY(cudaMemset(dst.ptr, 0, sizeof(int)));
    const size_t smem = (size_t)(kQM + N) * K;
    cudaFuncSetAttribute(k_tc_selftest_f8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launches(1);
    k_tc_selftest_f8<<<1, 128, smem>>>(dA.ptr, dB.ptr, N, K, dD.ptr, dst.ptr);
    PTS_CUDA_TRY(cudaGetLastError());
    PTS_CUDA_TRY(cudaDeviceSynchronize());
    std::vector<float> hD((size_t)kQM * N);
    int hst = 0;
    PTS_CUDA_TRY(cudaMemcpy(hD.data(), dD.ptr, hD.size() * 4, cudaMemcpyDeviceToHost));
    PTS_CUDA_TRY(cudaMemcpy(&hst, dst.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    double err = 0.0, ref_max = 0.0;
    for (int i = 0; i < kQM; ++i)
        for (int j = 0; j < N; ++j) {
            double sacc = 0.0;
            for (int k = 0; k < K; ++k) sacc += (double)fA[(size_t)i * K + k] * fB[(size_t)j * K + k];
            err = std::max(err, std::fabs(sacc - hD[(size_t)i * N + j]));
            ref_max = std::max(ref_max, std::fabs(sacc));
        }
    *max_abs_err = err;
    *max_abs_ref = ref_max;
    if (hst) return set_error(PTS_ERR_TIMEOUT, "pts_tc_selftest: MMA completion wait gave up");
    return PTS_OK;
}

template <typename T, bool TA>
pts_status run_selftest(int N, int K, uint32_t idesc, double *max_abs_err, double *max_abs_ref) {
    std::vector<T> hA((size_t)kQM * K), hB((size_t)N * K);
    std::vector<float> fA(hA.size()), fB(hB.size());
    uint64_t z = 0x1234567ull;
    auto nextf = [&]() {
        z = z * 6364136223846793005ull + 1442695040888963407ull;
        return (float)((z >> 40) & 0xFFFF) / 32768.0f - 1.0f;
    };
    auto cvt = [](float x) -> T {
        if constexpr (std::is_same<T, __half>::value)
            return __float2half_rn(x);
        else
            return __float2bfloat16_rn(x);
    };
    auto back = [](T x) -> float {
        if constexpr (std::is_same<T, __half>::value)
            return __half2float(x);
        else
            return __bfloat162float(x);
    };
    for (size_t i = 0; i < hA.size(); ++i) {
        hA[i] = cvt(nextf());
        fA[i] = back(hA[i]);
    }
    for (size_t i = 0; i < hB.size(); ++i) {
        hB[i] = cvt(nextf());
        fB[i] = back(hB[i]);
    }
    DevBuf<T> dA, dB;
    DevBuf<float> dD;
    DevBuf<int> dst;
    PTS_TRY(dA.ensure(hA.size(), "selftest A"));
    PTS_TRY(dB.ensure(hB.size(), "selftest B"));
    PTS_TRY(dD.ensure((size_t)kQM * N, "selftest D"));
    PTS_TRY(dst.ensure(1, "selftest status"));
    PTS_CUDA_TRY(cudaMemcpy(dA.ptr, hA.data(), hA.size() * 2, cudaMemcpyHostToDevice));
    PTS_CUDA_TRY(cudaMemcpy(dB.ptr, hB.data(), hB.size() * 2, cudaMemcpyHostToDevice));
    PTS_CUDA_TRY(cudaMemset(dst.ptr, 0, sizeof(int)));
    const size_t smem = (size_t)(kQM + N) * K * 2;
    cudaFuncSetAttribute(k_tc_selftest<T, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launches(1);
    k_tc_selftest<T, TA><<<1, 128, smem>>>(dA.ptr, dB.ptr, N, K, idesc, dD.ptr, dst.ptr);
    PTS_CUDA_TRY(cudaGetLastError());
    PTS_CUDA_TRY(cudaDeviceSynchronize());
    std::vector<float> hD((size_t)kQM * N);
    int hst = 0;
    PTS_CUDA_TRY(cudaMemcpy(hD.data(), dD.ptr, hD.size() * 4, cudaMemcpyDeviceToHost));
    PTS_CUDA_TRY(cudaMemcpy(&hst, dst.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    double err = 0.0, ref_max = 0.0;
    for (int i = 0; i < kQM; ++i)
        for (int j = 0; j < N; ++j) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += (double)fA[(size_t)i * K + k] * fB[(size_t)j * K + k];
            err = std::max(err, std::fabs(s - hD[(size_t)i * N + j]));
            ref_max = std::max(ref_max, std::fabs(s));
        }
    *max_abs_err = err;
    *max_abs_ref = ref_max;
    if (hst) return set_error(PTS_ERR_TIMEOUT, "pts_tc_selftest: MMA completion wait gave up");
    return PTS_OK;
}

}  // namespace

int tc_padded_k(int d) { return ((d + 4) + 15) / 16 * 16; }

int tc_query_blocks(int Q) { return (Q + kQM - 1) / kQM; }

int tc_tiles(int N) { return (N + kTN - 1) / kTN; }

int tc_tile_rows() { return kTN; }

// Parts per query block.  Each part keeps its own best groups per query (k_select_parts merges
// them), so every extra part adds a set of kept-group records, its own warm-up of the running
// lists and a wider merge; the split is used only when the query blocks alone leave SMs idle.
int tc_parts(int Q, int ntiles) {
    const int nqb = tc_query_blocks(Q);
    int p = 1;
    while (nqb * (p + 1) <= 152 && ntiles / (p + 1) >= 32) ++p;
    return p;
}

void launch_pack_queries(const float *qcoord, int Q, int d, int da, int K, __half *qtile, cudaStream_t st,
                         const int *qlist, const unsigned int *qcount) {
    const int nb = tc_query_blocks(Q);
    if (nb == 0) return;
    count_launches(1);
    k_pack_queries<<<std::min<long>(ceil_div((long)nb * kQM * K, 256), 152 * 8), 256, 0, st>>>(
        qcoord, Q, d, da, K, nb, qlist, qcount, qtile);
}

void launch_pack_exemplar(const float *et, const float *enorm, int N, int d, int da, int K, __half *out,
                          cudaStream_t st, const int *perm) {
    count_launches(1);
    k_pack_exemplar<<<152 * 4, 256, 0, st>>>(et, enorm, N, tc_tiles(N), d, da, K, perm, out);
}

int ivf_max_blocks(int Q, int C) { return (4 * Q + kQM - 1) / kQM + C; }

void launch_ivf_probe(const int *top, int Q, int C, const int *moff, const float *qcoord, const float *qnorm, int d,
                      int da, int K, const __half *etile_ivf, int ntiles, int N, const int *members, IvfBuffers &b,
                      int *cand_idx, float *cand_lb, int *status, cudaStream_t st) {
    if (Q == 0) return;
    const int maxb = ivf_max_blocks(Q, C);
    cudaMemsetAsync(b.cnt, 0, sizeof(int) * C, st);
    count_launches(5);
    const int nchunk = (int)ceil_div(4L * Q, kIvfChunk);
    k_ivf_count<<<nchunk, 1024, 0, st>>>(top, Q, C, b.cnt);
    k_ivf_plan<<<1, 1024, 0, st>>>(b.cnt, moff, C, maxb, b.poff, b.cursor, b.blk, b.nblk);
    k_ivf_scatter<<<nchunk, 1024, 0, st>>>(top, Q, C, b.cursor, b.pair_q, b.pair_r);
    k_pack_queries_ivf<<<maxb, 256, 0, st>>>(qcoord, d, da, K, b.blk, b.nblk, b.pair_q, b.qtile);
    // every (query, probe) pair has a row in some block, so every kept record is written
    const size_t smem = sizeof(TcSmem) + 1024;
    set_smem_attr(reinterpret_cast<const void *>(k_search_tc<2>), (int)smem);
    const int nstages = std::min(kMaxStages, kRing / (kTN * K * 2));
    {
        ProfScope ps(kProfProbe, st, 1);
        const IvfArgs ivf{b.blk, b.nblk, b.pair_q, b.pair_r};
        k_search_tc<2><<<maxb, kThreads, smem, st>>>(b.qtile, qnorm, Q, K, etile_ivf, ntiles, ntiles, nstages, nullptr,
                                                    nullptr, N, nullptr, nullptr, nullptr, ivf,
                                                    reinterpret_cast<KeptGroups *>(b.kept), status, 0, 0);
    }
    count_launches(2);
    k_select<<<ceil_div((long)Q * 4 * 32, 256), 256, 0, st>>>(reinterpret_cast<const KeptGroups *>(b.kept), Q, 4, qnorm,
                                                              nullptr, N, cand_idx, cand_lb, b.part_v, b.part_i);
    k_merge_parts<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(b.part_v, b.part_i, Q, 4, qnorm, cand_idx, cand_lb,
                                                               members, N);
}

void launch_warm_threshold(const int *prev_idx, const __half *qtile, const float *qnorm, const __half *etile,
                           const float *umax, int Q, int K, int N, float eps_scale, float *thr0, cudaStream_t st) {
    if (Q == 0) return;
    count_launches(1);
    k_warm_threshold<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(prev_idx, qtile, qnorm, etile, umax, Q, K, N,
                                                                   eps_scale, thr0);
}

void launch_search_tc(const void *qtile, const float *qnorm, int Q, int K, const void *etile, int ntiles,
                      int nparts, const float *thr0, int *cand_idx, float *cand_lb, float *part_v, int *part_i,
                      int *status, cudaStream_t st, const int *qlist, const unsigned int *qcount, int fp8,
                      const float *qscale, const float *enorm, int N, void *kept_buf) {
    const size_t smem = sizeof(TcSmem) + 1024;
    if (fp8)
        set_smem_attr(reinterpret_cast<const void *>(k_search_tc<1>), (int)smem);
    else
        set_smem_attr(reinterpret_cast<const void *>(k_search_tc<2>), (int)smem);
    // a listed search runs unsplit: the proposal's fallback lists about a third of the fine
    // level's queries, enough blocks to fill the SMs, and a split measured slower there
    // nparts 0: automatic, one part with the tail split of tc_tail_plan; >= 1: that many parts
    if (qlist) nparts = 1;
    const int nqb = tc_query_blocks(Q);
    if (nqb == 0) return;
    int tail_from = nqb, tail_parts = 1;
    if (nparts == 0) tc_tail_plan(Q, ntiles, &tail_from, &tail_parts);
    nparts = std::max(nparts, 1);
    const int tpp = tail_parts > 1 ? (ntiles + tail_parts - 1) / tail_parts : (ntiles + nparts - 1) / nparts;
    const int eb = fp8 ? 1 : 2;
    const int nstages = std::min(kMaxStages, kRing / (kTN * K * eb));
    KeptGroups *kept = reinterpret_cast<KeptGroups *>(kept_buf);
    ProfScope ps(qlist ? kProfSearchTcList : kProfSearchTc, st, tail_parts > 1 ? 3 : 2);
    const dim3 grid = tail_parts > 1 ? dim3(tail_from + (nqb - tail_from) * tail_parts, 1) : dim3(nqb, nparts);
    if (fp8)
        k_search_tc<1><<<grid, kThreads, smem, st>>>(qtile, qnorm, Q, K, etile, ntiles, tpp, nstages, qscale, enorm, N,
                                                     thr0, qlist, qcount, IvfArgs{}, kept, status, tail_from,
                                                     tail_parts);
    else
        k_search_tc<2><<<grid, kThreads, smem, st>>>(qtile, qnorm, Q, K, etile, ntiles, tpp, nstages, qscale, enorm, N,
                                                     thr0, qlist, qcount, IvfArgs{}, kept, status, tail_from,
                                                     tail_parts);
    if (tail_parts > 1) {
        // the unsplit blocks' queries, then the split ones (records in their own region)
        const int qmain = tail_from * kQM;
        k_select<<<ceil_div((long)qmain * 32, 256), 256, 0, st>>>(kept, qmain, 1, qnorm, nullptr, N, cand_idx, cand_lb,
                                                                 part_v, part_i);
        k_select_parts<<<ceil_div((long)(Q - qmain) * 32, 256), 256, 0, st>>>(
            kept + (size_t)qmain * 2, Q - qmain, tail_parts, tpp, qnorm + qmain, cand_idx + (size_t)qmain * kTopK,
            cand_lb + (size_t)qmain * kTopK);
        return;
    }
    if (qlist) {
        // listed queries only: select for every row of the list
        k_select_list<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(kept, qlist, qcount, Q, qnorm, cand_idx, cand_lb);
        return;
    }
    if (nparts > 1)
        k_select_parts<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(kept, Q, nparts, tpp, qnorm, cand_idx, cand_lb);
    else
        k_select<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(kept, Q, 1, qnorm, nullptr, N, cand_idx, cand_lb,
                                                              part_v, part_i);
}

size_t tc_kept_bytes(int Q, int nparts) { return sizeof(KeptGroups) * 2 * (size_t)std::max(Q, 1) * nparts; }

// A search over the whole exemplar runs its query blocks unsplit, except those of the last,
// partial wave (one CTA per SM): when at least one full wave precedes them and they would leave
// most SMs idle, each is cut into up to 4 parts of the tiles, so the tail takes a fraction of a
// wave instead of a whole one.  Results equal the unsplit search (the parts' groups are merged).
void tc_tail_plan(int Q, int ntiles, int *tail_from, int *tail_parts) {
    const int nqb = tc_query_blocks(Q), sms = 152;
    *tail_from = nqb;
    *tail_parts = 1;
    const int full = nqb / sms * sms, tail = nqb - full;
    if (full == 0 || tail == 0 || 2 * tail > sms) return;
    const int p = std::min(4, std::min(sms / tail, ntiles / 16));
    if (p < 2) return;
    *tail_from = full;
    *tail_parts = p;
}

size_t tc_kept_bytes_search(int Q, int ntiles, int nparts) {
    if (nparts >= 1) return tc_kept_bytes(Q, nparts);
    int tail_from = 0, tail_parts = 1;
    tc_tail_plan(Q, ntiles, &tail_from, &tail_parts);
    return tc_kept_bytes(Q, tail_parts);
}

int tc_padded_k8(int d) { return ((d + 1) + 31) / 32 * 32; }

void launch_fp8_tables(const float *et, int N, int d, int da, int K, float *scale, uint8_t *out, cudaStream_t st) {
    count_launches(2);
    k_fp8_dim_scale<<<d + 1, 256, 0, st>>>(et, N, d, da, scale);
    k_pack_exemplar_f8<<<152 * 4, 256, 0, st>>>(et, N, tc_tiles(N), d, da, K, scale, out);
}

void launch_pack_queries_f8(const float *qcoord, int Q, int d, int da, int K, const float *scale, uint8_t *qtile,
                            float *qscale, cudaStream_t st, const int *qlist, const unsigned int *qcount) {
    const int nb = tc_query_blocks(Q);
    if (nb == 0) return;
    count_launches(1);
    k_pack_queries_f8<<<(unsigned)ceil_div((long)nb * kQM * 32, 256), 256, 0, st>>>(qcoord, Q, d, da, K, nb, scale,
                                                                                     qlist, qcount, qtile, qscale);
}

pts_status tc_selftest(int N, int K, int f16, double *max_abs_err, double *max_abs_ref) {
    if (N < 16 || N > 256 || N % 16 || K < 16 || K > 128 || K % 16)
        return set_error(PTS_ERR_INVALID_ARG, "pts_tc_selftest: N in 16..256 and K in 16..128, multiples of 16");
    if (f16 == 3) {
        if (K % 32) return set_error(PTS_ERR_INVALID_ARG, "pts_tc_selftest: FP8 needs K a multiple of 32");
        return run_selftest_f8(N, K, max_abs_err, max_abs_ref);
    }
    if (f16 == 2) return run_selftest<__half, true>(N, K, idesc_f16(kQM, N), max_abs_err, max_abs_ref);
    if (f16) return run_selftest<__half, false>(N, K, idesc_f16(kQM, N), max_abs_err, max_abs_ref);
    return run_selftest<__nv_bfloat16, false>(N, K, idesc_bf16(kQM, N), max_abs_err, max_abs_ref);
}

}  // namespace pts
