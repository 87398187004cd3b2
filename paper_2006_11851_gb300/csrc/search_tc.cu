// search_tc.cu -- PCA-space search phase (E-step) on the tcgen05 tensor cores, BF16 operands,
// FP32 accumulation in tensor memory.
//
// The GEMM is laid out transposed: M = 128 exemplar windows per tile (TMEM lanes), N = 64
// queries per CTA (TMEM columns), K = the search vector (d PCA coordinates, the residual norm,
// and three slots that carry ||u_n||^2 as a BF16 hi/mid/lo split against query-side ones, so
// the accumulator already holds p(q, n) = ||u_n||^2 - 2 a_q . e_n with no epilogue add).
// An epilogue warp reads a 32-lane quarter of TMEM (32 exemplar windows) x 16 columns (16
// queries): its lanes span windows and its registers span queries, so the per-query top-32
// lists stay warp-resident (one sorted entry per lane) and insertions never diverge.
//
// Warp roles (18 warps): 0-15 epilogue (TMEM lane quarter = warp % 4, query chunk = warp / 4),
// 16 producer (1-D bulk copies of pre-laid-out exemplar tiles into an 8-stage ring), 17 MMA
// issuer and TMEM owner.  One accumulator stage holds 4 exemplar tiles (4 x 64 columns) so the
// MMA -> epilogue -> release handoff is paid once per 512 windows; two stages fill all 512 TMEM
// columns.  Every wait is bounded; on a timeout the kernel flags the status word, drains what
// it issued and frees TMEM.  Each quarter keeps its own partial lists; they are merged in shared
// memory at the end.  An optional per-query bound thr0 (warm start) caps the lists' threshold.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tc_common.cuh"

namespace pts {
namespace {

constexpr int kTcM = 128;
constexpr int kTcN = 64;
constexpr int kTcSub = 4;      // exemplar tiles per accumulator stage
constexpr int kTcStages = 5;   // exemplar tiles in flight
constexpr int kTcQueue = 16;   // pending candidates per query before a merge
constexpr int kTcEpiWarps = 16;
constexpr int kTcThreads = (kTcEpiWarps + 2) * 32;
constexpr int kTcMaxK = 80;
constexpr int kTcStageCols = kTcSub * kTcN;  // 256 TMEM columns per accumulator stage
constexpr int kTcCols = 2 * kTcStageCols;    // 512: all of TMEM (one CTA per SM)
constexpr unsigned kFull = 0xffffffffu;

struct TcSmem {
    alignas(128) __nv_bfloat16 q[kTcN * kTcMaxK];
    alignas(128) __nv_bfloat16 e[kTcStages][kTcM * kTcMaxK];
    // per epilogue warp, per query of its chunk: the partial top-32 list (entry = lane)
    float lst_d[kTcEpiWarps][16][kTopK];
    int lst_i[kTcEpiWarps][16][kTopK];
    // per epilogue warp, per query: candidates that passed the filter, not merged yet
    float que_d[kTcEpiWarps][16][kTcQueue];
    int que_i[kTcEpiWarps][16][kTcQueue];
    float cap[kTcN];
    uint64_t full[kTcStages], empty[kTcStages], acc_full[2], acc_empty[2], done;
    uint32_t tmem_base;
    int abort_flag;
};

// (a, ia) < (b, ib) lexicographically
__device__ __forceinline__ bool lex_less(float a, int ia, float b, int ib) {
    return (a < b) || (a == b && ia < ib);
}

// Ascending bitonic sort of one (value, index) pair per lane.
__device__ __forceinline__ void warp_sort32(float &v, int &i, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const float ov = __shfl_xor_sync(kFull, v, j);
            const int oi = __shfl_xor_sync(kFull, i, j);
            const bool keep_min = (((lane & k) == 0) == ((lane & j) == 0));
            const bool take = keep_min ? lex_less(ov, oi, v, i) : lex_less(v, i, ov, oi);
            if (take) {
                v = ov;
                i = oi;
            }
        }
    }
}

// Merge a sorted batch (v, i) into the sorted list (ld, li), keeping the 32
// smallest: min of the list and the reversed batch is bitonic; 5 merge stages
// sort it.
__device__ __forceinline__ void warp_merge32(float &ld, int &li, float &thr, float cap, float v, int i,
                                             int lane) {
    const float rv = __shfl_sync(kFull, v, 31 - lane);
    const int ri = __shfl_sync(kFull, i, 31 - lane);
    if (lex_less(rv, ri, ld, li)) {
        ld = rv;
        li = ri;
    }
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const float ov = __shfl_xor_sync(kFull, ld, j);
        const int oi = __shfl_xor_sync(kFull, li, j);
        const bool take = ((lane & j) == 0) ? lex_less(ov, oi, ld, li) : lex_less(ld, li, ov, oi);
        if (take) {
            ld = ov;
            li = oi;
        }
    }
    thr = fminf(cap, __shfl_sync(kFull, ld, 31));
}

// Merges a query's pending queue (count entries) into its list, both in
// shared memory (list entry / queue entry = lane), and returns the new
// threshold.  Out of line, so the unrolled per-query loop stays small.
__device__ __noinline__ float flush_queue(float *lst_d, int *lst_i, const float *que_d, const int *que_i,
                                          int count, float cap, float thr, int lane) {
    float ld = lst_d[lane];
    int li = lst_i[lane];
    float v = lane < count ? que_d[lane] : INFINITY;
    int i = lane < count ? que_i[lane] : 0x7fffffff;
    warp_sort32(v, i, lane);
    warp_merge32(ld, li, thr, cap, v, i, lane);
    lst_d[lane] = ld;
    lst_i[lane] = li;
    __syncwarp();
    return thr;
}

// Merges one candidate per lane (the lanes set in fl) straight into a list.
__device__ __noinline__ float merge_lanes(float *lst_d, int *lst_i, float cap, float thr, float cv, int ci,
                                          unsigned fl, int lane) {
    float ld = lst_d[lane];
    int li = lst_i[lane];
    float v = ((fl >> lane) & 1u) ? cv : INFINITY;
    int i = ((fl >> lane) & 1u) ? ci : 0x7fffffff;
    warp_sort32(v, i, lane);
    warp_merge32(ld, li, thr, cap, v, i, lane);
    lst_d[lane] = ld;
    lst_i[lane] = li;
    __syncwarp();
    return thr;
}

// Merges a sorted list held by another warp into this list (both in shared memory).
__device__ __noinline__ float merge_smem(float *lst_d, int *lst_i, float cap, float thr, const float *od,
                                         const int *oi, int lane) {
    float ld = lst_d[lane];
    int li = lst_i[lane];
    const float cv = od[lane];
    const int ci = oi[lane];
    if (__any_sync(kFull, cv < thr)) warp_merge32(ld, li, thr, cap, cv, ci, lane);
    lst_d[lane] = ld;
    lst_i[lane] = li;
    __syncwarp();
    return thr;
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_search_tc(const float *__restrict__ qcoord, const float *__restrict__ qnorm, int Q, int d, int da,
                int K, const __nv_bfloat16 *__restrict__ etile, int ntiles, const float *__restrict__ thr0,
                int *__restrict__ cand_idx, float *__restrict__ cand_lb, int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(smem_raw);
    volatile int *abort_flag = &sm.abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int qbase = blockIdx.x * kTcN;

    // query tile -> shared memory, core-matrix layout
    for (int i = tid; i < kTcN * K; i += kTcThreads) {
        const int r = i / K, k = i - r * K;
        const int q = qbase + r;
        float v = 0.0f;
        if (q < Q) {
            if (k <= d)
                v = qcoord[(size_t)q * da + k];
            else if (k <= d + 3)
                v = 1.0f;
        }
        *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<unsigned char *>(sm.q) + core_offset(r, k, kTcN)) =
            __float2bfloat16_rn(v);
    }
    fence_proxy_async_smem();
    if (warp == kTcEpiWarps + 1) {
        tmem_alloc(&sm.tmem_base, kTcCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sm.acc_full[b], 1);
            mbar_init(&sm.acc_empty[b], kTcEpiWarps);
        }
        mbar_init(&sm.done, 1);
        fence_mbar_init();
        sm.abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    const uint32_t tile_bytes = (uint32_t)(kTcM * K * 2);

    if (warp == kTcEpiWarps) {
        // ---------------- producer ----------------
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < ntiles; ++t) {
                const int s = t % kTcStages;
                if (t >= kTcStages &&
                    !mbar_wait_or_abort(&sm.empty[s], (uint32_t)(((t / kTcStages) - 1) & 1), status, abort_flag))
                    break;
                mbar_expect_tx(&sm.full[s], tile_bytes);
                bulk_g2s(&sm.e[s][0], etile + (size_t)t * kTcM * K, tile_bytes, &sm.full[s]);
                issued = t + 1;
            }
            if (*abort_flag) {  // let the copies this thread issued land
                for (int t = issued - kTcStages; t < issued; ++t)
                    if (t >= 0) mbar_wait_bounded(&sm.full[t % kTcStages], (uint32_t)((t / kTcStages) & 1), status);
            }
        }
    } else if (warp == kTcEpiWarps + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kTcM, kTcN);
            const uint32_t lbo_e = (uint32_t)(kTcM / 8) * 128u, lbo_q = (uint32_t)(kTcN / 8) * 128u;
            const uint32_t qaddr = smem_u32(sm.q);
            const int nsuper = (ntiles + kTcSub - 1) / kTcSub;
            bool ok = true;
            for (int u = 0; u < nsuper && ok; ++u) {
                const int b = u & 1;
                if (u >= 2 && !mbar_wait_or_abort(&sm.acc_empty[b], (uint32_t)(((u >> 1) - 1) & 1), status,
                                                  abort_flag))
                    break;
                tc_fence_after();
                for (int sub = 0; sub < kTcSub; ++sub) {
                    const int t = u * kTcSub + sub;
                    if (t >= ntiles) break;
                    const int s = t % kTcStages;
                    if (!mbar_wait_or_abort(&sm.full[s], (uint32_t)((t / kTcStages) & 1), status, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t eaddr = smem_u32(&sm.e[s][0]);
                    const uint32_t dcol = tmem + (uint32_t)(b * kTcStageCols + sub * kTcN);
                    for (int ks = 0; ks < K / 16; ++ks) {
                        const uint64_t adesc = smem_desc(eaddr + ks * 2u * lbo_e, lbo_e, 128u);
                        const uint64_t bdesc = smem_desc(qaddr + ks * 2u * lbo_q, lbo_q, 128u);
                        mma_bf16(dcol, adesc, bdesc, idesc, ks > 0 ? 1u : 0u);
                    }
                    mma_commit(&sm.empty[s]);
                }
                if (ok) mma_commit(&sm.acc_full[b]);
            }
            // all MMAs issued by this thread have completed once `done` fires
            mma_commit(&sm.done);
            mbar_wait_bounded(&sm.done, 0, status);
        }
    } else {
        // ---------------- epilogue ----------------
        const int quarter = warp & 3, chunk = warp >> 2;
        // thr[j] starts at the warm-start bound (an upper bound on the query's
        // 32nd best value) and never rises above it while the list fills
        float thr[16];
        int qc[16];  // pending queue lengths (warp-uniform)
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int q = qbase + chunk * 16 + j;
            thr[j] = (thr0 && q < Q) ? thr0[q] : INFINITY;
            qc[j] = 0;
            sm.lst_d[warp][j][lane] = INFINITY;
            sm.lst_i[warp][j][lane] = -1;
            if (quarter == 0 && lane == 0) sm.cap[chunk * 16 + j] = thr[j];
        }
        __syncwarp();
        const unsigned lt_mask = (1u << lane) - 1u;
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        const int nsuper = (ntiles + kTcSub - 1) / kTcSub;
        for (int u = 0; u < nsuper; ++u) {
            const int b = u & 1;
            const bool ok = mbar_wait_or_abort(&sm.acc_full[b], (uint32_t)((u >> 1) & 1), status, abort_flag);
            if (!__all_sync(kFull, ok)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            for (int sub = 0; sub < kTcSub; ++sub) {
                const int t = u * kTcSub + sub;
                if (t >= ntiles) break;
                float v[16];
                tmem_ld16(tmem + lane_addr + (uint32_t)(b * kTcStageCols + sub * kTcN + chunk * 16), v);
                bool any = false;
#pragma unroll
                for (int j = 0; j < 16; ++j) any |= v[j] < thr[j];
                if (__any_sync(kFull, any)) {
                    const int nb = t * kTcM + quarter * 32;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        unsigned fl = __ballot_sync(kFull, v[j] < thr[j]);
                        if (fl) {
                            int c = __popc(fl);
                            if (qc[j] + c > kTcQueue) {  // make room: merge the queue first
                                thr[j] = flush_queue(&sm.lst_d[warp][j][0], &sm.lst_i[warp][j][0], &sm.que_d[warp][j][0],
                                                     &sm.que_i[warp][j][0], qc[j], sm.cap[chunk * 16 + j], thr[j],
                                                     lane);
                                qc[j] = 0;
                                fl = __ballot_sync(kFull, v[j] < thr[j]);
                                c = __popc(fl);
                            }
                            if (c > kTcQueue) {
                                thr[j] = merge_lanes(&sm.lst_d[warp][j][0], &sm.lst_i[warp][j][0],
                                                     sm.cap[chunk * 16 + j], thr[j], v[j], nb + lane, fl, lane);
                            } else if (c) {
                                if ((fl >> lane) & 1u) {
                                    const int pos = qc[j] + __popc(fl & lt_mask);
                                    sm.que_d[warp][j][pos] = v[j];
                                    sm.que_i[warp][j][pos] = nb + lane;
                                }
                                qc[j] += c;
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.acc_empty[b]);
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (qc[j])
                thr[j] = flush_queue(&sm.lst_d[warp][j][0], &sm.lst_i[warp][j][0], &sm.que_d[warp][j][0],
                                     &sm.que_i[warp][j][0], qc[j], sm.cap[chunk * 16 + j], thr[j], lane);
        // merge the four quarters' partial lists (all in shared memory)
        __syncthreads();  // (1) every quarter's lists are final
        if (quarter == 0 && !*abort_flag) {
            for (int j = 0; j < 16; ++j) {
                const int qq = chunk * 16 + j;
                float t = fminf(sm.cap[qq], sm.lst_d[warp][j][31]);
                for (int o = 1; o < 4; ++o)
                    t = merge_smem(&sm.lst_d[warp][j][0], &sm.lst_i[warp][j][0], sm.cap[qq], t,
                                   &sm.lst_d[warp + o][j][0], &sm.lst_i[warp + o][j][0], lane);
                const int q = qbase + qq;
                if (q < Q) {
                    cand_idx[(size_t)q * kTopK + lane] = sm.lst_i[warp][j][lane];
                    cand_lb[(size_t)q * kTopK + lane] = sm.lst_d[warp][j][lane] + qnorm[q];
                }
            }
        }
        __syncthreads();  // (2)
    }
    if (warp >= kTcEpiWarps) {
        __syncthreads();  // (1)
        __syncthreads();  // (2)
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kTcEpiWarps + 1) {
        __syncwarp();
        tmem_dealloc(tmem, kTcCols);
    }
}

// Warm start: the previous search's 32 windows of each query, scored in FP32
// for the new query vector.  Their largest p (plus a rounding margin of the
// BF16 search) is an upper bound on the query's 32nd best p, so the search
// only has to insert windows below it.  One warp per query.
__global__ void k_warm_threshold(const int *__restrict__ prev_idx, const float *__restrict__ qcoord,
                                 const float *__restrict__ qnorm, const __nv_bfloat16 *__restrict__ etile,
                                 const float *__restrict__ umax, int Q, int d, int da, int K, int N,
                                 float eps_scale, float *__restrict__ thr0) {
    const int lane = threadIdx.x & 31;
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= Q) return;
    const int n = prev_idx[(size_t)q * kTopK + lane];
    float p = INFINITY;
    if (n >= 0 && n < N) {
        // the same BF16 operands the tensor-core search multiplies
        const unsigned char *e = reinterpret_cast<const unsigned char *>(etile + (size_t)(n / kTcM) * kTcM * K);
        const int m = n % kTcM;
        p = 0.0f;
        for (int k = 0; k <= d + 3; ++k) {
            const float a = k <= d ? __bfloat162float(__float2bfloat16_rn(qcoord[(size_t)q * da + k])) : 1.0f;
            p = fmaf(a, __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(e + core_offset(m, k, kTcM))), p);
        }
    }
    float m = p;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    if (lane == 0) thr0[q] = m + eps_scale * (qnorm[q] + *umax);
}

// BF16 exemplar tiles in the MMA operand layout: rows = windows, K = (-2 y, -2 r, norm hi/mid/lo, 0...)
__global__ void k_pack_exemplar_bf16(const float *__restrict__ et, const float *__restrict__ enorm, int ntiles,
                                     int d, int da, int K, __nv_bfloat16 *__restrict__ out) {
    const long total = (long)ntiles * kTcM * K;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int t = (int)(i / (kTcM * K));
        const int rem = (int)(i - (long)t * kTcM * K);
        const int m = rem / K, k = rem - m * K;
        const float nrm = enorm[(size_t)t * kTcM + m];
        float v = 0.0f;
        if (k <= d) {
            v = et[((size_t)t * da + k) * kTcM + m];
        } else if (k <= d + 3) {
            const float hi = __bfloat162float(__float2bfloat16_rn(nrm));
            if (k == d + 1) {
                v = nrm;  // rounds to hi below
            } else if (isinf(nrm)) {
                v = 0.0f;
            } else {
                const float r1 = nrm - hi;
                const float mid = __bfloat162float(__float2bfloat16_rn(r1));
                v = (k == d + 2) ? r1 : (r1 - mid);
            }
        }
        *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<unsigned char *>(out + (size_t)t * kTcM * K) +
                                           core_offset(m, k, kTcM)) = __float2bfloat16_rn(v);
    }
}

// --- self-test: one 128 x N x K tile through the same descriptors, written back row-major ---
__global__ void __launch_bounds__(128) k_tc_selftest(const __nv_bfloat16 *__restrict__ A,
                                                     const __nv_bfloat16 *__restrict__ B, int N, int K,
                                                     float *__restrict__ D, int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    unsigned char *sa = sm_raw;
    unsigned char *sb = sm_raw + kTcM * K * 2;
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < kTcM * K; i += 128)
        *reinterpret_cast<__nv_bfloat16 *>(sa + core_offset(i / K, i % K, kTcM)) = A[i];
    for (int i = tid; i < N * K; i += 128)
        *reinterpret_cast<__nv_bfloat16 *>(sb + core_offset(i / K, i % K, N)) = B[i];
    fence_proxy_async_smem();
    if (warp == 0) {
        tmem_alloc(&tbase, 256);
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
        const uint32_t lbo_a = (uint32_t)(kTcM / 8) * 128u, lbo_b = (uint32_t)(N / 8) * 128u;
        for (int ks = 0; ks < K / 16; ++ks)
            mma_bf16(tmem, smem_desc(smem_u32(sa) + ks * 2u * lbo_a, lbo_a, 128u),
                     smem_desc(smem_u32(sb) + ks * 2u * lbo_b, lbo_b, 128u), idesc_bf16(kTcM, N), ks > 0 ? 1u : 0u);
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
    if (warp == 0) tmem_dealloc(tmem, 256);
}

}  // namespace

int tc_padded_k(int d) { return ((d + 4) + 15) / 16 * 16; }

void launch_warm_threshold(const int *prev_idx, const float *qcoord, const float *qnorm,
                           const __nv_bfloat16 *etile, const float *umax, int Q, int d, int da, int K, int N,
                           float eps_scale, float *thr0, cudaStream_t st) {
    count_launches(1);
    k_warm_threshold<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(prev_idx, qcoord, qnorm, etile, umax, Q, d, da,
                                                                   K, N, eps_scale, thr0);
}

void launch_pack_exemplar_bf16(const float *et, const float *enorm, int ntiles, int d, int da, int K,
                               __nv_bfloat16 *out, cudaStream_t st) {
    count_launches(1);
    k_pack_exemplar_bf16<<<152 * 4, 256, 0, st>>>(et, enorm, ntiles, d, da, K, out);
}

void launch_search_tc(const float *qcoord, const float *qnorm, int Q, int d, int da, int K,
                      const __nv_bfloat16 *etile, int ntiles, const float *thr0, int *cand_idx, float *cand_lb,
                      int *status, cudaStream_t st) {
    static bool attr = false;
    const size_t smem = sizeof(TcSmem) + 1024;
    if (!attr) {
        cudaFuncSetAttribute(k_search_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int grid = ceil_div(Q, kTcN);
    if (grid == 0) return;
    ProfScope ps(kProfSearchTc, st, 1);
    k_search_tc<<<grid, kTcThreads, smem, st>>>(qcoord, qnorm, Q, d, da, K, etile, ntiles, thr0, cand_idx,
                                                cand_lb, status);
}

pts_status tc_selftest(int N, int K, double *max_abs_err, double *max_abs_ref) {
    if (N < 16 || N > 256 || N % 16 || K < 16 || K > 128 || K % 16)
        return set_error(PTS_ERR_INVALID_ARG, "pts_tc_selftest: N in 16..256 and K in 16..128, multiples of 16");
    std::vector<__nv_bfloat16> hA((size_t)kTcM * K), hB((size_t)N * K);
    std::vector<float> fA(hA.size()), fB(hB.size());
    uint64_t z = 0x1234567ull;
    auto nextf = [&]() {
        z = z * 6364136223846793005ull + 1442695040888963407ull;
        return (float)((z >> 40) & 0xFFFF) / 32768.0f - 1.0f;
    };
    for (size_t i = 0; i < hA.size(); ++i) {
        hA[i] = __float2bfloat16_rn(nextf());
        fA[i] = __bfloat162float(hA[i]);
    }
    for (size_t i = 0; i < hB.size(); ++i) {
        hB[i] = __float2bfloat16_rn(nextf());
        fB[i] = __bfloat162float(hB[i]);
    }
    DevBuf<__nv_bfloat16> dA, dB;
    DevBuf<float> dD;
    DevBuf<int> dst;
    PTS_TRY(dA.ensure(hA.size(), "selftest A"));
    PTS_TRY(dB.ensure(hB.size(), "selftest B"));
    PTS_TRY(dD.ensure((size_t)kTcM * N, "selftest D"));
    PTS_TRY(dst.ensure(1, "selftest status"));
    PTS_CUDA_TRY(cudaMemcpy(dA.ptr, hA.data(), hA.size() * 2, cudaMemcpyHostToDevice));
    PTS_CUDA_TRY(cudaMemcpy(dB.ptr, hB.data(), hB.size() * 2, cudaMemcpyHostToDevice));
    PTS_CUDA_TRY(cudaMemset(dst.ptr, 0, sizeof(int)));
    const size_t smem = (size_t)(kTcM + N) * K * 2;
    cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launches(1);
    k_tc_selftest<<<1, 128, smem>>>(dA.ptr, dB.ptr, N, K, dD.ptr, dst.ptr);
    PTS_CUDA_TRY(cudaGetLastError());
    PTS_CUDA_TRY(cudaDeviceSynchronize());
    std::vector<float> hD((size_t)kTcM * N);
    int hst = 0;
    PTS_CUDA_TRY(cudaMemcpy(hD.data(), dD.ptr, hD.size() * 4, cudaMemcpyDeviceToHost));
    PTS_CUDA_TRY(cudaMemcpy(&hst, dst.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    double err = 0.0, ref_max = 0.0;
    for (int i = 0; i < kTcM; ++i)
        for (int j = 0; j < N; ++j) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += (double)fA[(size_t)i * K + k] * fB[(size_t)j * K + k];
            err = std::max(err, std::fabs(s - hD[(size_t)i * N + j]));
            ref_max = std::max(ref_max, std::fabs(s));
        }
    dA.release();
    dB.release();
    dD.release();
    dst.release();
    *max_abs_err = err;
    *max_abs_ref = ref_max;
    if (hst) return set_error(PTS_ERR_TIMEOUT, "pts_tc_selftest: MMA completion wait gave up");
    return PTS_OK;
}

}  // namespace pts
