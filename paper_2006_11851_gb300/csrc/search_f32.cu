// search_f32.cu -- exact-mode search phase (E-step, Eq. 4) in PCA space on
// FP32 SIMT cores.
//
// Every exemplar window n carries the search vector e_n = (y_n, r_n) (PCA
// coordinates and residual norm, section 2.2) and ||u_n||^2 = ||v_n - mu||^2;
// every query q carries a_q = (y_q, r_q) and ||u_q||^2.  For an orthonormal
// basis,
//   LB(q, n) = ||y_q - y_n||^2 + (r_q - r_n)^2
//            = ||u_q||^2 + ||u_n||^2 - 2 a_q . e_n  <=  ||x_q - z_n||^2,
// so LB is a lower bound on the full-dimension distance of Eq. 4.  The
// exemplar side is stored pre-multiplied by -2 so that one FMA chain starting
// at ||u_n||^2 gives p(q, n) = LB(q, n) - ||u_q||^2.
//
// Layout: exemplar tiles [tile][da][kBN] (one contiguous block per tile,
// brought into shared memory by one bulk copy), norms [tile*kBN] with +inf
// in the padding columns.  Each CTA owns kBQ = 64 queries (8 warps x 8 rows)
// and streams all exemplar tiles through a double buffer; each lane computes
// 8 rows x 4 consecutive columns.
//
//   k_search<false>  keeps per query the 32 smallest p (lexicographic in
//                    (p, n)), one sorted entry per lane, inserted with warp
//                    ballots only when a value beats the current 32nd;
//   k_search<true>   for the queries whose re-ranked best distance U_q was
//                    not certified, emits every pair with
//                    LB(q, n) <= U_q + tau_q (the only windows that can beat
//                    U_q), for exact evaluation.
#include <float.h>

#include "pts_internal.cuh"

namespace pts {
namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

struct SearchSmem {
    // sized for the maximum da; the kernel uses the first da rows
    float a[kMaxDA][kBQ];          // query vectors, transposed
    float e[2][kMaxDA][kBN];       // exemplar tiles (double buffer)
    float en[2][kBN];              // exemplar norms
    uint64_t bar[2];
    int abort_flag;
};

template <bool kRange>
__global__ void __launch_bounds__(kThreads, 2)
    k_search(const float *__restrict__ qcoord, const float *__restrict__ qnorm,
             const float *__restrict__ tau, int Q, int da, const int *__restrict__ fail_list,
             const unsigned int *__restrict__ fail_count,
             const unsigned long long *__restrict__ best64, const float *__restrict__ et,
             const float *__restrict__ enorm, int ntiles, int N, int *__restrict__ cand_idx,
             float *__restrict__ cand_lb, unsigned int *__restrict__ pair_count,
             uint2 *__restrict__ pairs, unsigned int pair_cap, int *__restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SearchSmem &sm = *reinterpret_cast<SearchSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int qbase = blockIdx.x * kBQ;
    int nq = Q;
    if (kRange) {
        nq = static_cast<int>(*fail_count);
        if (qbase >= nq) return;  // uniform for the whole CTA
    }

    // ---- query tile -> shared (transposed), per-row state ----
    for (int i = tid; i < kBQ * da; i += kThreads) {
        const int r = i / da, k = i - r * da;
        int q = -1;
        if (qbase + r < nq) q = kRange ? fail_list[qbase + r] : qbase + r;
        sm.a[k][r] = (q >= 0 && q < Q) ? qcoord[(size_t)q * da + k] : 0.0f;
    }
    const int row0 = warp * 8;
    int qrow[8];
    float lim[8];  // range: p <= lim  <=>  LB <= U + tau
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int q = -1;
        if (qbase + row0 + i < nq) q = kRange ? fail_list[qbase + row0 + i] : qbase + row0 + i;
        if (q >= Q) {
            atomicOr(status, kDevErrBounds);
            q = -1;
        }
        qrow[i] = q;
        lim[i] = -INFINITY;
        if (kRange && q >= 0) {
            const float U = __uint_as_float(static_cast<unsigned int>(best64[q] >> 32));
            lim[i] = U + tau[q] - qnorm[q];
        }
    }
    float ld[8], thr[8];
    int li[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        ld[i] = INFINITY;
        li[i] = -1;
        thr[i] = INFINITY;
    }

    const uint32_t tile_floats = static_cast<uint32_t>(da) * kBN;
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
        sm.abort_flag = 0;
    }
    __syncthreads();
    auto issue = [&](int t, int buf) {
        mbar_expect_tx(&sm.bar[buf], tile_floats * 4u + kBN * 4u);
        bulk_g2s(&sm.e[buf][0][0], et + (size_t)t * tile_floats, tile_floats * 4u, &sm.bar[buf]);
        bulk_g2s(&sm.en[buf][0], enorm + (size_t)t * kBN, kBN * 4u, &sm.bar[buf]);
    };
    if (tid == 0) {
        issue(0, 0);
        if (ntiles > 1) issue(1, 1);
    }

    for (int t = 0; t < ntiles; ++t) {
        const int buf = t & 1;
        if (tid == 0) {
            if (!mbar_wait_bounded(&sm.bar[buf], (t >> 1) & 1, status)) sm.abort_flag = 1;
        }
        __syncthreads();
        if (sm.abort_flag) {
            // let any copy still in flight land before shared memory goes away
            if (tid == 0) {
                if (t + 1 < ntiles) mbar_wait_bounded(&sm.bar[buf ^ 1], ((t + 1) >> 1) & 1, status);
            }
            __syncthreads();
            return;
        }

        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
        const float *eb = &sm.e[buf][0][lane * 4];
#pragma unroll 4
        for (int k = 0; k < da; ++k) {
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
        const float4 nv = *reinterpret_cast<const float4 *>(&sm.en[buf][lane * 4]);
        const float norms[4] = {nv.x, nv.y, nv.z, nv.w};
        const int nbase = t * kBN + lane * 4;

        if (!kRange) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float p = acc[i][j] + norms[j];
                    unsigned fl = __ballot_sync(kFull, p < thr[i]);
                    while (fl) {
                        const int src = __ffs(fl) - 1;
                        const float cd = __shfl_sync(kFull, p, src);
                        const int ci = t * kBN + src * 4 + j;
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
                        thr[i] = __shfl_sync(kFull, ld[i], 31);
                        fl &= ~(1u << src);
                        fl &= __ballot_sync(kFull, p < thr[i]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float p = acc[i][j] + norms[j];
                    const int n = nbase + j;
                    if (p <= lim[i] && n < N) {
                        const unsigned int slot = atomicAdd(pair_count, 1u);
                        if (slot < pair_cap) pairs[slot] = make_uint2((unsigned)qrow[i], (unsigned)n);
                    }
                }
            }
        }

        __syncthreads();  // all warps are done with buffer `buf`
        if (tid == 0 && t + 2 < ntiles) issue(t + 2, buf);
    }

    if (!kRange) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int q = qrow[i];
            if (q >= 0) {
                cand_idx[(size_t)q * kTopK + lane] = li[i];
                cand_lb[(size_t)q * kTopK + lane] = ld[i] + qnorm[q];
            }
        }
    }
}

size_t search_smem_bytes() { return sizeof(SearchSmem); }

}  // namespace

void launch_search_topk(const float *qcoord, const float *qnorm, int Q, int da, const float *et,
                        const float *enorm, int ntiles, int *cand_idx, float *cand_lb, int *status,
                        cudaStream_t st) {
    static bool attr = false;
    const size_t smem = search_smem_bytes();
    if (!attr) {
        cudaFuncSetAttribute(k_search<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int grid = ceil_div(Q, kBQ);
    if (grid == 0) return;
    ProfScope ps(kProfSearchTopk, st, 1);
    k_search<false><<<grid, kThreads, smem, st>>>(qcoord, qnorm, nullptr, Q, da, nullptr, nullptr,
                                                  nullptr, et, enorm, ntiles, 0, cand_idx, cand_lb,
                                                  nullptr, nullptr, 0, status);
}

void launch_search_range(const float *qcoord, const float *qnorm, const float *tau, int Q, int da,
                         const int *fail_list, const unsigned int *fail_count,
                         const unsigned long long *best64, const float *et, const float *enorm,
                         int ntiles, int N, unsigned int *pair_count, uint2 *pairs,
                         unsigned int pair_cap, int *status, cudaStream_t st) {
    static bool attr = false;
    const size_t smem = search_smem_bytes();
    if (!attr) {
        cudaFuncSetAttribute(k_search<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int grid = ceil_div(Q, kBQ);
    if (grid == 0) return;
    ProfScope ps(kProfSearchRange, st, 1);
    k_search<true><<<grid, kThreads, smem, st>>>(qcoord, qnorm, tau, Q, da, fail_list, fail_count,
                                                 best64, et, enorm, ntiles, N, nullptr, nullptr,
                                                 pair_count, pairs, pair_cap, status);
}

}  // namespace pts
