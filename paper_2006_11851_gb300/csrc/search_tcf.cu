// search_tcf.cu -- the nearest windows of Eq. 4 through a full-dimension FP16 tensor-core GEMM:
// every (query, window) score over all D components, the 32 best per query, which the caller
// re-ranks in FP32 and certifies against the GEMM's rounding bound (capi.cu); what stays
// uncertified takes the FP32 full-dimension pass.  Meant for levels whose PCA keeps too little of
// the variance for a useful PCA-space bound (large windows on a small exemplar).
//
// Score (Eq. 4 expanded around the exemplar mean mu, u = x - mu):
//   p(q, n) = ||u_n||^2 - 2 u_q . u_n,   d2(q, n) = ||u_q||^2 + p(q, n).
// The operands are s u rounded to FP16 with s = 2^12: |u| <= 1 stays far below the FP16 maximum
// and every |u| >= 2^-26 is a normal FP16 number after scaling.  The MMAs accumulate
// s^2 u_q . u_n in FP32; the epilogue forms p = ||u_n||^2 - (2 / s^2) acc with the FP32 norms.
//
// Layout: K-major core matrices (tc_common.cuh) with K = D rounded up to 64, zero past D.  The
// 64 columns of one ring stage are contiguous both in a 128-query block (16 KB) and in a
// 256-window tile (32 KB), so a stage is two bulk copies.  One CTA per (query block, window
// tile): M = 128, N = 256, one 256-column TMEM accumulator over all of K through a 4-stage ring;
// then each of the 4 warps reads its 32 TMEM lanes (queries) and writes their 256 scores.
//
// Warps (4): 0 bulk-copy producer (lane 0), 1 MMA issuer and TMEM owner (lane 0); then all four
// run the epilogue.  Every wait is bounded; on a timeout the kernel flags the status word,
// drains its copies, skips the scores and frees TMEM.
#include <algorithm>

#include "tc_common.cuh"

namespace pts {
namespace {

constexpr int kFQ = 128;        // queries per CTA (MMA M)
constexpr int kFN = 256;        // windows per tile (MMA N)
constexpr int kFK = 64;         // K per ring stage
constexpr int kFStages = 4;
constexpr int kFThreads = 128;
constexpr uint32_t kFAbytes = kFQ * kFK * 2;  // 16 KB
constexpr uint32_t kFBbytes = kFN * kFK * 2;  // 32 KB
constexpr float kFScale = 4096.0f;            // s
constexpr float kFUnscale2 = 1.0f / 8388608.0f;  // 2 / s^2 = 2^-23
constexpr float kFHalfMax = 65504.0f;         // largest finite FP16
constexpr unsigned kFullMask = 0xffffffffu;

struct TcfSmem {
    alignas(1024) unsigned char a[kFStages][kFAbytes];
    alignas(1024) unsigned char b[kFStages][kFBbytes];
    uint64_t full[kFStages], empty[kFStages], done;
    uint32_t tmem_base;
    int abort_flag;
};
static_assert(sizeof(TcfSmem) + 1024 <= 227 * 1024, "full-dimension search tiles exceed shared memory");

__global__ void __launch_bounds__(kFThreads, 1)
    k_search_tcf(const __half *__restrict__ qtile,  // [nqb][128 x K] core layout, s u_q
                 const __half *__restrict__ etile,  // [ntiles][256 x K] core layout, s u_n
                 int K, int Q, int N, int npad, const float *__restrict__ enorm,
                 float *__restrict__ score,  // [Q][npad]
                 int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcfSmem &sm = *reinterpret_cast<TcfSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    volatile int *abort_flag = &sm.abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int qb = blockIdx.x, t = blockIdx.y;
    const int nk = K / kFK;
    const unsigned char *qa = reinterpret_cast<const unsigned char *>(qtile) + (size_t)qb * kFQ * K * 2;
    const unsigned char *eb = reinterpret_cast<const unsigned char *>(etile) + (size_t)t * kFN * K * 2;
    if (warp == 1) {
        tmem_alloc(&sm.tmem_base, kFN);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kFStages; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        mbar_init(&sm.done, 1);
        fence_mbar_init();
        sm.abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    if (warp == 0 && lane == 0) {
        // ---------------- producer ----------------
        int issued = 0;
        for (int c = 0; c < nk; ++c) {
            const int s = c % kFStages;
            if (c >= kFStages &&
                !mbar_wait_or_abort(&sm.empty[s], (uint32_t)(((c / kFStages) - 1) & 1), status, abort_flag))
                break;
            mbar_expect_tx(&sm.full[s], kFAbytes + kFBbytes);
            bulk_g2s(sm.a[s], qa + (size_t)c * kFAbytes, kFAbytes, &sm.full[s]);
            bulk_g2s(sm.b[s], eb + (size_t)c * kFBbytes, kFBbytes, &sm.full[s]);
            issued = c + 1;
        }
        // every copy this thread issued has landed before the CTA may exit
        for (int c = std::max(0, issued - kFStages); c < issued; ++c)
            mbar_wait_bounded(&sm.full[c % kFStages], (uint32_t)((c / kFStages) & 1), status);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = idesc_f16(kFQ, kFN);
        const uint32_t lbo_a = (uint32_t)(kFQ / 8) * 128u, lbo_b = (uint32_t)(kFN / 8) * 128u;
        for (int c = 0; c < nk; ++c) {
            const int s = c % kFStages;
            if (!mbar_wait_or_abort(&sm.full[s], (uint32_t)((c / kFStages) & 1), status, abort_flag)) break;
            tc_fence_after();
            const uint32_t aaddr = smem_u32(sm.a[s]), baddr = smem_u32(sm.b[s]);
#pragma unroll
            for (int ks = 0; ks < kFK / 16; ++ks)
                mma_bf16(tmem, smem_desc(aaddr + ks * 2u * lbo_a, lbo_a, 128u),
                         smem_desc(baddr + ks * 2u * lbo_b, lbo_b, 128u), idesc, (c > 0 || ks > 0) ? 1u : 0u);
            mma_commit(&sm.empty[s]);
        }
        // `done` fires once every MMA this thread issued has completed
        mma_commit(&sm.done);
    }
    __syncwarp();
    // ---------------- epilogue: warp w holds TMEM lanes 32w .. 32w + 31 ----------------
    const bool got = mbar_wait_or_abort(&sm.done, 0, status, abort_flag);
    const bool ok = __all_sync(kFullMask, got) && !*abort_flag;
    tc_fence_after();
    if (ok) {
        const int q = qb * kFQ + warp * 32 + lane;
        const uint32_t laddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < kFN; c0 += 64) {
            float v[64];
            tmem_ld64(laddr + (uint32_t)c0, v);  // warp-collective
            if (q < Q) {
                const int n0 = t * kFN + c0;
                float4 *dst = reinterpret_cast<float4 *>(score + (size_t)q * npad + n0);
#pragma unroll
                for (int j4 = 0; j4 < 16; ++j4) {
                    float p[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int n = n0 + 4 * j4 + j;
                        p[j] = n < N ? fmaf(-kFUnscale2, v[4 * j4 + j], __ldg(enorm + n)) : INFINITY;
                    }
                    dst[j4] = make_float4(p[0], p[1], p[2], p[3]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tmem, kFN);
    }
}

// The exemplar's FP16 tiles: one thread per (window, 8-column group) of a 256-window tile,
// s (z - mu) of 8 consecutive components of the window rounded to FP16 as one 16-byte row of a
// core matrix; windows past N and components past D are zero.  Window n sits at (n / nx, n % nx)
// of the exemplar (We wide, C channels).  A value past the FP16 range sets *over, and the host
// then does not use the tiles.
__global__ void k_pack_exemplar_full16(const float *__restrict__ Z, int We, int C, int w, int nx, int N, int K,
                                       const float *__restrict__ mu, __half *__restrict__ out, long nthreads,
                                       int *__restrict__ over) {
    const int D = C * w * w, row = C * w;
    const int kg = K / 8;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nthreads; i += (long)gridDim.x * blockDim.x) {
        const long blk = i / ((long)kFN * kg);
        const int rem = (int)(i - blk * kFN * kg);
        const int k8 = rem / kFN, r = rem - k8 * kFN;  // r fastest: consecutive threads, consecutive 16 bytes
        const long n = blk * kFN + r;
        __align__(16) __half h[8];
        if (n < N) {
            const int y0 = (int)(n / nx), x0 = (int)(n % nx);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = k8 * 8 + j;
                float u = 0.0f;
                if (k < D) {
                    const int dy = k / row, e = k - dy * row;
                    u = (Z[((size_t)(y0 + dy) * We + x0) * C + e] - mu[k]) * kFScale;
                }
                if (!(fabsf(u) <= kFHalfMax)) {  // out of range (or NaN)
                    atomicOr(over, 1);
                    u = u > 0.0f ? kFHalfMax : -kFHalfMax;
                }
                h[j] = __float2half_rn(u);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = __float2half_rn(0.0f);
        }
        unsigned char *base = reinterpret_cast<unsigned char *>(out) + (size_t)blk * kFN * K * 2;
        *reinterpret_cast<uint4 *>(base + core_offset(r, k8 * 8, kFN)) = *reinterpret_cast<const uint4 *>(h);
    }
}

// One warp per query window: s (x - mu) of its D components rounded to FP16 into the query tile
// (lane l takes the 8-component groups l, l + 32, ...: one 16-byte core-matrix row each), and in
// the same pass ||x - mu||^2 in FP32, exact mode's slack tau and the GEMM's slack tau_tc (+inf
// when a value leaves the FP16 range), both per unit of ||u_q||^2 + max_n ||u_n||^2.
__global__ void __launch_bounds__(256) k_pack_queries_full16(const float *__restrict__ X, int Wo, int C, int w,
                                                             int stride, int qx, int Q, const float *__restrict__ mu,
                                                             int K, __half *__restrict__ qtile,
                                                             float *__restrict__ qnorm, float *__restrict__ tau,
                                                             float tau_scale, float *__restrict__ tau_tc,
                                                             float tc_scale, const float *__restrict__ umax) {
    const int lane = threadIdx.x & 31;
    const int q = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5);
    if (q >= Q) return;
    const int D = C * w * w, row = C * w;
    const int y0 = (q / qx) * stride, x0 = (q % qx) * stride;
    const float *src = X + ((size_t)y0 * Wo + x0) * C;
    unsigned char *tile = reinterpret_cast<unsigned char *>(qtile + (size_t)(q / kFQ) * kFQ * K);
    const int r = q % kFQ;
    float un = 0.0f;
    bool over = false;
    for (int g = lane; g < K / 8; g += 32) {
        __align__(16) __half h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = g * 8 + j;
            float u = 0.0f;
            if (k < D) {
                const int dy = k / row, e = k - dy * row;
                u = __ldg(src + (size_t)dy * Wo * C + e) - __ldg(mu + k);
                un = fmaf(u, u, un);
                u *= kFScale;
            }
            if (!(fabsf(u) <= kFHalfMax)) {  // out of range (or NaN)
                over = true;
                u = u > 0.0f ? kFHalfMax : -kFHalfMax;
            }
            h[j] = __float2half_rn(u);
        }
        *reinterpret_cast<uint4 *>(tile + core_offset(r, g * 8, kFQ)) = *reinterpret_cast<const uint4 *>(h);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) un += __shfl_xor_sync(kFullMask, un, o);
    over = __any_sync(kFullMask, over);
    if (lane == 0) {
        const float m = un + *umax;
        qnorm[q] = un;
        tau[q] = tau_scale * m;
        tau_tc[q] = over ? INFINITY : tc_scale * m;
    }
}


}  // namespace

int tcf_k(int D) { return (D + kFK - 1) / kFK * kFK; }
int tcf_tiles(int N) { return (N + kFN - 1) / kFN; }
int tcf_query_blocks(int Q) { return (Q + kFQ - 1) / kFQ; }

void launch_pack_exemplar_full16(const float *Z, int We, int C, int w, int nx, int N, const float *mu,
                                 __half *etile, int *over, cudaStream_t st) {
    const int K = tcf_k(C * w * w);
    const long n = (long)tcf_tiles(N) * kFN * (K / 8);
    count_launches(1);
    k_pack_exemplar_full16<<<(int)std::min<long>(ceil_div(n, 256), 152L * 16), 256, 0, st>>>(Z, We, C, w, nx, N, K, mu,
                                                                                           etile, n, over);
}


void launch_pack_queries_full16(const float *X, int Wo, int C, int w, int stride, int qx, int Q, const float *mu,
                                __half *qtile, float *qnorm, float *tau, float tau_scale, float *tau_tc, float tc_scale,
                                const float *umax, cudaStream_t st) {
    if (Q <= 0) return;
    const int K = tcf_k(C * w * w);
    // the last tile's rows past the last query stay zero
    if (Q % kFQ) cudaMemsetAsync(qtile + (size_t)(Q / kFQ) * kFQ * K, 0, sizeof(__half) * kFQ * K, st);
    count_launches(1);
    k_pack_queries_full16<<<ceil_div((long)Q * 32, 256), 256, 0, st>>>(X, Wo, C, w, stride, qx, Q, mu, K, qtile, qnorm,
                                                                       tau, tau_scale, tau_tc, tc_scale, umax);
}

void launch_gemm_tcf(const __half *qtile, int Q, int C, int w, const __half *etile, int N, const float *enorm,
                     const float *qnorm, float *score, int *cand_idx, float *cand_lb, int *status, cudaStream_t st) {
    if (Q <= 0) return;
    const int K = tcf_k(C * w * w);
    const int nqb = tcf_query_blocks(Q), nt = tcf_tiles(N);
    const size_t smem = sizeof(TcfSmem) + 1024;
    set_smem_attr(reinterpret_cast<const void *>(k_search_tcf), (int)smem);
    {
        ProfScope ps(kProfSearchTcf, st, 1);
        k_search_tcf<<<dim3(nqb, nt), kFThreads, smem, st>>>(qtile, etile, K, Q, N, nt * kFN, enorm, score, status);
    }
    launch_full_select_range(score, 1, nt * kFN, N, 0, Q, Q, qnorm, cand_idx, cand_lb, status, st);
}


}  // namespace pts
