// mlp_infer.cu -- inference of the cluster-proposal network fused into one kernel: per CTA 128
// queries go through the three layers on the tcgen05 tensor cores and only their 4 best
// clusters leave the SM (the logits are never written).
//
//   x  = the query's first 64 PCA coordinates (BF16, zero-padded)
//   h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2)      (BF16 operands of the next layer)
//   z  = W3 h2 + b3, top-4 of z                       (256 clusters per MMA chunk)
//
// Weights are pre-packed in the operand layout of tc_common.cuh (rows = outputs, 256 per
// chunk) and staged by 1-D bulk copies into one 128 KB buffer, each load issued as soon as the
// MMAs reading the previous contents have completed.  Accumulators: TMEM columns 0..255 and
// 256..511.  The arithmetic is that of the generic GEMM path (same BF16 operands, K-order,
// bias add and GELU), so the clusters match mlp_forward + k_top4.  16 warps: warp w reads TMEM
// lane quarter w % 4 (its 32 query rows) and column group w / 4 (64 of every 256 columns), so
// each epilogue runs 4 warps per SM sub-partition; in the last layer each warp keeps the top-4
// of its column group and the four lists of a row are merged at the end.
#include <math.h>

#include <algorithm>
#include <climits>

#include "tc_common.cuh"

namespace pts {
namespace {

constexpr int kIM = 128;    // queries per CTA
constexpr int kIThreads = 512;  // 16 warps: 4 lane quarters x 4 column groups
constexpr int kIH = kMlpH;  // 256
constexpr int kIChunk = 256;
constexpr uint32_t kW1Bytes = kIH * 64 * 2, kWBytes = kIChunk * kIH * 2;

struct InferSmem {
    alignas(1024) unsigned char x[kIM * 64 * 2];
    alignas(1024) unsigned char h[kIM * kIH * 2];
    alignas(1024) unsigned char w[kWBytes];
    uint64_t bar_w, bar_m;
    uint32_t tmem;
};

__device__ __forceinline__ float gelu_i(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }

// D[tmem_col + 64 cg .. +63] (rows = TMEM lanes of quarter qt) + bias -> gelu -> BF16 rows of
// the next A operand
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem, uint32_t col, const float *__restrict__ bias,
                                                unsigned char *h, int qt, int cg, int lane) {
    const int r = qt * 32 + lane;
    {
        const int cc = cg * 64;
        float v[64];
        tmem_ld64(tmem + ((uint32_t)(qt * 32) << 16) + col + (uint32_t)cc, v);
#pragma unroll
        for (int k8 = 0; k8 < 8; ++k8) {
            uint4 pk;
            uint32_t *pw = reinterpret_cast<uint32_t *>(&pk);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int j = 8 * k8 + 2 * t;
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(gelu_i(v[j] + bias[cc + j]),
                                                                gelu_i(v[j + 1] + bias[cc + j + 1]));
                pw[t] = *reinterpret_cast<const uint32_t *>(&b2);
            }
            *reinterpret_cast<uint4 *>(h + core_offset(r, cc + 8 * k8, kIM)) = pk;
        }
    }
}

// (z, id) before (z2, id2): larger logit, then smaller cluster id
__device__ __forceinline__ bool logit_before(float z, int id, float z2, int id2) {
    return z > z2 || (z == z2 && id < id2);
}

__global__ void __launch_bounds__(kIThreads, 1)
    k_mlp_infer(const float *__restrict__ qcoord, int Q, int d, int ldq, const __nv_bfloat16 *__restrict__ wp1,
                const float *__restrict__ b1, const __nv_bfloat16 *__restrict__ wp2, const float *__restrict__ b2,
                const __nv_bfloat16 *__restrict__ wp3, const float *__restrict__ b3p, int nchunk,
                int *__restrict__ top, int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    InferSmem &sm = *reinterpret_cast<InferSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int qt = warp & 3, cg = warp >> 2;  // TMEM lane quarter, column group
    const int row = qt * 32 + lane;           // this thread's query row in the epilogues
    const int q = blockIdx.x * kIM + row;
    // x tile: row tid (threads < 128), 64 values, 8 per 16-byte core-matrix row
    for (int k8 = 0; k8 < 8 && tid < kIM; ++k8) {
        uint4 pk;
        uint32_t *pw = reinterpret_cast<uint32_t *>(&pk);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int k = 8 * k8 + 2 * t;
            const long qx = (long)blockIdx.x * kIM + tid;
            const float a = (qx < Q && k < d) ? qcoord[(size_t)qx * ldq + k] : 0.0f;
            const float b = (qx < Q && k + 1 < d) ? qcoord[(size_t)qx * ldq + k + 1] : 0.0f;
            const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
            pw[t] = *reinterpret_cast<const uint32_t *>(&v);
        }
        *reinterpret_cast<uint4 *>(sm.x + core_offset(tid, 8 * k8, kIM)) = pk;
    }
    fence_proxy_async_smem();
    if (warp == 0) {
        tmem_alloc(&sm.tmem, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&sm.bar_w, 1);
        mbar_init(&sm.bar_m, 1);
        fence_mbar_init();
        mbar_expect_tx(&sm.bar_w, kW1Bytes);
        bulk_g2s(sm.w, wp1, kW1Bytes, &sm.bar_w);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;
    const uint32_t lbo_a = (kIM / 8) * 128u, lbo_w = (kIChunk / 8) * 128u;
    const uint32_t idesc = idesc_bf16(kIM, kIChunk);
    const uint32_t xa = smem_u32(sm.x), ha = smem_u32(sm.h), wa = smem_u32(sm.w);
    uint32_t pw = 0, pm = 0;
    bool ok = true;
    // layer 1: K = 64
    if (tid == 0) {
        ok = mbar_wait_bounded(&sm.bar_w, pw, status);
        tc_fence_after();
        for (int ks = 0; ks < 4 && ok; ++ks)
            mma_bf16(tmem, smem_desc(xa + ks * 2u * lbo_a, lbo_a, 128u), smem_desc(wa + ks * 2u * lbo_w, lbo_w, 128u),
                     idesc, ks > 0 ? 1u : 0u);
        mma_commit(&sm.bar_m);
    }
    pw ^= 1u;
    mbar_wait_bounded(&sm.bar_m, pm, status);
    pm ^= 1u;
    tc_fence_after();
    if (tid == 0) {  // W1 is no longer read
        mbar_expect_tx(&sm.bar_w, kWBytes);
        bulk_g2s(sm.w, wp2, kWBytes, &sm.bar_w);
    }
    hidden_epilogue(tmem, 0, b1, sm.h, qt, cg, lane);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // layer 2: K = 256, accumulator in columns 256..511
    if (tid == 0) {
        ok = mbar_wait_bounded(&sm.bar_w, pw, status) && ok;
        tc_fence_after();
        for (int ks = 0; ks < kIH / 16 && ok; ++ks)
            mma_bf16(tmem + 256u, smem_desc(ha + ks * 2u * lbo_a, lbo_a, 128u),
                     smem_desc(wa + ks * 2u * lbo_w, lbo_w, 128u), idesc, ks > 0 ? 1u : 0u);
        mma_commit(&sm.bar_m);
    }
    pw ^= 1u;
    mbar_wait_bounded(&sm.bar_m, pm, status);
    pm ^= 1u;
    tc_fence_after();
    if (tid == 0) {
        mbar_expect_tx(&sm.bar_w, kWBytes);
        bulk_g2s(sm.w, wp3, kWBytes, &sm.bar_w);
    }
    hidden_epilogue(tmem, 256u, b2, sm.h, qt, cg, lane);  // h1 is no longer read
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // layer 3 in chunks of 256 clusters, running top-4 per row (largest logit, smallest id on ties)
    float tv[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
    int ti[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
    for (int c = 0; c < nchunk; ++c) {
        const uint32_t dcol = (uint32_t)(c & 1) * 256u;
        if (tid == 0) {
            ok = mbar_wait_bounded(&sm.bar_w, pw, status) && ok;
            tc_fence_after();
            for (int ks = 0; ks < kIH / 16 && ok; ++ks)
                mma_bf16(tmem + dcol, smem_desc(ha + ks * 2u * lbo_a, lbo_a, 128u),
                         smem_desc(wa + ks * 2u * lbo_w, lbo_w, 128u), idesc, ks > 0 ? 1u : 0u);
            mma_commit(&sm.bar_m);
        }
        pw ^= 1u;
        mbar_wait_bounded(&sm.bar_m, pm, status);
        pm ^= 1u;
        tc_fence_after();
        if (tid == 0 && c + 1 < nchunk) {
            mbar_expect_tx(&sm.bar_w, kWBytes);
            bulk_g2s(sm.w, wp3 + (size_t)(c + 1) * kIChunk * kIH, kWBytes, &sm.bar_w);
        }
        {
            const int cc = cg * 64;  // ids rise along the scan: a strict test keeps the smaller id first
            float v[64];
            tmem_ld64(tmem + ((uint32_t)(qt * 32) << 16) + dcol + (uint32_t)cc, v);
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                const int id = c * kIChunk + cc + j;
                const float z = v[j] + b3p[id];
                if (z > tv[3]) {
                    if (z > tv[2]) {
                        tv[3] = tv[2];
                        ti[3] = ti[2];
                        if (z > tv[1]) {
                            tv[2] = tv[1];
                            ti[2] = ti[1];
                            if (z > tv[0]) {
                                tv[1] = tv[0];
                                ti[1] = ti[0];
                                tv[0] = z;
                                ti[0] = id;
                            } else {
                                tv[1] = z;
                                ti[1] = id;
                            }
                        } else {
                            tv[2] = z;
                            ti[2] = id;
                        }
                    } else {
                        tv[3] = z;
                        ti[3] = id;
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    // merge the column groups' lists of each row (the x tile is no longer read)
    float *mv = reinterpret_cast<float *>(sm.x);                // [3][128][4]
    int *mi = reinterpret_cast<int *>(sm.x) + 3 * kIM * 4;      // [3][128][4]
    if (cg > 0)
        for (int j = 0; j < 4; ++j) {
            mv[((cg - 1) * kIM + row) * 4 + j] = tv[j];
            mi[((cg - 1) * kIM + row) * 4 + j] = ti[j];
        }
    __syncthreads();
    if (cg == 0) {
        for (int g = 0; g < 3; ++g)
            for (int j = 0; j < 4; ++j) {
                float z = mv[(g * kIM + row) * 4 + j];
                int id = mi[(g * kIM + row) * 4 + j];
                for (int k = 0; k < 4; ++k)  // insert (z, id): swap down the sorted list
                    if (logit_before(z, id, tv[k], ti[k])) {
                        const float tz = tv[k];
                        const int tid2 = ti[k];
                        tv[k] = z;
                        ti[k] = id;
                        z = tz;
                        id = tid2;
                    }
            }
        if (q < Q)
            for (int j = 0; j < 4; ++j) top[(size_t)q * 4 + j] = ti[j] == INT_MAX ? 0 : ti[j];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        __syncwarp();
        tmem_dealloc(tmem, 512);
    }
}

// W [rows x K] row-major BF16 -> operand tiles of 256 rows (zero rows past `rows`)
__global__ void k_pack_weight(const __nv_bfloat16 *__restrict__ W, int rows, int K, int nchunk,
                              __nv_bfloat16 *__restrict__ out) {
    const long total = (long)nchunk * kIChunk * K;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int c = (int)(i / ((long)kIChunk * K));
        const int rem = (int)(i - (long)c * kIChunk * K);
        const int r = rem / K, k = rem - r * K;
        const int row = c * kIChunk + r;
        const __nv_bfloat16 v = row < rows ? W[(size_t)row * K + k] : __float2bfloat16_rn(0.0f);
        *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<unsigned char *>(out + (size_t)c * kIChunk * K) +
                                           core_offset(r, k, kIChunk)) = v;
    }
}

__global__ void k_pad_bias(const float *__restrict__ b, int C, int n, float *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = i < C ? b[i] : -INFINITY;
}

}  // namespace

pts_status mlp_pack_infer(MlpState &s, MlpInfer &f, cudaStream_t st) {
    const int C = s.C;
    f.nchunk = (C + kIChunk - 1) / kIChunk;
    PTS_TRY(f.wp1.ensure((size_t)kIChunk * 64, "packed W1"));
    PTS_TRY(f.wp2.ensure((size_t)kIChunk * kIH, "packed W2"));
    PTS_TRY(f.wp3.ensure((size_t)f.nchunk * kIChunk * kIH, "packed W3"));
    PTS_TRY(f.b3p.ensure((size_t)f.nchunk * kIChunk, "padded b3"));
    const long w1 = 0, b1 = w1 + (long)kIH * 64, w2 = b1 + kIH, b2 = w2 + (long)kIH * kIH, w3 = b2 + kIH,
               b3 = w3 + (long)C * kIH;
    count_launches(4);
    k_pack_weight<<<152, 256, 0, st>>>(s.wb.ptr + w1, kIH, 64, 1, f.wp1.ptr);
    k_pack_weight<<<152, 256, 0, st>>>(s.wb.ptr + w2, kIH, kIH, 1, f.wp2.ptr);
    k_pack_weight<<<152 * 2, 256, 0, st>>>(s.wb.ptr + w3, C, kIH, f.nchunk, f.wp3.ptr);
    k_pad_bias<<<8, 256, 0, st>>>(s.params.ptr + b3, C, f.nchunk * kIChunk, f.b3p.ptr);
    f.b1 = s.params.ptr + b1;
    f.b2 = s.params.ptr + b2;
    f.ready = 1;
    return PTS_OK;
}

void launch_mlp_top4(const MlpInfer &f, const float *qcoord, int Q, int d, int ldq, int *top, int *status,
                     cudaStream_t st) {
    if (Q <= 0) return;
    const size_t smem = sizeof(InferSmem) + 1024;
    set_smem_attr(reinterpret_cast<const void *>(k_mlp_infer), (int)smem);
    ProfScope ps(kProfMlp, st, 1);
    k_mlp_infer<<<ceil_div(Q, kIM), kIThreads, smem, st>>>(qcoord, Q, std::min(d, 64), ldq, f.wp1.ptr, f.b1, f.wp2.ptr, f.b2,
                                                     f.wp3.ptr, f.b3p.ptr, f.nchunk, top, status);
}

}  // namespace pts
