// gemm_tc.cu -- general BF16 GEMM on the tcgen05 tensor cores for the proposal network:
//   C[M x N] = A[M x K] * B[N x K]^T  (+ bias[n], optional GELU), FP32 accumulation in TMEM.
// A and B are row-major with K contiguous (both "K-major").  A CTA computes a 128 x 128 tile:
// 16-byte cp.async copies move each 8-element row segment straight into its place in the
// core-matrix operand layout (tc_common.cuh) through a 2-stage ring of 64-wide K chunks; one
// thread issues 4 MMAs (K = 16 each) per chunk and commits them to the chunk's mbarrier, which
// also tells the copiers when the stage may be overwritten.  The epilogue reads the 128 x 128
// FP32 accumulator back with tcgen05.ld (each warp its 32 TMEM lanes) and writes FP32 and/or
// BF16 results.  Ragged edges are zero-filled on load and masked on store.
#include <math.h>

#include <algorithm>
#include <vector>

#include "tc_common.cuh"

namespace pts {
namespace {

constexpr int kGM = 128, kGN = 128, kGK = 64;
constexpr int kGThreads = 128;

struct GemmSmem {
    alignas(128) __nv_bfloat16 a[2][kGM * kGK];
    alignas(128) __nv_bfloat16 b[2][kGN * kGK];
    uint64_t bar[2];
    uint32_t tmem;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
    const int sz = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(sz)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ float gelu_f(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }

// stage (rows x 64) of a K-major matrix into the core-matrix layout; rows/cols beyond the
// matrix are zero-filled (K must be a multiple of 8 so 16-byte segments never straddle the end)
__device__ __forceinline__ void load_tile(unsigned char *dst, const __nv_bfloat16 *src, int ld, int rows_total,
                                          int row0, int k0, int K, int tid) {
    for (int c = tid; c < 128 * (kGK / 8); c += kGThreads) {
        const int r = c / (kGK / 8), kk = (c % (kGK / 8)) * 8;
        const int gr = row0 + r, gk = k0 + kk;
        const bool valid = gr < rows_total && gk < K;
        const __nv_bfloat16 *g = valid ? src + (size_t)gr * ld + gk : src;
        cp_async16(dst + core_offset(r, kk, 128), g, valid);
    }
}

__global__ void __launch_bounds__(kGThreads)
    k_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int lda,
                const __nv_bfloat16 *__restrict__ B, int ldb, const float *__restrict__ bias, int gelu,
                float *__restrict__ Cf, __nv_bfloat16 *__restrict__ Cb, float *__restrict__ Cpre, int ldc,
                int *__restrict__ status) {
    extern __shared__ __align__(128) unsigned char gsm_raw[];
    GemmSmem &sm = *reinterpret_cast<GemmSmem *>(gsm_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kGM, n0 = blockIdx.x * kGN;
    if (warp == 0) {
        tmem_alloc(&sm.tmem, 128);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;
    const int nk = (K + kGK - 1) / kGK;
    const uint32_t idesc = idesc_bf16(kGM, kGN);
    const uint32_t lbo = 16u * 128u;  // (128 rows / 8) core matrices per K slab

    load_tile(reinterpret_cast<unsigned char *>(sm.a[0]), A, lda, M, m0, 0, K, tid);
    load_tile(reinterpret_cast<unsigned char *>(sm.b[0]), B, ldb, N, n0, 0, K, tid);
    cp_async_commit();
    bool ok = true;
    for (int kc = 0; kc < nk; ++kc) {
        const int s = kc & 1;
        if (kc + 1 < nk) {
            // stage s^1 was read by the MMAs of chunk kc-1: wait for them before overwriting
            if (kc >= 1 && !mbar_wait_bounded(&sm.bar[s ^ 1], (uint32_t)(((kc - 1) >> 1) & 1), status)) ok = false;
            load_tile(reinterpret_cast<unsigned char *>(sm.a[s ^ 1]), A, lda, M, m0, (kc + 1) * kGK, K, tid);
            load_tile(reinterpret_cast<unsigned char *>(sm.b[s ^ 1]), B, ldb, N, n0, (kc + 1) * kGK, K, tid);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && ok) {
            tc_fence_after();
            const uint32_t abase = smem_u32(sm.a[s]), bbase = smem_u32(sm.b[s]);
            for (int ks = 0; ks < kGK / 16; ++ks)
                mma_bf16(tmem, smem_desc(abase + ks * 2u * lbo, lbo, 128u), smem_desc(bbase + ks * 2u * lbo, lbo, 128u),
                         idesc, (kc > 0 || ks > 0) ? 1u : 0u);
            mma_commit(&sm.bar[s]);
        }
    }
    // the last chunk's commit covers every MMA issued before it
    const int last = nk - 1;
    mbar_wait_bounded(&sm.bar[last & 1], (uint32_t)((last >> 1) & 1), status);
    tc_fence_after();
    const int row = m0 + warp * 32 + lane;
    for (int c = 0; c < kGN; c += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        if (row < M) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = n0 + c + j;
                if (col >= N) continue;
                float x = v[j] + (bias ? bias[col] : 0.0f);
                if (Cpre) Cpre[(size_t)row * ldc + col] = x;
                if (gelu) x = gelu_f(x);
                if (Cf) Cf[(size_t)row * ldc + col] = x;
                if (Cb) Cb[(size_t)row * ldc + col] = __float2bfloat16_rn(x);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        __syncwarp();
        tmem_dealloc(tmem, 128);
    }
}

// out[c][r] = in[r][c] for a rows x cols BF16 matrix (32 x 32 tiles through shared memory)
__global__ void k_transpose_bf16(const __nv_bfloat16 *__restrict__ in, int rows, int cols,
                                 __nv_bfloat16 *__restrict__ out) {
    __shared__ __nv_bfloat16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * cols + c] : __float2bfloat16_rn(0.0f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[(size_t)c * rows + r] = t[threadIdx.x][i];
    }
}

__global__ void k_f32_to_bf16(const float *__restrict__ in, long n, __nv_bfloat16 *__restrict__ out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

}  // namespace

void launch_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                      const float *bias, int gelu, float *Cf, __nv_bfloat16 *Cb, float *Cpre, int ldc, int *status,
                      cudaStream_t st) {
    const size_t smem = sizeof(GemmSmem) + 128;
    set_smem_attr(reinterpret_cast<const void *>(k_gemm_bf16), (int)smem);
    dim3 grid(ceil_div(N, kGN), ceil_div(M, kGM));
    ProfScope ps(kProfMlp, st, 1);
    k_gemm_bf16<<<grid, kGThreads, smem, st>>>(M, N, K, A, lda, B, ldb, bias, gelu, Cf, Cb, Cpre, ldc, status);
}

void launch_transpose_bf16(const __nv_bfloat16 *in, int rows, int cols, __nv_bfloat16 *out, cudaStream_t st) {
    count_launches(1);
    k_transpose_bf16<<<dim3(ceil_div(cols, 32), ceil_div(rows, 32)), dim3(32, 8), 0, st>>>(in, rows, cols, out);
}

void launch_f32_to_bf16(const float *in, long n, __nv_bfloat16 *out, cudaStream_t st) {
    count_launches(1);
    k_f32_to_bf16<<<152 * 4, 256, 0, st>>>(in, n, out);
}

pts_status gemm_selftest(int M, int N, int K, double *max_rel_err) {
    if (M < 1 || N < 1 || K < 8 || K % 8)
        return set_error(PTS_ERR_INVALID_ARG, "pts_gemm_selftest: need M, N >= 1 and K a multiple of 8");
    std::vector<__nv_bfloat16> hA((size_t)M * K), hB((size_t)N * K);
    std::vector<float> fA(hA.size()), fB(hB.size()), hbias(N);
    uint64_t z = 0x9E37ull;
    auto nextf = [&]() {
        z = z * 6364136223846793005ull + 1442695040888963407ull;
        return (float)((z >> 40) & 0xFFFF) / 32768.0f - 1.0f;
    };
    for (size_t i = 0; i < hA.size(); ++i) fA[i] = __bfloat162float(hA[i] = __float2bfloat16_rn(nextf()));
    for (size_t i = 0; i < hB.size(); ++i) fB[i] = __bfloat162float(hB[i] = __float2bfloat16_rn(nextf()));
    for (int j = 0; j < N; ++j) hbias[j] = nextf();
    DevBuf<__nv_bfloat16> dA, dB;
    DevBuf<float> dC, dP, dbias;
    DevBuf<int> dst;
    PTS_TRY(dA.ensure(hA.size(), "A"));
    PTS_TRY(dB.ensure(hB.size(), "B"));
    PTS_TRY(dC.ensure((size_t)M * N, "C"));
    PTS_TRY(dP.ensure((size_t)M * N, "pre"));
    PTS_TRY(dbias.ensure(N, "bias"));
    PTS_TRY(dst.ensure(1, "status"));
    PTS_CUDA_TRY(cudaMemcpy(dA.ptr, hA.data(), hA.size() * 2, cudaMemcpyHostToDevice));
    PTS_CUDA_TRY(cudaMemcpy(dB.ptr, hB.data(), hB.size() * 2, cudaMemcpyHostToDevice));
    PTS_CUDA_TRY(cudaMemcpy(dbias.ptr, hbias.data(), N * 4, cudaMemcpyHostToDevice));
    PTS_CUDA_TRY(cudaMemset(dst.ptr, 0, sizeof(int)));
    launch_gemm_bf16(M, N, K, dA.ptr, K, dB.ptr, K, dbias.ptr, 1, dC.ptr, nullptr, dP.ptr, N, dst.ptr, 0);
    PTS_CUDA_TRY(cudaGetLastError());
    PTS_CUDA_TRY(cudaDeviceSynchronize());
    std::vector<float> hP((size_t)M * N), hC((size_t)M * N);
    int hst = 0;
    PTS_CUDA_TRY(cudaMemcpy(hP.data(), dP.ptr, hP.size() * 4, cudaMemcpyDeviceToHost));
    PTS_CUDA_TRY(cudaMemcpy(hC.data(), dC.ptr, hC.size() * 4, cudaMemcpyDeviceToHost));
    PTS_CUDA_TRY(cudaMemcpy(&hst, dst.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    double err = 0.0;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < N; ++j) {
            double s = hbias[j];
            double sa = std::fabs(hbias[j]);
            for (int k = 0; k < K; ++k) {
                s += (double)fA[(size_t)i * K + k] * fB[(size_t)j * K + k];
                sa += std::fabs((double)fA[(size_t)i * K + k] * fB[(size_t)j * K + k]);
            }
            err = std::max(err, std::fabs(s - hP[(size_t)i * N + j]) / std::max(sa, 1e-30));
            const double g = 0.5 * s * (1.0 + std::erf(s / std::sqrt(2.0)));
            err = std::max(err, std::fabs(g - hC[(size_t)i * N + j]) / std::max(std::fabs(g) + 1e-3, sa * 1e-3));
        }
    *max_rel_err = err;
    if (hst) return set_error(PTS_ERR_TIMEOUT, "pts_gemm_selftest: a completion wait gave up");
    return PTS_OK;
}

}  // namespace pts
