// project_tc.cu -- the FP16 search's query projection (section 2.2) on the tcgen05 tensor cores.
//
// For each query window v on the stride grid of the image:
//   u = v - mu,  y = B^T u  (the d <= 124 components the FP16 search ranks by),
//   ||u||^2 and r = sqrt(max(0, ||u||^2 - ||y||^2)),
// written as the tensor-core search's FP16 query rows (y, r, 1, 1, 1, 0, ...) in the core-matrix
// layout, with ||u||^2 and tau = tau_scale * (||u||^2 + max_n ||u_n||^2) -- the outputs of the
// SIMT projection's FP16 layout (project.cu).
//
// The contraction runs on FP16 operands with FP32 accumulation, at close to FP32 accuracy: each
// value x is split as x = x_hi + x_lo with x_hi of 11 significant bits (exact in FP16) and x_lo
// rounded to FP16 (22 significant bits together, or an absolute 2^-25 below |x| = 2^-3, where x_lo
// is an FP16 subnormal; the window side by Veltkamp's splitting in FP32,
// t = 8193 x, x_hi = t - (t - x), the basis side by rounding, x_hi = fp16(x)), and u . b is
// accumulated as u_hi b_hi + u_lo b_hi + u_hi b_lo; every FP16 product is exact in FP32, and the
// dropped u_lo b_lo is about 2^-22 of |u b|.  The result is
// rounded to FP16 for the search, so the split only has to keep the coordinates far more accurate
// than that rounding.  Components past the FP16 range (|u_i| >= 65520) make the row non-finite,
// as they would the FP16 query row itself.
//
// A CTA owns 128 windows (the MMA's M) and all 128 output columns (N; columns >= d have zero
// basis rows).  The window vector runs in chunks of 32 elements through two stages: 256 threads
// gather the chunk's 128 x 32 centred values straight from the HWC image (two threads per window,
// 8 consecutive elements each, split and stored as 16-byte rows of core matrices), one bulk copy
// brings the chunk's prepacked basis slices (hi and lo, built once per index), and one thread
// issues the 2 x 3 MMAs (K = 16) and commits them to the stage's mbarrier, which frees the stage
// two chunks later.  The 128 x 128 FP32 accumulator stays in TMEM (128 columns); the epilogue
// reads it with tcgen05.ld, warp w taking TMEM lanes 32 (w % 4) .. + 31 and columns
// 64 (w / 4) .. + 63, and writes each row's FP16 values as 16-byte stores.  A grid of few query
// blocks also splits the window vector into chunk ranges (blockIdx.y): each CTA then writes its
// range's FP32 partial coordinates and ||u||^2, and k_project_tc_finish adds the ranges in order
// and writes the rows.
#include <math.h>

#include <algorithm>

#include "tc_common.cuh"

namespace pts {
namespace {

constexpr int kPR = 128;                            // windows per CTA (the MMA's M)
constexpr int kPC = 32;                             // window-vector elements per chunk
constexpr int kPThreads = 256;
constexpr uint32_t kPTile = kPR * kPC * 2;          // one 128 x 32 FP16 operand tile (8 KB)
constexpr uint32_t kPLbo = (kPR / 8) * 128;         // bytes between core matrices adjacent along K
constexpr int kPartRow = 132;                       // a window's partial sums: 128 coordinates, ||u||^2, padding

struct ProjTcSmem {
    alignas(128) unsigned char a[2][2][kPTile];  // [stage][hi, lo] window slices
    alignas(128) unsigned char b[2][2][kPTile];  // [stage][hi, lo] basis slices
    uint64_t b_full[2];                          // the stage's basis slices landed
    uint64_t mma_done[2];                        // the stage's MMAs completed (the stage is free)
    float un[2][kPR];                            // ||u||^2, the two staging threads of each window
    float yn[2][kPR];                            // ||y||^2, the two column halves of each window
    uint32_t tmem;
};

// 32 TMEM lanes x 16 consecutive 32-bit columns, the wait inside the same asm statement
__device__ __forceinline__ void tmem_ld16w(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// x = hi + lo for 8 values -> two 16-byte rows: Veltkamp's splitting with factor 2^13 + 1 leaves
// hi with 11 significant bits (exact in FP16 inside its normal range) and lo = x - hi exact in
// FP32; the explicit roundings keep the compiler from fusing the steps
__device__ __forceinline__ void split8(const float (&v)[8], uint4 &hi, uint4 &lo) {
    float h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float t = __fmul_rn(v[i], 8193.0f);
        h[i] = __fsub_rn(t, __fsub_rn(t, v[i]));
        l[i] = __fsub_rn(v[i], h[i]);
    }
    hi = make_uint4(pack_half2(h[0], h[1]), pack_half2(h[2], h[3]), pack_half2(h[4], h[5]), pack_half2(h[6], h[7]));
    lo = make_uint4(pack_half2(l[0], l[1]), pack_half2(l[2], l[3]), pack_half2(l[4], l[5]), pack_half2(l[6], l[7]));
}

__global__ void __launch_bounds__(kPThreads, 2)
    k_project_tc(const float *__restrict__ img, int img_vec, int W, int C, int w, int stride, int qx_n, int Qn,
                 const float *__restrict__ mu, const unsigned char *__restrict__ basis16, int d, int ktile,
                 __half *__restrict__ tile16, float *__restrict__ out_norm, float *__restrict__ out_tau,
                 float tau_scale, const float *__restrict__ umax, int *__restrict__ status, int kc_per,
                 float *__restrict__ part) {
    extern __shared__ __align__(128) unsigned char ptc_raw[];
    ProjTcSmem &sm = *reinterpret_cast<ProjTcSmem *>(ptc_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = C * w, D = row * w, W3 = C * W;
    // this CTA's chunks of the window vector (blockIdx.y splits them when part is given)
    const int c_begin = blockIdx.y * kc_per;
    const int nk = min((D + kPC - 1) / kPC - c_begin, kc_per);
    const long q0 = (long)blockIdx.x * kPR;
    if (warp == 0) {
        tmem_alloc(&sm.tmem, 128);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&sm.b_full[s], 1);
            mbar_init(&sm.mma_done[s], 1);
        }
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;
    // staging role: window r of the block; half h takes the 8-element groups h and h + 2 of a chunk
    const int r = tid & (kPR - 1), h = tid >> 7;
    const long q = q0 + r;
    const bool valid = q < Qn;
    int base = 0;
    if (valid) {
        const int qy = (int)(q / qx_n), qx = (int)(q - (long)qy * qx_n);
        base = (qy * stride * W + qx * stride) * C;
    }
    const float *const src = img + base;
    // The two groups' first elements (offset e in their window row, image offset off), advanced
    // 32 elements per chunk.  When the window row (C w floats) is a multiple of 8 long, a group
    // never crosses a row: its 8 floats are contiguous, read as float4 or float2 where the
    // window's and the rows' offsets allow, and the mean as two float4.
    const bool rows8 = (row & 7) == 0;
    const int vec = !rows8                                       ? 0
                    : (((base | W3) & 3) == 0 && img_vec == 4)   ? 4
                    : (((base | W3) & 1) == 0 && img_vec >= 2) ? 2
                                                                 : 1;
    int ge[2], goff[2];
#pragma unroll
    for (int gi = 0; gi < 2; ++gi) {
        const int k = c_begin * kPC + (h + 2 * gi) * 8, dy = k / row;
        ge[gi] = k - dy * row;
        goff[gi] = dy * W3 + ge[gi];
    }
    const uint32_t idesc = idesc_f16(kPR, 128);
    float un = 0.0f;
    bool ok = true;
    // chunk c of this CTA (absolute chunk c_begin + c) in stage s = c % 2
    for (int c = 0; c < nk; ++c) {
        const int s = c & 1;
        // the stage was last read by the MMAs of chunk c - 2 (after a wait gave up, the thread
        // waits no more: the status word already carries the timeout)
        if (c >= 2 && ok && !mbar_wait_bounded(&sm.mma_done[s], (uint32_t)(((c - 2) >> 1) & 1), status)) ok = false;
        if (tid == 0 && ok) {
            mbar_expect_tx(&sm.b_full[s], 2 * kPTile);
            bulk_g2s(sm.b[s][0], basis16 + (size_t)(c_begin + c) * 2 * kPTile, 2 * kPTile, &sm.b_full[s]);
        }
#pragma unroll
        for (int gi = 0; gi < 2; ++gi) {
            const int g = h + 2 * gi;
            const int k0 = (c_begin + c) * kPC + g * 8;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = 0.0f;
            if (valid && k0 < D) {
                const float *p = src + goff[gi];
                if (vec == 4) {
                    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
                    const float4 b = __ldg(reinterpret_cast<const float4 *>(p + 4));
                    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
                } else if (vec == 2) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 a = __ldg(reinterpret_cast<const float2 *>(p + 2 * i));
                        v[2 * i] = a.x, v[2 * i + 1] = a.y;
                    }
                } else if (vec == 1) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = __ldg(p + i);
                } else {  // the group may cross window rows and the vector's end
                    int e = ge[gi], off = goff[gi];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        if (k0 + i < D) v[i] = __ldg(src + off);
                        if (++e == row) {
                            e = 0;
                            off += W3 - row + 1;
                        } else {
                            ++off;
                        }
                    }
                }
                if (rows8) {
                    const float4 m0 = __ldg(reinterpret_cast<const float4 *>(mu + k0));
                    const float4 m1 = __ldg(reinterpret_cast<const float4 *>(mu + k0 + 4));
                    v[0] -= m0.x, v[1] -= m0.y, v[2] -= m0.z, v[3] -= m0.w;
                    v[4] -= m1.x, v[5] -= m1.y, v[6] -= m1.z, v[7] -= m1.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (k0 + i < D) v[i] -= __ldg(mu + k0 + i);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) un = fmaf(v[i], v[i], un);
            }
            // the same group of the next chunk, 32 elements on
            int e = ge[gi] + kPC, off = goff[gi] + kPC;
            while (e >= row) {
                e -= row;
                off += W3 - row;
            }
            ge[gi] = e;
            goff[gi] = off;
            uint4 hi, lo;
            split8(v, hi, lo);
            const uint32_t o = core_offset(r, g * 8, kPR);
            *reinterpret_cast<uint4 *>(sm.a[s][0] + o) = hi;
            *reinterpret_cast<uint4 *>(sm.a[s][1] + o) = lo;
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && ok) {
            ok = mbar_wait_bounded(&sm.b_full[s], (uint32_t)((c >> 1) & 1), status);
            if (ok) {
                tc_fence_after();
                const uint32_t ah = smem_u32(sm.a[s][0]), al = smem_u32(sm.a[s][1]);
                const uint32_t bh = smem_u32(sm.b[s][0]), bl = smem_u32(sm.b[s][1]);
#pragma unroll
                for (int ks = 0; ks < kPC / 16; ++ks) {
                    const uint32_t o = (uint32_t)ks * 2u * kPLbo;
                    mma_bf16(tmem, smem_desc(ah + o, kPLbo, 128u), smem_desc(bh + o, kPLbo, 128u), idesc,
                             (c > 0 || ks > 0) ? 1u : 0u);
                    mma_bf16(tmem, smem_desc(al + o, kPLbo, 128u), smem_desc(bh + o, kPLbo, 128u), idesc, 1u);
                    mma_bf16(tmem, smem_desc(ah + o, kPLbo, 128u), smem_desc(bl + o, kPLbo, 128u), idesc, 1u);
                }
                mma_commit(&sm.mma_done[s]);
            }
        }
    }
    sm.un[h][r] = un;
    // the last chunk's commit covers every MMA issued before it
    const int last = nk - 1;
    if (ok && !mbar_wait_bounded(&sm.mma_done[last & 1], (uint32_t)((last >> 1) & 1), status)) ok = false;
    tc_fence_after();
    __syncthreads();
    // epilogue: the accumulator row of window rr, columns 64 half .. 64 half + 63
    const int quarter = warp & 3, half = warp >> 2;
    const int rr = quarter * 32 + lane;
    const long qq = q0 + rr;
    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 64);
    if (part) {
        // split vector: this range's partial coordinates and ||u||^2, [y][q][kPartRow]
        float *const pr = part + ((size_t)blockIdx.y * Qn + qq) * kPartRow;
#pragma unroll
        for (int c16 = 0; c16 < 4; ++c16) {
            float v[16];
            tmem_ld16w(taddr + (uint32_t)(c16 * 16), v);
            if (qq < Qn && ok)
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    *reinterpret_cast<float4 *>(pr + half * 64 + c16 * 16 + j) =
                        make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
        if (qq < Qn && half == 0) pr[128] = sm.un[0][rr] + sm.un[1][rr];
    } else {
    float yn = 0.0f;
#pragma unroll
    for (int c16 = 0; c16 < 4; ++c16) {
        float v[16];
        tmem_ld16w(taddr + (uint32_t)(c16 * 16), v);
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (half * 64 + c16 * 16 + j < d) yn = fmaf(v[j], v[j], yn);
    }
    sm.yn[half][rr] = yn;
    __syncthreads();
    const float u2 = sm.un[0][rr] + sm.un[1][rr];
    const float res = sqrtf(fmaxf(u2 - (sm.yn[0][rr] + sm.yn[1][rr]), 0.0f));
    unsigned char *const t = reinterpret_cast<unsigned char *>(tile16 + (size_t)blockIdx.x * kPR * ktile);
#pragma unroll
    for (int c16 = 0; c16 < 4; ++c16) {
        const int col0 = half * 64 + c16 * 16;
        if (col0 >= ktile) break;  // uniform in the warp
        float v[16];
        tmem_ld16w(taddr + (uint32_t)(c16 * 16), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int col = col0 + j;
            v[j] = col < d ? v[j] : (col == d ? res : (col <= d + 3 ? 1.0f : 0.0f));
        }
        if (qq < Qn && ok) {
            *reinterpret_cast<uint4 *>(t + core_offset(rr, col0, kPR)) =
                make_uint4(pack_half2(v[0], v[1]), pack_half2(v[2], v[3]), pack_half2(v[4], v[5]),
                           pack_half2(v[6], v[7]));
            *reinterpret_cast<uint4 *>(t + core_offset(rr, col0 + 8, kPR)) =
                make_uint4(pack_half2(v[8], v[9]), pack_half2(v[10], v[11]), pack_half2(v[12], v[13]),
                           pack_half2(v[14], v[15]));
        }
    }
    if (qq < Qn && half == 0) {
        out_norm[qq] = u2;
        out_tau[qq] = tau_scale * (u2 + *umax);
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

// basis16 chunk c = [hi tile][lo tile], each 128 rows (output coordinates n) x 32 elements
// (k = 32 c + kk) in the core-matrix layout; rows n >= d and elements k >= D are zero
__global__ void k_pack_basis16(const float *__restrict__ basisT, int D, int d, int nk,
                               unsigned char *__restrict__ basis16) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)nk * kPR * kPC) return;
    const int c = (int)(i / (kPR * kPC));
    const int n = (int)(i / kPC % kPR), kk = (int)(i % kPC);
    const int k = c * kPC + kk;
    const float b = (n < d && k < D) ? basisT[(size_t)k * kMaxDPca + n] : 0.0f;
    const __half bh = __float2half_rn(b);
    const __half bl = __float2half_rn(b - __half2float(bh));
    unsigned char *const tile = basis16 + (size_t)c * 2 * kPTile;
    *reinterpret_cast<__half *>(tile + core_offset(n, kk, kPR)) = bh;
    *reinterpret_cast<__half *>(tile + kPTile + core_offset(n, kk, kPR)) = bl;
}

// Sums the split ranges' partials of each window in range order (deterministic) and writes its
// FP16 row, ||u||^2 and tau, one warp per window
__global__ void __launch_bounds__(256) k_project_tc_finish(const float *__restrict__ part, int nsplit, int Qn, int d,
                                                           int ktile, __half *__restrict__ tile16,
                                                           float *__restrict__ out_norm, float *__restrict__ out_tau,
                                                           float tau_scale, const float *__restrict__ umax) {
    const int lane = threadIdx.x & 31;
    const long q = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= Qn) return;
    float y[4], u2 = 0.0f, yn = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) y[i] = 0.0f;
    for (int p = 0; p < nsplit; ++p) {
        const float *pr = part + ((size_t)p * Qn + q) * kPartRow;
#pragma unroll
        for (int i = 0; i < 4; ++i) y[i] += pr[lane + 32 * i];
        u2 += pr[128];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (lane + 32 * i < d) yn = fmaf(y[i], y[i], yn);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) yn += __shfl_xor_sync(0xffffffffu, yn, o);
    const float res = sqrtf(fmaxf(u2 - yn, 0.0f));
    unsigned char *const t = reinterpret_cast<unsigned char *>(tile16 + (size_t)(q / kPR) * kPR * ktile);
    const int rr = (int)(q % kPR);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int col = lane + 32 * i;
        if (col >= ktile) continue;
        const float v = col < d ? y[i] : (col == d ? res : (col <= d + 3 ? 1.0f : 0.0f));
        *reinterpret_cast<__half *>(t + core_offset(rr, col, kPR)) = __float2half_rn(v);
    }
    if (lane == 0) {
        out_norm[q] = u2;
        out_tau[q] = tau_scale * (u2 + *umax);
    }
}

__global__ void k_tile16_rows(const __half *__restrict__ qtile, int Q, int K, __half *__restrict__ rows) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)Q * K) return;
    const int q = (int)(i / K), j = (int)(i % K);
    const unsigned char *t = reinterpret_cast<const unsigned char *>(qtile + (size_t)(q / kTcQueryRows) * kTcQueryRows * K);
    rows[i] = *reinterpret_cast<const __half *>(t + core_offset(q % kTcQueryRows, j, kTcQueryRows));
}

}  // namespace

void launch_tile16_rows(const __half *qtile, int Q, int K, __half *rows, cudaStream_t st) {
    if (Q <= 0) return;
    count_launches(1);
    k_tile16_rows<<<(unsigned)ceil_div((long)Q * K, 256), 256, 0, st>>>(qtile, Q, K, rows);
}

size_t basis16_bytes(int D) { return (size_t)ceil_div(D, kPC) * 2 * kPTile; }

void launch_pack_basis16(const float *basisT, int D, int d, unsigned char *basis16, cudaStream_t st) {
    const int nk = ceil_div(D, kPC);
    count_launches(1);
    k_pack_basis16<<<(unsigned)ceil_div((long)nk * kPR * kPC, 256), 256, 0, st>>>(basisT, D, d, nk, basis16);
}

bool project_tc16_fits(int H, int W, int C) { return (long)H * W * C < (1L << 31); }

void launch_project_tc16(const float *img, int H, int W, int C, int w, int stride, const float *mu,
                         const unsigned char *basis16, int d, int K, __half *qtile, float *out_norm, float *out_tau,
                         float tau_scale, const float *umax, int *status, cudaStream_t st, DevBuf<float> *scratch) {
    const uintptr_t ia = reinterpret_cast<uintptr_t>(img);
    const int img_vec = ia % 16 == 0 ? 4 : (ia % 8 == 0 ? 2 : 1);  // widest load the image's base allows
    const int qy_n = (H - w) / stride + 1, qx_n = (W - w) / stride + 1;
    const long Qn = (long)qy_n * qx_n;
    if (Qn <= 0) return;
    // rows past the last query of the last tile stay zero (the kernel writes only real rows)
    if (Qn % kTcQueryRows)
        cudaMemsetAsync(qtile + (size_t)(Qn / kTcQueryRows) * kTcQueryRows * K, 0, sizeof(__half) * kTcQueryRows * K,
                        st);
    // A grid of at most a quarter as many query blocks as SMs splits the window vector as well (at
    // least 4 chunks a range, at most 8 ranges, about two CTAs per SM); the ranges' partial sums
    // are added in range order by k_project_tc_finish.  (At 115 blocks a 2-way split measured
    // slower than none: 35.1 against 33.0 us.)
    const long nblk = ceil_div(Qn, kPR);
    const int nk = ceil_div(C * w * w, kPC);
    int nsplit = 1;
    if (scratch && 4 * nblk <= 152)
        nsplit = (int)std::max(1L, std::min<long>(std::min<long>(8, 2 * 152 / nblk), nk / 4));
    if (nsplit > 1 && scratch->ensure((size_t)nsplit * Qn * kPartRow, "projection partials") != PTS_OK) nsplit = 1;
    const int kc_per = ceil_div(nk, nsplit);
    nsplit = ceil_div(nk, kc_per);
    float *part = nsplit > 1 ? scratch->ptr : nullptr;
    set_smem_attr(reinterpret_cast<const void *>(k_project_tc), (int)sizeof(ProjTcSmem));
    ProfScope ps(kProfProject, st, nsplit > 1 ? 2 : 1);
    k_project_tc<<<dim3((unsigned)nblk, (unsigned)nsplit), kPThreads, sizeof(ProjTcSmem), st>>>(
        img, img_vec, W, C, w, stride, qx_n, (int)Qn, mu, basis16, d, K, qtile, out_norm, out_tau, tau_scale, umax,
        status, kc_per, part);
    if (nsplit > 1)
        k_project_tc_finish<<<(unsigned)ceil_div(Qn * 32, 256), 256, 0, st>>>(part, nsplit, (int)Qn, d, K, qtile,
                                                                              out_norm, out_tau, tau_scale, umax);
}

}  // namespace pts
