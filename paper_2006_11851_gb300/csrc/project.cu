// project.cu -- projection of windows onto the PCA basis (section 2.2).
//
// For each window v on the stride grid of an image:
//   y = B^T (v - mu)         (d coordinates)
//   ||u||^2 = ||v - mu||^2
//   r = sqrt(max(0, ||u||^2 - ||y||^2))  (norm of the discarded part)
// A tiled SIMT GEMM (windows x D) (D x d): a block owns 64 windows and all d <= 128 outputs.
// Windows are read straight from the HWC image, never materialised: per 32-element slice of
// the window vector the block stages the 64 centred slices and the basis slice in shared memory
// (per-window base offsets and per-element offsets are precomputed, so a staged element is one
// gather), and each thread accumulates a 4-window x 8-coordinate register tile.
//
// layout 0 (queries):  coord[win][da]              = (y, r, 0, ...)
//                      tau[win] = tau_scale * (||u||^2 + max_n ||u_n||^2)
// layout 1 (exemplar): coord[win/kBN][da][win%kBN] = -2 (y, r, 0, ...)
//                      (the tiled, pre-scaled form the search streams)
#include <math.h>

#include "pts_internal.cuh"

namespace pts {
namespace {

constexpr int kPWin = 64;           // windows per block
constexpr int kPK = 32;             // window-vector elements per slice
constexpr int kPD = kMaxDPca;       // coordinates per block (d <= 128)
constexpr int kXs = kPWin + 1;      // row stride of the staged window slices
constexpr int kBs = kPD + 4;        // row stride of the staged basis slice (16-byte rows)

struct ProjSmem {
    union {
        struct {
            float xs[kPK * kXs];              // [k][window], centred
            alignas(16) float bs[kPK * kBs];  // [k][coordinate]
        } st;
        float ys[kPWin * (kPD + 1)];          // the finished tile, [window][coordinate]
    } u;
    long base[kPWin];               // image offset of each window's first element
    int koff[kPK];                  // image offset of each element of the slice
    float un[kPWin];
};

__global__ void __launch_bounds__(256)
    k_project(const float *__restrict__ img, int W, int w, int stride, int qx_n, int Qn,
              const float *__restrict__ mu, const float *__restrict__ basis, int d, int da,
              int layout, float *__restrict__ out_coord, float *__restrict__ out_norm,
              float *__restrict__ out_tau, float tau_scale, const float *__restrict__ umax) {
    __shared__ ProjSmem sm;
    float *const xs = sm.u.st.xs;
    float *const bs = sm.u.st.bs;
    float *const ys = sm.u.ys;
    const int row = 3 * w, D = row * w;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long win0 = (long)blockIdx.x * kPWin;
    if (tid < kPWin) {
        const long win = win0 + tid;
        const long wq = win < Qn ? win : 0;
        const long qy = wq / qx_n, qx = wq - qy * qx_n;
        sm.base[tid] = (qy * stride * (long)W + qx * stride) * 3;
        sm.un[tid] = 0.0f;
    }
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    float un = 0.0f;
    for (int k0 = 0; k0 < D; k0 += kPK) {
        if (tid < kPK) {
            const int k = min(k0 + tid, D - 1);
            const int dy = k / row, e = k - dy * row;
            sm.koff[tid] = dy * W * 3 + e;
        }
        __syncthreads();
        // window slices: consecutive threads take consecutive elements of one window
#pragma unroll
        for (int it = 0; it < kPWin * kPK / 256; ++it) {
            const int idx = tid + 256 * it;
            const int wl = idx / kPK, kk = idx - wl * kPK;
            const int k = k0 + kk;
            float v = 0.0f;
            if (k < D && win0 + wl < Qn) v = __ldg(img + sm.base[wl] + sm.koff[kk]) - __ldg(mu + k);
            xs[kk * kXs + wl] = v;
        }
        // basis slice: row j of the basis is contiguous in k
        for (int idx = tid; idx < kPD * kPK; idx += 256) {
            const int j = idx / kPK, kk = idx - j * kPK;
            const int k = k0 + kk;
            bs[kk * kBs + j] = (j < d && k < D) ? __ldg(basis + (size_t)j * D + k) : 0.0f;
        }
        __syncthreads();
        if (tid < kPWin) {
#pragma unroll 8
            for (int kk = 0; kk < kPK; ++kk) {
                const float a = xs[kk * kXs + tid];
                un = fmaf(a, a, un);
            }
        }
#pragma unroll 4
        for (int kk = 0; kk < kPK; ++kk) {
            float a[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = xs[kk * kXs + ty * 4 + i];
            const float4 b0 = *reinterpret_cast<const float4 *>(&bs[kk * kBs + tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&bs[kk * kBs + tx * 8 + 4]);
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    // (the loop ends with a barrier, so the staging buffers may be overwritten)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) ys[(ty * 4 + i) * (kPD + 1) + tx * 8 + j] = acc[i][j];
    if (tid < kPWin) sm.un[tid] = un;
    __syncthreads();
    // one warp per window row of the tile: ||y||^2, r, and the coalesced writes
    const int lane = tid & 31, wp = tid >> 5;
    for (int wl = wp; wl < kPWin; wl += 8) {
        const long win = win0 + wl;
        if (win >= Qn) break;
        const float *yr = &ys[wl * (kPD + 1)];
        float yn = 0.0f;
        for (int j = lane; j < d; j += 32) yn = fmaf(yr[j], yr[j], yn);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) yn += __shfl_xor_sync(0xffffffffu, yn, o);
        const float u2 = sm.un[wl];
        const float r = sqrtf(fmaxf(u2 - yn, 0.0f));
        if (layout == 0) {
            float *o = out_coord + win * da;
            for (int j = lane; j < da; j += 32) o[j] = j < d ? yr[j] : (j == d ? r : 0.0f);
            if (lane == 0) out_tau[win] = tau_scale * (u2 + *umax);
        } else {
            const long tile = win / kBN, col = win - tile * kBN;
            float *o = out_coord + tile * (long)da * kBN + col;
            for (int j = lane; j < da; j += 32) o[(long)j * kBN] = j < d ? -2.0f * yr[j] : (j == d ? -2.0f * r : 0.0f);
        }
        if (lane == 0) out_norm[win] = u2;
    }
}

__global__ void k_fill(float *p, long n, float v) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        p[i] = v;
}

// max of non-negative floats (order-independent, hence deterministic)
__global__ void k_norm_max(const float *__restrict__ v, int n, float *__restrict__ out) {
    __shared__ float red[1024];
    float m = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, v[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

void launch_project(const float *img, int H, int W, int w, int stride, const float *mu,
                    const float *basis, int d, int da, int layout, float *out_coord,
                    float *out_norm, float *out_tau, float tau_scale, const float *umax,
                    cudaStream_t st) {
    const int qy_n = (H - w) / stride + 1, qx_n = (W - w) / stride + 1;
    const long Qn = (long)qy_n * qx_n;
    if (Qn <= 0) return;
    ProfScope ps(kProfProject, st, 1);
    k_project<<<(unsigned)ceil_div(Qn, kPWin), 256, 0, st>>>(img, W, w, stride, qx_n, (int)Qn, mu, basis, d, da,
                                                            layout, out_coord, out_norm, out_tau, tau_scale, umax);
}

void launch_exemplar_pad(float *et, float *enorm, int N, int ntiles, int da, cudaStream_t st) {
    (void)N;
    cudaMemsetAsync(et, 0, sizeof(float) * (size_t)ntiles * da * kBN, st);
    count_launches(1);
    k_fill<<<64, 256, 0, st>>>(enorm, (long)ntiles * kBN, INFINITY);
}

void launch_norm_max(const float *norm, int n, float *out, cudaStream_t st) {
    count_launches(1);
    k_norm_max<<<1, 1024, 0, st>>>(norm, n, out);
}

}  // namespace pts
