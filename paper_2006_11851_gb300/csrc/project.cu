// project.cu -- projection of windows onto the PCA basis (section 2.2).
//
// For each window v on the stride grid of an image:
//   y = B^T (v - mu)         (d coordinates)
//   ||u||^2 = ||v - mu||^2
//   r = sqrt(max(0, ||u||^2 - ||y||^2))  (norm of the discarded part)
// Windows are read straight from the HWC image, never materialised: a block
// owns 32 consecutive windows of one window row; for each window row dy it
// stages the shared pixel strip, the matching D/w slice of the basis and of mu
// in shared memory, and 8 thread groups each accumulate d/8 coordinates of
// all 32 windows (d <= 128).
//
// layout 0 (queries):  coord[win][da]              = (y, r, 0, ...)
//                      tau[win] = tau_scale * (||u||^2 + max_n ||u_n||^2)
// layout 1 (exemplar): coord[win/kBN][da][win%kBN] = -2 (y, r, 0, ...)
//                      (the tiled, pre-scaled form the search streams)
#include <math.h>

#include "pts_internal.cuh"

namespace pts {
namespace {

constexpr int kPW = 32;

__global__ void __launch_bounds__(256)
    k_project(const float *__restrict__ img, int W, int w, int stride, int qx_n,
              const float *__restrict__ mu, const float *__restrict__ basis, int d, int da,
              int layout, float *__restrict__ out_coord, float *__restrict__ out_norm,
              float *__restrict__ out_tau, float tau_scale, const float *__restrict__ umax) {
    extern __shared__ __align__(16) float smp[];
    const int row = 3 * w, D = row * w;
    const int strip = ((kPW - 1) * stride + w) * 3;
    float *s_strip = smp;
    float *s_basis = s_strip + ((strip + 3) & ~3);
    float *s_mu = s_basis + d * row;
    float *s_y = s_mu + ((row + 3) & ~3);  // [kPW][d]

    const int qy = blockIdx.y, qx0 = blockIdx.x * kPW;
    const int tid = threadIdx.x, m = tid & 31, g = tid >> 5;
    const int y0 = qy * stride, x0 = qx0 * stride;
    float acc[kMaxDPca / 8];
#pragma unroll
    for (int jj = 0; jj < kMaxDPca / 8; ++jj) acc[jj] = 0.0f;
    float un = 0.0f;
    const size_t img_row = (size_t)W * 3;
    for (int dy = 0; dy < w; ++dy) {
        const float *src = img + (size_t)(y0 + dy) * img_row + (size_t)x0 * 3;
        const int avail = (W - x0) * 3;
        for (int i = tid; i < strip; i += 256) s_strip[i] = (i < avail) ? __ldg(src + i) : 0.0f;
        for (int i = tid; i < d * row; i += 256) {
            const int j = i / row, e = i - j * row;
            s_basis[i] = __ldg(basis + (size_t)j * D + dy * row + e);
        }
        for (int i = tid; i < row; i += 256) s_mu[i] = __ldg(mu + dy * row + i);
        __syncthreads();
        const float *xs = s_strip + m * stride * 3;
        for (int e = 0; e < row; ++e) {
            const float a = xs[e] - s_mu[e];
            un = fmaf(a, a, un);
#pragma unroll
            for (int jj = 0; jj < kMaxDPca / 8; ++jj) {
                const int j = g + 8 * jj;
                if (j < d) acc[jj] = fmaf(s_basis[j * row + e], a, acc[jj]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int jj = 0; jj < kMaxDPca / 8; ++jj) {
        const int j = g + 8 * jj;
        if (j < d) s_y[m * d + j] = acc[jj];
    }
    __syncthreads();
    if (g != 0 || qx0 + m >= qx_n) return;
    const long win = (long)qy * qx_n + qx0 + m;
    float yn = 0.0f;
    for (int j = 0; j < d; ++j) yn = fmaf(s_y[m * d + j], s_y[m * d + j], yn);
    const float r = sqrtf(fmaxf(un - yn, 0.0f));
    out_norm[win] = un;
    if (layout == 0) {
        float *o = out_coord + win * da;
        for (int j = 0; j < d; ++j) o[j] = s_y[m * d + j];
        o[d] = r;
        for (int j = d + 1; j < da; ++j) o[j] = 0.0f;
        out_tau[win] = tau_scale * (un + *umax);
    } else {
        const long tile = win / kBN, col = win - tile * kBN;
        float *o = out_coord + tile * (long)da * kBN + col;
        for (int j = 0; j < d; ++j) o[(long)j * kBN] = -2.0f * s_y[m * d + j];
        o[(long)d * kBN] = -2.0f * r;
        for (int j = d + 1; j < da; ++j) o[(long)j * kBN] = 0.0f;
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
    const int row = 3 * w;
    const int strip = ((kPW - 1) * stride + w) * 3;
    const size_t smem = sizeof(float) * (((strip + 3) & ~3) + d * row + ((row + 3) & ~3) + kPW * d);
    static size_t attr_set = 0;
    if (smem > 48 * 1024 && smem > attr_set) {
        cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = smem;
    }
    dim3 grid(ceil_div(qx_n, kPW), qy_n);
    ProfScope ps(kProfProject, st, 1);
    k_project<<<grid, 256, smem, st>>>(img, W, w, stride, qx_n, mu, basis, d, da, layout, out_coord,
                                       out_norm, out_tau, tau_scale, umax);
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
