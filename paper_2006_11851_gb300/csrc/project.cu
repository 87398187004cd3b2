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

#include <algorithm>

#include "pts_internal.cuh"

namespace pts {
namespace {

constexpr int kPWin = 64;           // windows per block
constexpr int kPK = 32;             // window-vector elements per slice
constexpr int kXs = kPWin + 1;      // row stride of the staged window slices

template <int PD>
struct ProjSmem {
    static constexpr int kBs = PD + 4;  // row stride of the staged basis slice (16-byte rows)
    union {
        struct {
            float xs[kPK * kXs];              // [k][window], centred
            alignas(16) float bs[kPK * kBs];  // [k][coordinate]
        } st;
        float ys[kPWin * (PD + 1)];           // the finished tile, [window][coordinate]
    } u;
    long base[kPWin];               // image offset of each window's first element
    int koff[kPK];                  // image offset of each element of the slice
    float un[kPWin];
};

struct ProjOut {
    int d, da, layout;
    float *coord, *norm, *tau;
    float tau_scale;
    const float *umax;
};

// ||y||^2, r and the output rows of one window, written by one warp (y in shared or global
// memory, row of PD + 1 floats: coordinates then ||u||^2)
__device__ __forceinline__ void write_window(const ProjOut &o, long win, const float *yr, float u2, int lane) {
    float yn = 0.0f;
    for (int j = lane; j < o.d; j += 32) yn = fmaf(yr[j], yr[j], yn);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) yn += __shfl_xor_sync(0xffffffffu, yn, s);
    const float r = sqrtf(fmaxf(u2 - yn, 0.0f));
    if (o.layout == 0) {
        float *c = o.coord + win * o.da;
        for (int j = lane; j < o.da; j += 32) c[j] = j < o.d ? yr[j] : (j == o.d ? r : 0.0f);
        if (lane == 0) o.tau[win] = o.tau_scale * (u2 + *o.umax);
    } else {
        const long tile = win / kBN, col = win - tile * kBN;
        float *c = o.coord + tile * (long)o.da * kBN + col;
        for (int j = lane; j < o.da; j += 32) c[(long)j * kBN] = j < o.d ? -2.0f * yr[j] : (j == o.d ? -2.0f * r : 0.0f);
    }
    if (lane == 0) o.norm[win] = u2;
}

// PD = 64 or 128 output columns (d <= PD); thread tile 4 windows x PD/16 coordinates.  With
// gridDim.y > 1 the block covers one slice range of the window vector and writes its partial
// sums to part[blockIdx.y][win][PD + 1] (coordinates, then ||u||^2), reduced by k_project_finish.
template <int PD>
__global__ void __launch_bounds__(256)
    k_project(const float *__restrict__ img, int W, int w, int stride, int qx_n, int Qn,
              const float *__restrict__ mu, const float *__restrict__ basis, int kper, ProjOut o,
              float *__restrict__ part) {
    constexpr int JD = PD / 16;
    constexpr int kBs = ProjSmem<PD>::kBs;
    __shared__ ProjSmem<PD> sm;
    float *const xs = sm.u.st.xs;
    float *const bs = sm.u.st.bs;
    float *const ys = sm.u.ys;
    const int row = 3 * w, D = row * w, d = o.d;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long win0 = (long)blockIdx.x * kPWin;
    const int kbeg = blockIdx.y * kper, kend = min(D, kbeg + kper);
    if (tid < kPWin) {
        const long win = win0 + tid;
        const long wq = win < Qn ? win : 0;
        const long qy = wq / qx_n, qx = wq - qy * qx_n;
        sm.base[tid] = (qy * stride * (long)W + qx * stride) * 3;
        sm.un[tid] = 0.0f;
    }
    float acc[4][JD];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < JD; ++j) acc[i][j] = 0.0f;
    float un = 0.0f;
    for (int k0 = kbeg; k0 < kend; k0 += kPK) {
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
            if (k < kend && win0 + wl < Qn) v = __ldg(img + sm.base[wl] + sm.koff[kk]) - __ldg(mu + k);
            xs[kk * kXs + wl] = v;
        }
        // basis slice: row j of the basis is contiguous in k
        for (int idx = tid; idx < PD * kPK; idx += 256) {
            const int j = idx / kPK, kk = idx - j * kPK;
            const int k = k0 + kk;
            bs[kk * kBs + j] = (j < d && k < kend) ? __ldg(basis + (size_t)j * D + k) : 0.0f;
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
            float b[JD];
#pragma unroll
            for (int j4 = 0; j4 < JD / 4; ++j4) {
                const float4 bv = *reinterpret_cast<const float4 *>(&bs[kk * kBs + tx * JD + 4 * j4]);
                b[4 * j4] = bv.x;
                b[4 * j4 + 1] = bv.y;
                b[4 * j4 + 2] = bv.z;
                b[4 * j4 + 3] = bv.w;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < JD; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    if (gridDim.y > 1) {
        float *pb = part + (size_t)blockIdx.y * Qn * (PD + 1);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const long win = win0 + ty * 4 + i;
            if (win < Qn)
#pragma unroll
                for (int j = 0; j < JD; ++j) pb[win * (PD + 1) + tx * JD + j] = acc[i][j];
        }
        if (tid < kPWin && win0 + tid < Qn) pb[(win0 + tid) * (PD + 1) + PD] = un;
        return;
    }
    // (the loop ends with a barrier, so the staging buffers may be overwritten)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < JD; ++j) ys[(ty * 4 + i) * (PD + 1) + tx * JD + j] = acc[i][j];
    if (tid < kPWin) sm.un[tid] = un;
    __syncthreads();
    const int lane = tid & 31, wp = tid >> 5;
    for (int wl = wp; wl < kPWin; wl += 8) {
        const long win = win0 + wl;
        if (win >= Qn) break;
        write_window(o, win, &ys[wl * (PD + 1)], sm.un[wl], lane);
    }
}

// Sums the slice partials of each window in slice order (deterministic) and writes its outputs.
template <int PD>
__global__ void __launch_bounds__(256) k_project_finish(const float *__restrict__ part, int nsplit, int Qn, ProjOut o) {
    __shared__ float ys[8][PD + 1];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const long win = (long)blockIdx.x * 8 + wp;
    if (win >= Qn) return;
    for (int j = lane; j <= PD; j += 32) {
        float sacc = 0.0f;
        for (int p = 0; p < nsplit; ++p) sacc += part[((size_t)p * Qn + win) * (PD + 1) + j];
        ys[wp][j] = sacc;
    }
    __syncwarp();
    write_window(o, win, ys[wp], ys[wp][PD], lane);
}

// ||v - mu||^2 (and tau) of each window only, one warp per window (the search needs no
// coordinates when it runs in full dimension).
__global__ void __launch_bounds__(256) k_window_norms(const float *__restrict__ img, int W, int w, int stride, int qx_n,
                                                      int Qn, const float *__restrict__ mu, ProjOut o) {
    const int lane = threadIdx.x & 31;
    const long win = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (win >= Qn) return;
    const int row = 3 * w;
    const long qy = win / qx_n, qx = win - qy * qx_n;
    const float *src = img + (qy * stride * (long)W + qx * stride) * 3;
    float un = 0.0f;
    for (int dy = 0; dy < w; ++dy)
        for (int e = lane; e < row; e += 32) {
            const float a = __ldg(src + (size_t)dy * W * 3 + e) - __ldg(mu + dy * row + e);
            un = fmaf(a, a, un);
        }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) un += __shfl_xor_sync(0xffffffffu, un, s);
    if (lane == 0) {
        o.norm[win] = un;
        if (o.tau) o.tau[win] = o.tau_scale * (un + *o.umax);
        if (o.coord) {
            float *c = o.coord + win * o.da;
            c[0] = sqrtf(un);
            for (int j = 1; j < o.da; ++j) c[j] = 0.0f;
        }
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
                    cudaStream_t st, DevBuf<float> *scratch) {
    const int qy_n = (H - w) / stride + 1, qx_n = (W - w) / stride + 1;
    const long Qn = (long)qy_n * qx_n;
    if (Qn <= 0) return;
    const ProjOut o{d, da, layout, out_coord, out_norm, out_tau, tau_scale, umax};
    ProfScope ps(kProfProject, st, 1);
    if (d <= 0) {
        k_window_norms<<<(unsigned)ceil_div(Qn * 32, 256), 256, 0, st>>>(img, W, w, stride, qx_n, (int)Qn, mu, o);
        return;
    }
    const int D = 3 * w * w;
    const long nblk = ceil_div(Qn, kPWin);
    // slices of the window vector per block: enough blocks for two per SM when the windows alone
    // leave SMs idle, each slice range at least 256 long
    int nsplit = 1;
    if (scratch && nblk < 2 * 152) nsplit = (int)std::max(1L, std::min<long>(2 * 152 / nblk, D / 256));
    const int PDc = d <= 64 ? 64 : 128;
    if (nsplit > 1 && scratch->ensure((size_t)nsplit * Qn * (PDc + 1), "projection partials") != PTS_OK)
        nsplit = 1;
    const int kper = ceil_div(ceil_div(D, nsplit), kPK) * kPK;
    nsplit = ceil_div(D, kper);
    const dim3 grid((unsigned)nblk, nsplit);
    float *part = nsplit > 1 ? scratch->ptr : nullptr;
    if (PDc == 64)
        k_project<64><<<grid, 256, 0, st>>>(img, W, w, stride, qx_n, (int)Qn, mu, basis, kper, o, part);
    else
        k_project<128><<<grid, 256, 0, st>>>(img, W, w, stride, qx_n, (int)Qn, mu, basis, kper, o, part);
    if (nsplit > 1) {
        count_launches(1);
        if (PDc == 64)
            k_project_finish<64><<<(unsigned)ceil_div(Qn, 8), 256, 0, st>>>(part, nsplit, (int)Qn, o);
        else
            k_project_finish<128><<<(unsigned)ceil_div(Qn, 8), 256, 0, st>>>(part, nsplit, (int)Qn, o);
    }
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
