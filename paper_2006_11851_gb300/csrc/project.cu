// project.cu -- projection of windows onto the PCA basis (section 2.2).
//
// For each window v on the stride grid of an image:
//   y = B^T (v - mu)         (d coordinates)
//   ||u||^2 = ||v - mu||^2
//   r = sqrt(max(0, ||u||^2 - ||y||^2))  (norm of the discarded part)
// A tiled SIMT GEMM (windows x D) (D x d): a block owns 128 windows and all d <= 128 outputs.
// Windows are read straight from the HWC image (C = 3 or 4 channels), never materialised: per
// 32-element slice of
// the window vector the block stages the 128 centred slices and the slice of the transposed
// basis ([D][128], built with the index) in shared memory, and each thread accumulates an
// 8-window x 8-coordinate (4 for d <= 64) register tile.
//
// layout 0 (queries):  coord[win][da]              = (y, r, 0, ...)
//                      tau[win] = tau_scale * (||u||^2 + max_n ||u_n||^2)
// layout 1 (exemplar): coord[win/kBN][da][win%kBN] = -2 (y, r, 0, ...)
//                      (the tiled, pre-scaled form the search streams)
// layout 2 (queries, FP16 search): (y, r, 1, 1, 1, 0, ...) rounded to FP16 straight into the
//                      tensor-core query tiles (128 rows x K each, core-matrix layout), and tau
#include <math.h>

#include <algorithm>

#include "tc_common.cuh"

namespace pts {
namespace {

constexpr int kPWin = 128;          // windows per block
constexpr int kPK = 32;             // window-vector elements per slice
constexpr int kXs = kPWin + 4;      // row stride of the staged window slices (16-byte rows)
constexpr int kBT = kMaxDPca;       // row stride of the transposed basis [D][kBT]

template <int PD>
struct ProjSmem {
    union {
        struct {
            alignas(16) float xs[kPK * kXs];  // [k][window], centred
            alignas(16) float bs[kPK * PD];   // [k][coordinate]
        } st;
        float ys[kPWin * (PD + 1)];           // the finished tile, [window][coordinate]
    } u;
    long base[kPWin];                 // image offset of each window's first element
    float un[2][kPWin];               // ||u||^2 of each window, the two staging halves
};

struct ProjOut {
    int d, da, layout;
    float *coord, *norm, *tau;
    float tau_scale;
    const float *umax;
    __half *tile16;  // layout 2: the FP16 query tiles
    int ktile;       // layout 2: their K
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
    } else if (o.layout == 2) {
        // the values the FP16 search multiplies: coordinates, the residual, then three ones
        // against the exemplar's norm slots (hi, mid, lo)
        unsigned char *t = reinterpret_cast<unsigned char *>(o.tile16 + (size_t)(win / kTcQueryRows) * kTcQueryRows * o.ktile);
        const int rr = (int)(win % kTcQueryRows);
        for (int j = lane; j < o.ktile; j += 32) {
            const float v = j < o.d ? yr[j] : (j == o.d ? r : (j <= o.d + 3 ? 1.0f : 0.0f));
            *reinterpret_cast<__half *>(t + core_offset(rr, j, kTcQueryRows)) = __float2half_rn(v);
        }
        if (lane == 0) o.tau[win] = o.tau_scale * (u2 + *o.umax);
    } else {
        const long tile = win / kBN, col = win - tile * kBN;
        float *c = o.coord + tile * (long)o.da * kBN + col;
        for (int j = lane; j < o.da; j += 32) c[(long)j * kBN] = j < o.d ? -2.0f * yr[j] : (j == o.d ? -2.0f * r : 0.0f);
    }
    if (lane == 0) o.norm[win] = u2;
}

// PD = 64 or 128 output columns (d <= PD).  Thread (tx, ty) of 16 x 16 accumulates windows
// ty*4 + {0..3} + {0, 64} times coordinates tx*4 + {0..3} + 64 g (g < PD/64): every operand
// read is a 16-byte shared load, the window reads broadcast and the basis reads contiguous.
// Staging: thread t gathers window t % 128 at the slice rows t / 128 + 2i (i < 16), adding its
// squares to the window's norm, and four (PD = 128) or two float4 of the transposed basis; the
// next slice is loaded into registers while the current one is multiplied.  With gridDim.y > 1
// the block covers one slice range of the window vector and writes its partial sums to
// part[blockIdx.y][win][PD + 1] (coordinates, then ||u||^2), reduced by k_project_finish.
template <int PD>
__global__ void __launch_bounds__(256, 2)
    k_project(const float *__restrict__ img, int W, int C, int w, int stride, int qx_n, int Qn,
              const float *__restrict__ mu, const float *__restrict__ basisT, int kper, ProjOut o,
              float *__restrict__ part) {
    constexpr int NG = PD / 64;      // float4 groups of coordinates per thread
    constexpr int TJ = 4 * NG;       // coordinates per thread
    constexpr int NB = PD / 32;      // float4 of the basis slice per thread
    extern __shared__ __align__(16) unsigned char proj_smem[];
    ProjSmem<PD> &sm = *reinterpret_cast<ProjSmem<PD> *>(proj_smem);
    float *const xs = sm.u.st.xs;
    float *const bs = sm.u.st.bs;
    float *const ys = sm.u.ys;
    const int row = C * w, D = row * w, d = o.d, W3 = C * W;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long win0 = (long)blockIdx.x * kPWin;
    const int kbeg = blockIdx.y * kper, kend = min(D, kbeg + kper);
    if (tid < kPWin) {
        const long win = win0 + tid;
        const long wq = win < Qn ? win : 0;
        const long qy = wq / qx_n, qx = wq - qy * qx_n;
        sm.base[tid] = (qy * stride * (long)W + qx * stride) * C;
    }
    __syncthreads();
    const int sw = tid & (kPWin - 1), sk = tid >> 7;
    const bool wvalid = win0 + sw < Qn;
    const float *const src = img + sm.base[sw];
    // element k0 + sk of the window vector at (row dy, offset e): image offset dy * W3 + e
    int e0 = (kbeg + sk) % row;
    long off0 = (long)((kbeg + sk) / row) * W3 + e0;
    float xr[16];
    float4 br[NB];
    auto load_slice = [&](int k0) {
        int e = e0;
        long off = off0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int k = k0 + sk + 2 * i;
            xr[i] = (k < kend && wvalid) ? __ldg(src + off) - __ldg(mu + k) : 0.0f;
            e += 2;
            off += 2;
            if (e >= row) {  // row >= 3: one wrap at most (e advances by 2)
                e -= row;
                off += W3 - row;
            }
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int f = tid + 256 * i;  // float4 index in the 32 x PD slice
            const int kk = f / (PD / 4), j4 = f - kk * (PD / 4);
            br[i] = (k0 + kk < kend) ? __ldg(reinterpret_cast<const float4 *>(basisT + (size_t)(k0 + kk) * kBT) + j4)
                                     : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    };
    auto advance = [&]() {  // e0, off0 -> the same role in the next slice (32 elements on)
        int e = e0 + kPK;
        long off = off0 + kPK;
        while (e >= row) {
            e -= row;
            off += W3 - row;
        }
        e0 = e;
        off0 = off;
    };
    float acc[8][TJ];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) acc[i][j] = 0.0f;
    float un = 0.0f;
    load_slice(kbeg);
    for (int k0 = kbeg; k0 < kend; k0 += kPK) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            xs[(sk + 2 * i) * kXs + sw] = xr[i];
            un = fmaf(xr[i], xr[i], un);
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int f = tid + 256 * i;
            const int kk = f / (PD / 4), j = 4 * (f - kk * (PD / 4));
            float4 b = br[i];
            b.x = j < d ? b.x : 0.0f;
            b.y = j + 1 < d ? b.y : 0.0f;
            b.z = j + 2 < d ? b.z : 0.0f;
            b.w = j + 3 < d ? b.w : 0.0f;
            *reinterpret_cast<float4 *>(&bs[kk * PD + j]) = b;
        }
        __syncthreads();
        if (k0 + kPK < kend) {
            advance();
            load_slice(k0 + kPK);
        }
#pragma unroll 4
        for (int kk = 0; kk < kPK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&xs[kk * kXs + ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&xs[kk * kXs + ty * 4 + 64]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float b[TJ];
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const float4 bv = *reinterpret_cast<const float4 *>(&bs[kk * PD + g * 64 + tx * 4]);
                b[4 * g] = bv.x;
                b[4 * g + 1] = bv.y;
                b[4 * g + 2] = bv.z;
                b[4 * g + 3] = bv.w;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < TJ; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    sm.un[sk][sw] = un;
    __syncthreads();
    if (gridDim.y > 1) {
        float *pb = part + (size_t)blockIdx.y * Qn * (PD + 1);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const long win = win0 + ty * 4 + (i & 3) + 64 * (i >> 2);
            if (win < Qn)
#pragma unroll
                for (int j = 0; j < TJ; ++j) pb[win * (PD + 1) + (j >> 2) * 64 + tx * 4 + (j & 3)] = acc[i][j];
        }
        if (tid < kPWin && win0 + tid < Qn) pb[(win0 + tid) * (PD + 1) + PD] = sm.un[0][tid] + sm.un[1][tid];
        return;
    }
    // (the loop ends with a barrier, so the staging buffers may be overwritten)
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j)
            ys[(ty * 4 + (i & 3) + 64 * (i >> 2)) * (PD + 1) + (j >> 2) * 64 + tx * 4 + (j & 3)] = acc[i][j];
    __syncthreads();
    const int lane = tid & 31, wp = tid >> 5;
    for (int wl = wp; wl < kPWin; wl += 8) {
        const long win = win0 + wl;
        if (win >= Qn) break;
        write_window(o, win, &ys[wl * (PD + 1)], sm.un[0][wl] + sm.un[1][wl], lane);
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
__global__ void __launch_bounds__(256) k_window_norms(const float *__restrict__ img, int W, int C, int w, int stride, int qx_n,
                                                      int Qn, const float *__restrict__ mu, ProjOut o) {
    const int lane = threadIdx.x & 31;
    const long win = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (win >= Qn) return;
    const int row = C * w;
    const long qy = win / qx_n, qx = win - qy * qx_n;
    const float *src = img + (qy * stride * (long)W + qx * stride) * C;
    const size_t pitch = (size_t)W * C;
    // four window rows at a time into four partial sums, so that their loads are in flight together
    float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f, u3 = 0.0f;
    int dy = 0;
    for (; dy + 4 <= w; dy += 4)
        for (int e = lane; e < row; e += 32) {
            const float *s0 = src + dy * pitch + e;
            const float *m0 = mu + dy * row + e;
            const float a0 = __ldg(s0) - __ldg(m0);
            const float a1 = __ldg(s0 + pitch) - __ldg(m0 + row);
            const float a2 = __ldg(s0 + 2 * pitch) - __ldg(m0 + 2 * row);
            const float a3 = __ldg(s0 + 3 * pitch) - __ldg(m0 + 3 * row);
            u0 = fmaf(a0, a0, u0);
            u1 = fmaf(a1, a1, u1);
            u2 = fmaf(a2, a2, u2);
            u3 = fmaf(a3, a3, u3);
        }
    for (; dy < w; ++dy)
        for (int e = lane; e < row; e += 32) {
            const float a = __ldg(src + dy * pitch + e) - __ldg(mu + dy * row + e);
            u0 = fmaf(a, a, u0);
        }
    float un = (u0 + u1) + (u2 + u3);
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

// basisT[k][j] = basis[j][k] for the computed components j < dcount, 0 past them
__global__ void k_basis_transpose(const float *__restrict__ basis, int dcount, int D, float *__restrict__ basisT) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)D * kBT) return;
    const int k = (int)(i / kBT), j = (int)(i - (long)k * kBT);
    basisT[i] = j < dcount ? basis[(size_t)j * D + k] : 0.0f;
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

static void launch_project_impl(const float *img, int H, int W, int C, int w, int stride, const float *mu,
                                const float *basisT, int d, int da, int layout, float *out_coord, float *out_norm,
                                float *out_tau, float tau_scale, const float *umax, cudaStream_t st,
                                DevBuf<float> *scratch, __half *tile16, int ktile) {
    const int qy_n = (H - w) / stride + 1, qx_n = (W - w) / stride + 1;
    const long Qn = (long)qy_n * qx_n;
    if (Qn <= 0) return;
    const ProjOut o{d, da, layout, out_coord, out_norm, out_tau, tau_scale, umax, tile16, ktile};
    ProfScope ps(kProfProject, st, 1);
    if (d <= 0) {
        k_window_norms<<<(unsigned)ceil_div(Qn * 32, 256), 256, 0, st>>>(img, W, C, w, stride, qx_n, (int)Qn, mu, o);
        return;
    }
    const int D = C * w * w;
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
    set_smem_attr(reinterpret_cast<const void *>(k_project<64>), (int)sizeof(ProjSmem<64>));
    set_smem_attr(reinterpret_cast<const void *>(k_project<128>), (int)sizeof(ProjSmem<128>));
    if (PDc == 64)
        k_project<64><<<grid, 256, sizeof(ProjSmem<64>), st>>>(img, W, C, w, stride, qx_n, (int)Qn, mu, basisT, kper,
                                                               o, part);
    else
        k_project<128><<<grid, 256, sizeof(ProjSmem<128>), st>>>(img, W, C, w, stride, qx_n, (int)Qn, mu, basisT,
                                                                 kper, o, part);
    if (nsplit > 1) {
        count_launches(1);
        if (PDc == 64)
            k_project_finish<64><<<(unsigned)ceil_div(Qn, 8), 256, 0, st>>>(part, nsplit, (int)Qn, o);
        else
            k_project_finish<128><<<(unsigned)ceil_div(Qn, 8), 256, 0, st>>>(part, nsplit, (int)Qn, o);
    }
}

void launch_project(const float *img, int H, int W, int C, int w, int stride, const float *mu,
                    const float *basisT, int d, int da, int layout, float *out_coord,
                    float *out_norm, float *out_tau, float tau_scale, const float *umax,
                    cudaStream_t st, DevBuf<float> *scratch) {
    launch_project_impl(img, H, W, C, w, stride, mu, basisT, d, da, layout, out_coord, out_norm, out_tau, tau_scale,
                        umax, st, scratch, nullptr, 0);
}

void launch_project_tile16(const float *img, int H, int W, int C, int w, int stride, const float *mu,
                           const float *basisT, int d, int K, __half *qtile, float *out_norm, float *out_tau,
                           float tau_scale, const float *umax, cudaStream_t st, DevBuf<float> *scratch) {
    const int qy_n = (H - w) / stride + 1, qx_n = (W - w) / stride + 1;
    const long Qn = (long)qy_n * qx_n;
    if (Qn <= 0) return;
    // rows past the last query of the last tile stay zero (the projection writes only real rows)
    if (Qn % kTcQueryRows)
        cudaMemsetAsync(qtile + (size_t)(Qn / kTcQueryRows) * kTcQueryRows * K, 0,
                        sizeof(__half) * kTcQueryRows * K, st);
    launch_project_impl(img, H, W, C, w, stride, mu, basisT, d, 0, 2, nullptr, out_norm, out_tau, tau_scale, umax,
                        st, scratch, qtile, K);
}

void launch_basis_transpose(const float *basis, int dcount, int D, float *basisT, cudaStream_t st) {
    count_launches(1);
    k_basis_transpose<<<(unsigned)ceil_div((long)D * kBT, 256), 256, 0, st>>>(basis, dcount, D, basisT);
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
