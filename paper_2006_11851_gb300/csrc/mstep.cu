// mstep.cu -- optimization phase (M-step), IRLS weights/energy and the
// pyramid filters.
//
// M-step (Eq. 8 minimised over x): pixel i becomes
//   x_i = sum_{p covers i} W_p z_{nn(p)}[i - p] / sum_{p covers i} W_p.
// With the patch stride s dividing w, the s x s pixels of a patch share one
// covering set of query windows (section 2.2, 2x2 patch processing), so one
// thread owns one patch: it walks the covering windows in increasing query
// order (the order of the sum above), gathers the co-located s x s block of
// each matched exemplar window and writes its s*s*3 colour outputs once.  No
// atomics, deterministic.  The exemplar (<= a few MB) stays in L2, read from
// an RGBA copy (fourth value 0, or the scale channel of an RGBS exemplar) so
// that each gathered pixel is one 16-byte load.  The output has C = 3 or 4
// channels; with 4 its fourth (the scale map, section 1) is left as it is.
#include <algorithm>

#include "pts_internal.cuh"

namespace pts {
namespace {

// HIST: the weights of Eq. 9 (section 3).  The contribution of window p to pixel i is weighted
// w_p / (1 + sum_j max[0, H_x,j(b_j(c)) - H_z,j(b_j(c))]), c the exemplar pixel it brings, the
// excess table (3 x nbins, from the two images' channel counts) built per block in shared memory;
// every pixel is normalised by its own sum of weights.  Without HIST the patch's four pixels share
// one sum.
template <int S, bool HIST, int SPL = 1>
__global__ void __launch_bounds__(128)
    k_m_step(const int *__restrict__ nn, const float *__restrict__ wts, const float4 *__restrict__ Z4,
             int We, int ex, int N, int C, int w, int Ho, int Wo, int qy_n, int qx_n,
             float *__restrict__ out, int *__restrict__ status, int nbins, const unsigned int *__restrict__ cx,
             long nx, const unsigned int *__restrict__ cz, long nz) {
    __shared__ float hex[HIST ? 3 * kMaxHistBins : 1];
    if constexpr (HIST) {
        for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x)
            hex[i] = (float)fmax(0.0, (double)cx[i] / (double)nx - (double)cz[i] / (double)nz);
        __syncthreads();
    }
    // SPL consecutive threads share a patch, each taking every SPL-th row of its covering windows;
    // their sums meet in a fixed xor tree, so the result is deterministic
    const int sub = (int)threadIdx.x % SPL;
    const int px = (int)((blockIdx.x * blockDim.x + threadIdx.x) / SPL);
    const int py = blockIdx.y;
    const bool live = px < Wo / S && py < Ho / S;
    if (SPL == 1 && !live) return;
    const int ws = w / S;
    const int qy_lo = max(0, py - ws + 1), qy_hi = min(py, qy_n - 1);
    const int qx_lo = max(0, px - ws + 1), qx_hi = min(px, qx_n - 1);
    float num[S][S][3];
    float dpix[HIST ? S : 1][HIST ? S : 1];
#pragma unroll
    for (int t = 0; t < S; ++t)
#pragma unroll
        for (int u = 0; u < S; ++u)
#pragma unroll
            for (int c = 0; c < 3; ++c) num[t][u][c] = 0.0f;
    if constexpr (HIST)
#pragma unroll
        for (int t = 0; t < S; ++t)
#pragma unroll
            for (int u = 0; u < S; ++u) dpix[t][u] = 0.0f;
    float den = 0.0f;
    bool bad = false;
    for (int qy = live ? qy_lo + sub : qy_hi + 1; qy <= qy_hi; qy += SPL) {
        const int oy = (py - qy) * S;
        for (int qx = qx_lo; qx <= qx_hi; ++qx) {
            const int p = qy * qx_n + qx;
            int n = __ldg(nn + p);
            if (n < 0 || n >= N) {
                bad = true;
                n = n < 0 ? 0 : N - 1;
            }
            const float wt = wts ? __ldg(wts + p) : 1.0f;
            const int ey = n / ex, exx = n - ey * ex;
            const int ox = (px - qx) * S;
            const float4 *zb = Z4 + (size_t)(ey + oy) * We + (exx + ox);
#pragma unroll
            for (int t = 0; t < S; ++t)
#pragma unroll
                for (int u = 0; u < S; ++u) {
                    const float4 v = __ldg(zb + (size_t)t * We + u);
                    float wv = wt;
                    if constexpr (HIST) {
                        wv = wt / (1.0f + hex[hist_bin(v.x, nbins)] + hex[nbins + hist_bin(v.y, nbins)] +
                                   hex[2 * nbins + hist_bin(v.z, nbins)]);
                        dpix[t][u] += wv;
                    }
                    num[t][u][0] = fmaf(wv, v.x, num[t][u][0]);
                    num[t][u][1] = fmaf(wv, v.y, num[t][u][1]);
                    num[t][u][2] = fmaf(wv, v.z, num[t][u][2]);
                }
            den += wt;
        }
    }
    if (bad) atomicOr(status, kDevErrBounds);
    if constexpr (SPL > 1) {
#pragma unroll
        for (int m = SPL / 2; m > 0; m >>= 1) {
#pragma unroll
            for (int t = 0; t < S; ++t)
#pragma unroll
                for (int u = 0; u < S; ++u) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) num[t][u][c] += __shfl_xor_sync(0xffffffffu, num[t][u][c], m);
                    if constexpr (HIST) dpix[t][u] += __shfl_xor_sync(0xffffffffu, dpix[t][u], m);
                }
            den += __shfl_xor_sync(0xffffffffu, den, m);
        }
        if (!live || sub != 0) return;
    }
#pragma unroll
    for (int t = 0; t < S; ++t) {
        float *o = out + ((size_t)(py * S + t) * Wo + px * S) * C;
#pragma unroll
        for (int u = 0; u < S; ++u) {
            float d = den;
            if constexpr (HIST) d = dpix[t][u];
#pragma unroll
            for (int c = 0; c < 3; ++c) o[u * C + c] = num[t][u][c] / d;
        }
    }
}

// how many entries of a and b differ (the stopping rule of section 2.1: no window changed)
__global__ void __launch_bounds__(256) k_count_diff(const int *__restrict__ a, const int *__restrict__ b, int n,
                                                    unsigned int *__restrict__ count) {
    unsigned int c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) c += a[i] != b[i] ? 1u : 0u;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) c += __shfl_xor_sync(0xffffffffu, c, s);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

__global__ void k_rgba(const float *__restrict__ Z, long npix, int C, float4 *__restrict__ out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < npix; i += (long)gridDim.x * blockDim.x)
        out[i] = make_float4(Z[C * i], Z[C * i + 1], Z[C * i + 2], C == 4 ? Z[C * i + 3] : 0.0f);
}

// IRLS weights and energy (Eqs. 5-8).  Fixed grid; each block sums its
// grid-stride slice in FP64, tree-reduces, and the last block to finish loads
// the block partials and adds them by the same fixed tree, so the energy is
// bitwise reproducible.
static_assert(kIrlsGrid <= 256, "the last block loads one partial per thread");

__global__ void __launch_bounds__(256)
    k_irls(const float *__restrict__ d2, int Q, float r, float delta, float *__restrict__ wts,
           double *__restrict__ energy_out, double *__restrict__ partial,
           unsigned int *__restrict__ ticket) {
    __shared__ double red[256];
    __shared__ bool last;
    double acc = 0.0;
    const bool quad = (r == 2.0f);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q; i += gridDim.x * blockDim.x) {
        const float t = fmaxf(d2[i], 0.0f);
        if (quad) {
            if (wts) wts[i] = 1.0f;
            acc += (double)t;
        } else {
            const float dp = sqrtf(t);
            if (wts) wts[i] = powf(fmaxf(dp, delta), r - 2.0f);
            acc += (double)powf(dp, r);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = red[0];
        __threadfence();
        last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {  // the whole last block: the partials loaded together, then the same fixed tree
        __threadfence();
        red[threadIdx.x] = threadIdx.x < gridDim.x ? ((volatile double *)partial)[threadIdx.x] : 0.0;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (energy_out) *energy_out = red[0];
            *ticket = 0u;
        }
    }
}

__device__ __forceinline__ int mirror_idx(int i, int n) {
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * (n - 1) - i;
    }
    return i;
}

// binomial [1 4 6 4 1]/16 separable down-sampling by 2, mirrored border
__global__ void k_downsample2(const float *__restrict__ in, int H, int W, float *__restrict__ out) {
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= Wo || y >= Ho) return;
    const float k[5] = {1.0f / 16, 4.0f / 16, 6.0f / 16, 4.0f / 16, 1.0f / 16};
    float s[3] = {0.0f, 0.0f, 0.0f};
    for (int a = 0; a < 5; ++a) {
        const int yy = mirror_idx(2 * y + a - 2, H);
        for (int b = 0; b < 5; ++b) {
            const int xx = mirror_idx(2 * x + b - 2, W);
            const float kk = k[a] * k[b];
            for (int c = 0; c < 3; ++c) s[c] = fmaf(kk, in[((size_t)yy * W + xx) * 3 + c], s[c]);
        }
    }
    for (int c = 0; c < 3; ++c) out[((size_t)y * Wo + x) * 3 + c] = s[c];
}

// bilinear up-sampling by 2 with half-pixel centres, clamped
__global__ void k_upsample2(const float *__restrict__ in, int H, int W, float *__restrict__ out) {
    const int Ho = 2 * H, Wo = 2 * W;
    const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y;
    if (X >= Wo || Y >= Ho) return;
    float sy = (Y + 0.5f) * 0.5f - 0.5f, sx = (X + 0.5f) * 0.5f - 0.5f;
    sy = fminf(fmaxf(sy, 0.0f), (float)(H - 1));
    sx = fminf(fmaxf(sx, 0.0f), (float)(W - 1));
    const int y0 = (int)floorf(sy), x0 = (int)floorf(sx);
    const int y1 = min(y0 + 1, H - 1), x1 = min(x0 + 1, W - 1);
    const float fy = sy - y0, fx = sx - x0;
    for (int c = 0; c < 3; ++c) {
        const float v00 = in[((size_t)y0 * W + x0) * 3 + c], v01 = in[((size_t)y0 * W + x1) * 3 + c];
        const float v10 = in[((size_t)y1 * W + x0) * 3 + c], v11 = in[((size_t)y1 * W + x1) * 3 + c];
        out[((size_t)Y * Wo + X) * 3 + c] =
            (1.0f - fy) * ((1.0f - fx) * v00 + fx * v01) + fy * ((1.0f - fx) * v10 + fx * v11);
    }
}

}  // namespace

void launch_count_diff(const int *a, const int *b, int n, unsigned int *count, cudaStream_t st) {
    cudaMemsetAsync(count, 0, sizeof(unsigned int), st);
    if (n <= 0) return;
    count_launches(1);
    k_count_diff<<<(unsigned)std::min<long>(ceil_div((long)n, 256), 152 * 4), 256, 0, st>>>(a, b, n, count);
}

void launch_rgba(const float *Z, long npix, int C, float4 *out, cudaStream_t st) {
    if (npix <= 0) return;
    count_launches(1);
    k_rgba<<<(unsigned)std::min<long>(ceil_div(npix, 256), 152 * 8), 256, 0, st>>>(Z, npix, C, out);
}

void launch_m_step(const int *nn, const float *wts, const float4 *Z4, int We, int ex, int N, int C, int w,
                   int Ho, int Wo, int stride, float *out, int *status, cudaStream_t st) {
    const int qy_n = (Ho - w) / stride + 1, qx_n = (Wo - w) / stride + 1;
    const int PX = Wo / stride, PY = Ho / stride;
    dim3 block(128), grid(ceil_div(PX, 128), PY);
    ProfScope ps(kProfMStep, st, 1);
    switch (stride) {
        case 1:
            k_m_step<1, false><<<grid, block, 0, st>>>(nn, wts, Z4, We, ex, N, C, w, Ho, Wo, qy_n, qx_n, out, status, 0,
                                                       nullptr, 1, nullptr, 1);
            break;
        case 2: {
            // wide windows cover a patch many times: 4 or 8 threads share a patch's windows
            const int ws = w / 2;
            if (ws >= 16) {
                const dim3 g8(ceil_div(PX, 128 / 8), PY);
                k_m_step<2, false, 8><<<g8, block, 0, st>>>(nn, wts, Z4, We, ex, N, C, w, Ho, Wo, qy_n, qx_n, out,
                                                             status, 0, nullptr, 1, nullptr, 1);
            } else if (ws >= 8) {
                const dim3 g4(ceil_div(PX, 128 / 4), PY);
                k_m_step<2, false, 4><<<g4, block, 0, st>>>(nn, wts, Z4, We, ex, N, C, w, Ho, Wo, qy_n, qx_n, out,
                                                             status, 0, nullptr, 1, nullptr, 1);
            } else {
                k_m_step<2, false><<<grid, block, 0, st>>>(nn, wts, Z4, We, ex, N, C, w, Ho, Wo, qy_n, qx_n, out,
                                                           status, 0, nullptr, 1, nullptr, 1);
            }
            break;
        }
        case 4:
            k_m_step<4, false><<<grid, block, 0, st>>>(nn, wts, Z4, We, ex, N, C, w, Ho, Wo, qy_n, qx_n, out, status, 0,
                                                       nullptr, 1, nullptr, 1);
            break;
        default:
            break;  // rejected by the caller
    }
}

void launch_m_step_hist(const int *nn, const float *wts, const float4 *Z4, int We, int ex, int N, int w, int Ho, int Wo,
                        int stride, int nbins, const unsigned int *cx, long nx, const unsigned int *cz, long nz,
                        float *out, int *status, cudaStream_t st) {
    const int qy_n = (Ho - w) / stride + 1, qx_n = (Wo - w) / stride + 1;
    const int PX = Wo / stride, PY = Ho / stride;
    dim3 block(128), grid(ceil_div(PX, 128), PY);
    ProfScope ps(kProfMStep, st, 1);
    switch (stride) {
        case 1:
            k_m_step<1, true><<<grid, block, 0, st>>>(nn, wts, Z4, We, ex, N, 3, w, Ho, Wo, qy_n, qx_n, out, status,
                                                      nbins, cx, nx, cz, nz);
            break;
        case 2:
            k_m_step<2, true><<<grid, block, 0, st>>>(nn, wts, Z4, We, ex, N, 3, w, Ho, Wo, qy_n, qx_n, out, status,
                                                      nbins, cx, nx, cz, nz);
            break;
        case 4:
            k_m_step<4, true><<<grid, block, 0, st>>>(nn, wts, Z4, We, ex, N, 3, w, Ho, Wo, qy_n, qx_n, out, status,
                                                      nbins, cx, nx, cz, nz);
            break;
        default:
            break;  // rejected by the caller
    }
}

void launch_irls(const float *d2, int Q, float r, float delta, float *wts, double *energy_out,
                 double *partial, unsigned int *ticket, cudaStream_t st) {
    ProfScope ps(kProfIrls, st, 1);
    k_irls<<<kIrlsGrid, 256, 0, st>>>(d2, Q, r, delta, wts, energy_out, partial, ticket);
}

void launch_downsample2(const float *in, int H, int W, float *out, cudaStream_t st) {
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    count_launches(1);
    k_downsample2<<<dim3(ceil_div(Wo, 128), Ho), 128, 0, st>>>(in, H, W, out);
}

void launch_upsample2(const float *in, int H, int W, float *out, cudaStream_t st) {
    count_launches(1);
    k_upsample2<<<dim3(ceil_div(2 * W, 128), 2 * H), 128, 0, st>>>(in, H, W, out);
}

}  // namespace pts

// ---------------------------------------------------------------------------
// irls_weights_noalloc: the IRLS reduction with its scratch in a fixed array
// compiled into the library, for callers that cannot allocate device memory.
// Scratch: one double per block of kNoAllocPerBlock distances plus the
// completion ticket.  The array's device address belongs to a CUDA context: it is
// looked up (cudaGetSymbolAddress) by the first call made in each context and
// cached under the context's process-unique id (cuCtxGetId), so a reset device
// or a second context on the same device gets its own lookup.
// ---------------------------------------------------------------------------
#include <cuda.h>

#include <mutex>
#include <utility>
#include <vector>

namespace pts {
namespace {
constexpr int kNoAllocMaxBlocks = 4096;
constexpr int kNoAllocPerBlock = 256 * 8;
constexpr size_t kNoAllocTicketOffset = kNoAllocMaxBlocks * sizeof(double);
static __device__ __align__(256) unsigned char g_irls_scratch[kNoAllocTicketOffset + 256];

std::mutex g_noalloc_mu;
std::vector<std::pair<unsigned long long, void *>> g_noalloc_addr;  // (context id, array address)

// driver entry points through the runtime, so the library does not link libcuda itself
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

bool load_ctx_entry_points() {
    if (g_ctx_get_current && g_ctx_get_id) return true;
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
        return false;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(a);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(b);
    return true;
}
}  // namespace
}  // namespace pts

extern "C" pts_status irls_weights_noalloc(const float *dist2, int Q, float r, float delta,
                                           float *weights_out, double *energy_out, void *stream) {
    using namespace pts;
    if (!dist2 || Q < 0) return set_error(PTS_ERR_INVALID_ARG, "irls_weights_noalloc: bad input");
    if (!(r > 0.0f && r <= 2.0f) || !(delta > 0.0f))
        return set_error(PTS_ERR_INVALID_ARG, "irls_weights_noalloc: need 0 < r <= 2 and delta > 0");
    if ((long)Q > (long)kNoAllocMaxBlocks * kNoAllocPerBlock)
        return set_error(PTS_ERR_INVALID_ARG,
                         "irls_weights_noalloc: Q exceeds the fixed scratch limit of 8388608 distances");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!load_ctx_entry_points())
            return set_error(PTS_ERR_CUDA, "irls_weights_noalloc: driver context entry points unavailable");
        CUcontext ctx = nullptr;
        unsigned long long ctx_id = 0;
        if (g_ctx_get_current(&ctx) != CUDA_SUCCESS)
            return set_error(PTS_ERR_CUDA, "irls_weights_noalloc: cuCtxGetCurrent failed");
        if (!ctx) {
            // no context current yet: a runtime call makes the device's primary context current
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_irls_scratch);
            if (e != cudaSuccess) return cuda_error(e, "irls_weights_noalloc: cudaGetSymbolAddress");
            if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx)
                return set_error(PTS_ERR_CUDA, "irls_weights_noalloc: no current CUDA context");
        }
        if (g_ctx_get_id(ctx, &ctx_id) != CUDA_SUCCESS)
            return set_error(PTS_ERR_CUDA, "irls_weights_noalloc: cuCtxGetId failed");
        for (const auto &e : g_noalloc_addr)
            if (e.first == ctx_id) base = e.second;
        if (!base) {
            cudaError_t e = cudaGetSymbolAddress(&base, g_irls_scratch);
            if (e != cudaSuccess) return cuda_error(e, "irls_weights_noalloc: cudaGetSymbolAddress");
            g_noalloc_addr.emplace_back(ctx_id, base);
        }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double *partial = static_cast<double *>(base);
    unsigned int *ticket = reinterpret_cast<unsigned int *>(static_cast<char *>(base) + kNoAllocTicketOffset);
    // the array keeps the previous call's contents: the ticket must start at 0
    PTS_CUDA_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st));
    const int grid = Q > 0 ? ceil_div(Q, kNoAllocPerBlock) : 1;
    count_launches(1);
    k_irls<<<grid, 256, 0, st>>>(dist2, Q, r, delta, weights_out, energy_out, partial, ticket);
    PTS_CUDA_TRY(cudaGetLastError());
    return PTS_OK;
}
