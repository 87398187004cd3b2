// scale.cu -- the scale map of the perspective texture (Methodology section 1, Eqs. 1-3) and its
// use in synthesis (section 3): the map itself, its resampling to the output size, the initial
// output filled from exemplar pixels of the same scale, and the RGBS images whose fourth channel
// is the map.
//
// Readings (the paper is silent or garbled here):
//   image-plane origin  the bottom-left pixel, so array row r has p(y) = h - 1 - r and column c
//                       has p(x) = c; w / 2 and h / 2 are real halves;
//   Eq. 3               its leading term, printed as Y_max, is read as S_max (only then is S a
//                       scale: S_max where p(Y_proj) = Y_min, S_min where it is Y_max, and 1 on
//                       a fronto-parallel plane);
//   angles              slant sigma in [0, 90), tilt tau in [0, 90] degrees (section 1 mirrors the
//                       exemplar until its largest texel is at the origin, which keeps sin tau
//                       and cos tau non-negative in Eq. 2); a map with Y_delta = 0 is refused;
//   resampling          bilinear and corner-aligned, so the output spans the exemplar's scales;
//   "the same scale"    the same of nbins equal bins over the exemplar map's range [lo, hi]; an
//                       output pixel copies pixel floor(u m) (u a given uniform) of its bin's m
//                       exemplar pixels in raster order, and an empty bin borrows the nearest
//                       filled one (the lower one on a tie).
// Every value is computed in FP64 with each product, quotient, sum and difference rounded on
// its own (no fused multiply-add) in the order the formulas are written, and the trigonometric
// and Eq. 1-2 scalars are computed on the host, so the maps and bins are reproducible bit for
// bit by any IEEE FP64 evaluation of the same formulas.
#include <math.h>

#include <string>

#include "pts_internal.cuh"

namespace pts {
namespace {

constexpr int kChunk = 1024;     // exemplar pixels per block of the bin counting sort
constexpr int kMaxBins = 1024;

// Eq. 3 for every pixel: S = S_max - ((p(Y_proj) - Y_min) S_delta) / Y_delta with
// p(Y_proj) = (p(x) - w/2) sin tau + (p(y) - h/2) cos tau.
__global__ void k_scale_map(int h, int w, double sin_t, double cos_t, double s_max, double s_delta, double y_min,
                            double y_delta, double *__restrict__ S) {
    const long n = (long)h * w;
    const double hw = (double)w / 2.0, hh = (double)h / 2.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / w), c = (int)(i - (long)r * w);
        const double px = (double)c, py = (double)(h - 1 - r);
        const double proj = __dadd_rn(__dmul_rn(__dsub_rn(px, hw), sin_t), __dmul_rn(__dsub_rn(py, hh), cos_t));
        S[i] = __dsub_rn(s_max, __ddiv_rn(__dmul_rn(__dsub_rn(proj, y_min), s_delta), y_delta));
    }
}

// bilinear, corner-aligned: output (xo, yo) reads the map at ((We-1) xo / (Wo-1), (He-1) yo / (Ho-1))
__global__ void k_scale_resample(const double *__restrict__ S, int He, int We, int Ho, int Wo,
                                 double *__restrict__ out) {
    const long n = (long)Ho * Wo;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int yo = (int)(i / Wo), xo = (int)(i - (long)yo * Wo);
        const double sy = __ddiv_rn((double)((long)(He - 1) * yo), (double)(Ho - 1));
        const double sx = __ddiv_rn((double)((long)(We - 1) * xo), (double)(Wo - 1));
        const int y0 = min((int)floor(sy), He - 2), x0 = min((int)floor(sx), We - 2);
        const double fy = __dsub_rn(sy, (double)y0), fx = __dsub_rn(sx, (double)x0);
        const double gx = __dsub_rn(1.0, fx), gy = __dsub_rn(1.0, fy);
        const double *r0 = S + (size_t)y0 * We + x0, *r1 = r0 + We;
        const double top = __dadd_rn(__dmul_rn(gx, r0[0]), __dmul_rn(fx, r0[1]));
        const double bot = __dadd_rn(__dmul_rn(gx, r1[0]), __dmul_rn(fx, r1[1]));
        out[i] = __dadd_rn(__dmul_rn(gy, top), __dmul_rn(fy, bot));
    }
}

// min and max of the exemplar's map (one block; min/max are exact, so the order does not matter)
__global__ void __launch_bounds__(1024) k_range(const double *__restrict__ S, long n, double *__restrict__ lohi) {
    __shared__ double lo_s[1024], hi_s[1024];
    double lo = INFINITY, hi = -INFINITY;
    for (long i = threadIdx.x; i < n; i += blockDim.x) {
        lo = fmin(lo, S[i]);
        hi = fmax(hi, S[i]);
    }
    lo_s[threadIdx.x] = lo;
    hi_s[threadIdx.x] = hi;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            lo_s[threadIdx.x] = fmin(lo_s[threadIdx.x], lo_s[threadIdx.x + o]);
            hi_s[threadIdx.x] = fmax(hi_s[threadIdx.x], hi_s[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        lohi[0] = lo_s[0];
        lohi[1] = hi_s[0];
    }
}

// bin of a scale: floor(((s - lo) / (hi - lo)) nbins) clamped to [0, nbins - 1]; 0 when hi <= lo
__device__ __forceinline__ int scale_bin(double s, double lo, double hi, int nbins) {
    if (!(hi > lo)) return 0;
    const double f = floor(__dmul_rn(__ddiv_rn(__dsub_rn(s, lo), __dsub_rn(hi, lo)), (double)nbins));
    return f < 0.0 ? 0 : (f > (double)(nbins - 1) ? nbins - 1 : (int)f);
}

// per chunk of exemplar pixels: the bin of each pixel and the chunk's count per bin
__global__ void __launch_bounds__(kChunk) k_bin_count(const double *__restrict__ S, long n, const double *__restrict__ lohi,
                                                      int nbins, int *__restrict__ bin_of, int *__restrict__ counts) {
    __shared__ int cnt[kMaxBins];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    const long i = (long)blockIdx.x * kChunk + threadIdx.x;
    if (i < n) {
        const int b = scale_bin(S[i], lohi[0], lohi[1], nbins);
        bin_of[i] = b;
        atomicAdd(&cnt[b], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) counts[(size_t)blockIdx.x * nbins + b] = cnt[b];
}

// one block: every bin's total and first slot, each chunk's first slot within each bin, and the
// bin each output bin reads from (itself if filled, else the nearest filled one, lower on a tie)
__global__ void __launch_bounds__(kMaxBins) k_bin_offsets(const int *__restrict__ counts, int nchunks, int nbins,
                                                          int *__restrict__ total, int *__restrict__ bin_off,
                                                          int *__restrict__ chunk_off, int *__restrict__ src_bin) {
    __shared__ int tot[kMaxBins], off[kMaxBins];
    const int b = threadIdx.x;
    int t = 0;
    if (b < nbins)
        for (int c = 0; c < nchunks; ++c) t += counts[(size_t)c * nbins + b];
    tot[b] = b < nbins ? t : 0;
    __syncthreads();
    if (b == 0) {
        int run = 0;
        for (int k = 0; k < nbins; ++k) {
            off[k] = run;
            run += tot[k];
        }
    }
    __syncthreads();
    if (b < nbins) {
        total[b] = tot[b];
        bin_off[b] = off[b];
        int run = off[b];
        for (int c = 0; c < nchunks; ++c) {
            chunk_off[(size_t)c * nbins + b] = run;
            run += counts[(size_t)c * nbins + b];
        }
        int s = -1;
        for (int dist = 0; dist < nbins && s < 0; ++dist) {
            if (b - dist >= 0 && tot[b - dist] > 0)
                s = b - dist;
            else if (b + dist < nbins && tot[b + dist] > 0)
                s = b + dist;
        }
        src_bin[b] = s < 0 ? 0 : s;
    }
}

// stable scatter: a pixel's slot is its chunk's first slot in its bin plus the number of earlier
// pixels of the chunk in the same bin, so every bin lists its pixels in raster order
__global__ void __launch_bounds__(kChunk) k_bin_scatter(const int *__restrict__ bin_of, long n, int nbins,
                                                        const int *__restrict__ chunk_off, int *__restrict__ members) {
    __shared__ int bins[kChunk];
    const long i = (long)blockIdx.x * kChunk + threadIdx.x;
    bins[threadIdx.x] = i < n ? bin_of[i] : -1;
    __syncthreads();
    if (i >= n) return;
    const int b = bins[threadIdx.x];
    int rank = 0;
    for (int j = 0; j < (int)threadIdx.x; ++j) rank += bins[j] == b ? 1 : 0;
    members[chunk_off[(size_t)blockIdx.x * nbins + b] + rank] = (int)i;
}

// each output pixel copies one exemplar pixel of its scale bin (section 3, step 3)
__global__ void k_guided_gather(const float *__restrict__ Z, const double *__restrict__ Sx, const double *__restrict__ u,
                                long n, const double *__restrict__ lohi, int nbins, const int *__restrict__ total,
                                const int *__restrict__ bin_off, const int *__restrict__ src_bin,
                                const int *__restrict__ members, float *__restrict__ out, int *__restrict__ src_out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int sb = src_bin[scale_bin(Sx[i], lohi[0], lohi[1], nbins)];
        const int m = total[sb];
        const double f = floor(__dmul_rn(u[i], (double)m));
        const int k = f < 0.0 ? 0 : (f > (double)(m - 1) ? m - 1 : (int)f);
        const int src = members[bin_off[sb] + k];
        out[3 * i] = Z[3 * (size_t)src];
        out[3 * i + 1] = Z[3 * (size_t)src + 1];
        out[3 * i + 2] = Z[3 * (size_t)src + 2];
        if (src_out) src_out[i] = src;
    }
}

__global__ void k_rgbs(const float *__restrict__ rgb, const double *__restrict__ S, double lam, long n,
                       float4 *__restrict__ out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        out[i] = make_float4(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], (float)__dmul_rn(lam, S[i]));
}

__global__ void k_rgb_of(const float4 *__restrict__ in, long n, float *__restrict__ rgb) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float4 v = in[i];
        rgb[3 * i] = v.x;
        rgb[3 * i + 1] = v.y;
        rgb[3 * i + 2] = v.z;
    }
}

unsigned grid_for(long n) { return (unsigned)std::max<long>(1, std::min<long>(ceil_div(n, 256), 152 * 8)); }

constexpr long kMaxPixels = 1L << 26;

}  // namespace
}  // namespace pts

using namespace pts;

extern "C" {

pts_status pts_scale_map(int h, int w, double slant_deg, double tilt_deg, double *S_out, void *stream) {
    if (!S_out) return set_error(PTS_ERR_INVALID_ARG, "pts_scale_map: null output");
    if (h < 1 || w < 1 || (long)h * w > kMaxPixels) return set_error(PTS_ERR_INVALID_ARG, "pts_scale_map: bad size");
    if (!(slant_deg >= 0.0 && slant_deg < 90.0))
        return set_error(PTS_ERR_INVALID_ARG, "pts_scale_map: slant must lie in [0, 90) degrees");
    if (!(tilt_deg >= 0.0 && tilt_deg <= 90.0))
        return set_error(PTS_ERR_INVALID_ARG, "pts_scale_map: tilt must lie in [0, 90] degrees");
    const double deg = M_PI / 180.0;
    // Eq. 1
    const double c = cos(slant_deg * deg);
    const double s_max = 1.0 / c, s_min = c, s_delta = s_max - s_min;
    // Eq. 2
    const double t = tilt_deg * deg, sin_t = sin(t), cos_t = cos(t);
    volatile double a = (double)(w - 1) - w / 2.0, b = (double)(h - 1) - h / 2.0;  // no contraction
    volatile double pa = a * sin_t, pb = b * cos_t;
    const double y_max = pa + pb, y_min = -y_max, y_delta = y_max - y_min;
    if (!(y_delta > 0.0))
        return set_error(PTS_ERR_INVALID_ARG, "pts_scale_map: Y_delta = 0 (no extent along the projected axis)");
    count_launches(1);
    k_scale_map<<<grid_for((long)h * w), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        h, w, sin_t, cos_t, s_max, s_delta, y_min, y_delta, S_out);
    PTS_CUDA_TRY(cudaGetLastError());
    return PTS_OK;
}

pts_status pts_scale_resample(const double *S, int He, int We, int Ho, int Wo, double *S_out, void *stream) {
    if (!S || !S_out) return set_error(PTS_ERR_INVALID_ARG, "pts_scale_resample: null pointer");
    if (He < 2 || We < 2 || Ho < 2 || Wo < 2 || (long)Ho * Wo > kMaxPixels || (long)He * We > kMaxPixels)
        return set_error(PTS_ERR_INVALID_ARG, "pts_scale_resample: both maps need at least 2 x 2 pixels");
    count_launches(1);
    k_scale_resample<<<grid_for((long)Ho * Wo), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(S, He, We, Ho, Wo,
                                                                                                 S_out);
    PTS_CUDA_TRY(cudaGetLastError());
    return PTS_OK;
}

pts_status pts_scale_guided_init(const float *exemplar, const double *S_z, int He, int We, const double *S_x,
                                 const double *u, int Ho, int Wo, int nbins, float *out, int32_t *src_out,
                                 void *stream) {
    if (!exemplar || !S_z || !S_x || !u || !out)
        return set_error(PTS_ERR_INVALID_ARG, "pts_scale_guided_init: null pointer");
    if (He < 1 || We < 1 || Ho < 1 || Wo < 1 || (long)He * We > kMaxPixels || (long)Ho * Wo > kMaxPixels)
        return set_error(PTS_ERR_INVALID_ARG, "pts_scale_guided_init: bad size");
    if (nbins < 1 || nbins > kMaxBins) return set_error(PTS_ERR_INVALID_ARG, "pts_scale_guided_init: nbins in 1..1024");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long nz = (long)He * We, nx = (long)Ho * Wo;
    const int nchunks = (int)ceil_div(nz, kChunk);
    DevBuf<double> lohi;
    DevBuf<int> bin_of, counts, total, bin_off, chunk_off, src_bin, members;
    PTS_TRY(lohi.ensure(2, "scale range"));
    PTS_TRY(bin_of.ensure(nz, "scale bins"));
    PTS_TRY(counts.ensure((size_t)nchunks * nbins, "scale bin counts"));
    PTS_TRY(chunk_off.ensure((size_t)nchunks * nbins, "scale bin offsets"));
    PTS_TRY(total.ensure(nbins, "scale bin totals"));
    PTS_TRY(bin_off.ensure(nbins, "scale bin starts"));
    PTS_TRY(src_bin.ensure(nbins, "scale bin sources"));
    PTS_TRY(members.ensure(nz, "scale bin members"));
    count_launches(5);
    k_range<<<1, 1024, 0, st>>>(S_z, nz, lohi.ptr);
    k_bin_count<<<nchunks, kChunk, 0, st>>>(S_z, nz, lohi.ptr, nbins, bin_of.ptr, counts.ptr);
    k_bin_offsets<<<1, kMaxBins, 0, st>>>(counts.ptr, nchunks, nbins, total.ptr, bin_off.ptr, chunk_off.ptr,
                                          src_bin.ptr);
    k_bin_scatter<<<nchunks, kChunk, 0, st>>>(bin_of.ptr, nz, nbins, chunk_off.ptr, members.ptr);
    k_guided_gather<<<grid_for(nx), 256, 0, st>>>(exemplar, S_x, u, nx, lohi.ptr, nbins, total.ptr, bin_off.ptr,
                                                  src_bin.ptr, members.ptr, out, src_out);
    PTS_CUDA_TRY(cudaGetLastError());
    PTS_CUDA_TRY(cudaStreamSynchronize(st));  // the scratch goes back before returning
    return PTS_OK;
}

pts_status pts_rgbs(const float *rgb, const double *S, double lam, int H, int W, float *out, void *stream) {
    if (!rgb || !S || !out) return set_error(PTS_ERR_INVALID_ARG, "pts_rgbs: null pointer");
    if (H < 1 || W < 1 || (long)H * W > kMaxPixels) return set_error(PTS_ERR_INVALID_ARG, "pts_rgbs: bad size");
    if (reinterpret_cast<uintptr_t>(out) % 16) return set_error(PTS_ERR_INVALID_ARG, "pts_rgbs: out not 16-byte aligned");
    count_launches(1);
    k_rgbs<<<grid_for((long)H * W), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        rgb, S, lam, (long)H * W, reinterpret_cast<float4 *>(out));
    PTS_CUDA_TRY(cudaGetLastError());
    return PTS_OK;
}

pts_status pts_rgb_of(const float *rgbs, int H, int W, float *rgb_out, void *stream) {
    if (!rgbs || !rgb_out) return set_error(PTS_ERR_INVALID_ARG, "pts_rgb_of: null pointer");
    if (H < 1 || W < 1 || (long)H * W > kMaxPixels) return set_error(PTS_ERR_INVALID_ARG, "pts_rgb_of: bad size");
    if (reinterpret_cast<uintptr_t>(rgbs) % 16)
        return set_error(PTS_ERR_INVALID_ARG, "pts_rgb_of: input not 16-byte aligned");
    count_launches(1);
    k_rgb_of<<<grid_for((long)H * W), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const float4 *>(rgbs), (long)H * W, rgb_out);
    PTS_CUDA_TRY(cudaGetLastError());
    return PTS_OK;
}

}  // extern "C"
