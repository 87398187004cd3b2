// histogram.cu -- histogram matching (section 3, Eq. 9; the last step of the synthesis procedure,
// section 4): per-channel histograms of an image and the final mapping of an image's channels
// onto the exemplar's distribution.  The M-step with the weights of Eq. 9 is k_m_step<S, true>
// in mstep.cu.
//
// Histograms: one per colour channel, nbins equal bins over [0, 1] holding integer pixel counts
// (shared-memory atomics per block, one global atomic per non-empty bin: deterministic).  The bin
// of a value: clamped to [0, 1], times nbins in FP32, floored, capped at the last bin.
//
// Final matching: v -> F_z^-1(F_x(v)) per channel, both CDFs piecewise linear inside the bins
// (C[m] = fraction of pixels below bin m from the integer counts, h[m] the bin's fraction):
// F_x(v) = C_x[b] + (v nbins - b) h_x[b] for v in bin b, and F_z^-1(u) = (m + (u - C_z[m]) /
// h_z[m]) / nbins for the bin m with C_z[m] <= u < C_z[m+1] (never an empty one), 1 beyond.
#include <algorithm>

#include "pts_internal.cuh"

namespace pts {
namespace {

__global__ void __launch_bounds__(256) k_hist3(const float *__restrict__ img, long npix, int nbins,
                                               unsigned int *__restrict__ counts) {
    __shared__ unsigned int sh[3 * kMaxHistBins];
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < npix; p += (long)gridDim.x * blockDim.x) {
        const float *px = img + 3 * p;
        atomicAdd(&sh[hist_bin(px[0], nbins)], 1u);
        atomicAdd(&sh[nbins + hist_bin(px[1], nbins)], 1u);
        atomicAdd(&sh[2 * nbins + hist_bin(px[2], nbins)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x)
        if (sh[i]) atomicAdd(&counts[i], sh[i]);
}

__global__ void __launch_bounds__(256) k_hist_match(float *__restrict__ img, long npix, int nbins,
                                                    const unsigned int *__restrict__ cx, long nx,
                                                    const unsigned int *__restrict__ cz, long nz) {
    __shared__ float Cx[3][kMaxHistBins + 1], Cz[3][kMaxHistBins + 1], hx[3][kMaxHistBins], hz[3][kMaxHistBins];
    if (threadIdx.x < 3) {
        const int j = threadIdx.x;
        unsigned long long ax = 0, az = 0;
        Cx[j][0] = 0.0f;
        Cz[j][0] = 0.0f;
        for (int b = 0; b < nbins; ++b) {
            const unsigned int kx = cx[j * nbins + b], kz = cz[j * nbins + b];
            ax += kx;
            az += kz;
            Cx[j][b + 1] = (float)((double)ax / (double)nx);
            Cz[j][b + 1] = (float)((double)az / (double)nz);
            hx[j][b] = (float)((double)kx / (double)nx);
            hz[j][b] = (float)((double)kz / (double)nz);
        }
    }
    __syncthreads();
    const float fb = (float)nbins;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * npix; i += (long)gridDim.x * blockDim.x) {
        const int j = (int)(i % 3);
        const float v = img[i];
        const float c = fminf(fmaxf(v, 0.0f), 1.0f);
        const int b = hist_bin(v, nbins);
        const float u = Cx[j][b] + (c * fb - (float)b) * hx[j][b];
        // m = how many of C_z[1..nbins] are <= u (C_z is non-decreasing)
        int lo = 0, hi = nbins;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Cz[j][mid + 1] <= u)
                lo = mid + 1;
            else
                hi = mid;
        }
        img[i] = lo < nbins ? ((float)lo + (u - Cz[j][lo]) / hz[j][lo]) / fb : 1.0f;
    }
}

}  // namespace

void launch_hist3(const float *img, long npix, int nbins, unsigned int *counts, cudaStream_t st) {
    cudaMemsetAsync(counts, 0, sizeof(unsigned int) * 3 * nbins, st);
    if (npix <= 0) return;
    count_launches(1);
    k_hist3<<<(unsigned)std::min<long>(ceil_div(npix, 256), 152 * 4), 256, 0, st>>>(img, npix, nbins, counts);
}

void launch_hist_match(float *img, long npix, int nbins, const unsigned int *cx, long nx, const unsigned int *cz,
                       long nz, cudaStream_t st) {
    if (npix <= 0) return;
    count_launches(1);
    k_hist_match<<<(unsigned)std::min<long>(ceil_div(3 * npix, 256), 152 * 4), 256, 0, st>>>(img, npix, nbins, cx,
                                                                                              nx, cz, nz);
}

}  // namespace pts
