// pca.cu -- PCA of the exemplar neighbourhood vectors (section 2.2) in FP64.
//
//   mu    = (1/N) sum_n v_n                         k_win_mean
//   Sigma = (1/N) sum_n (v_n - mu)(v_n - mu)^T      k_cov (+ k_cov_reduce)
// Windows are gathered from the image on the fly (no N x D matrix).  Sigma
// is accumulated as a split-K tiled FP64 GEMM over n; the slices are added
// in slice order, so the result is deterministic.
//
// Top-d eigenpairs: block subspace iteration with Rayleigh-Ritz (Golub & Van
// Loan, "Matrix Computations", section 8.2.4; Saad, "Numerical Methods for
// Large Eigenvalue Problems", chapter 5) on m = d + max(16, d/2) vectors:
//   Y = Sigma V;  H = V^T Y;  H = S Theta S^T (Jacobi, one CTA);
//   Vr = V S, Yr = Y S;  stop when ||Yr_j - theta_j Vr_j|| <= 1e-12 theta_1
//   for all j < d, else V = orth(Yr) and repeat.
// orth() is Cholesky QR applied twice (G = V^T V = L L^T, V <- V L^-T).
#include <math.h>

#include <algorithm>
#include <vector>

#include "pts_internal.cuh"

namespace pts {
namespace {

constexpr int kMaxM = 112;     // subspace widths up to this keep the m x m work in shared memory
constexpr int kMaxMBig = 256;  // beyond it (up to this) the m x m matrices live in global memory
constexpr int kRitzEvery = 4;  // subspace-iteration steps per Rayleigh-Ritz solve

__global__ void __launch_bounds__(256)
    k_win_mean(const float *__restrict__ Z, int We, int C, int w, int ex, long N, double *__restrict__ mu) {
    __shared__ double red[256];
    const int k = blockIdx.x;
    const int row = C * w;
    const int dy = k / row, rem = k - dy * row;
    double acc = 0.0;
    for (long n = threadIdx.x; n < N; n += 256) {
        const long ey = n / ex, exx = n - ey * ex;
        acc += (double)Z[((ey + dy) * We + exx) * C + rem];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) mu[k] = red[0] / (double)N;
}

// partial covariance of n in [slice*slice_len, ...) for the 64x64 tile pair
// (bi, bj), bi <= bj, enumerated by blockIdx.x
__global__ void __launch_bounds__(256)
    k_cov(const float *__restrict__ Z, int We, int C, int w, int ex, long N, const double *__restrict__ mu,
          int D, int T, long slice_len, double *__restrict__ part) {
    __shared__ double sA[16][64 + 1];
    __shared__ double sB[16][64 + 1];
    __shared__ int koffA[64], koffB[64];
    __shared__ double muA[64], muB[64];
    // decode tile pair
    int rem = blockIdx.x, bi = 0;
    while (rem >= T - bi) {
        rem -= T - bi;
        ++bi;
    }
    const int bj = bi + rem;
    const int row = C * w;
    const int tid = threadIdx.x;
    if (tid < 64) {
        const int k = bi * 64 + tid;
        const int kk = k < D ? k : 0;
        koffA[tid] = (kk / row) * We * C + (kk % row);
        muA[tid] = k < D ? mu[k] : 0.0;
    } else if (tid < 128) {
        const int k = bj * 64 + tid - 64;
        const int kk = k < D ? k : 0;
        koffB[tid - 64] = (kk / row) * We * C + (kk % row);
        muB[tid - 64] = k < D ? mu[k] : 0.0;
    }
    __syncthreads();
    const long n0 = (long)blockIdx.y * slice_len;
    const long n1 = min(N, n0 + slice_len);
    const int ti = tid >> 4, tj = tid & 15;
    double acc[4][4] = {};
    for (long nb = n0; nb < n1; nb += 16) {
        for (int idx = tid; idx < 16 * 64; idx += 256) {
            const int t = idx >> 6, c = idx & 63;
            const long n = nb + t;
            double va = 0.0, vb = 0.0;
            if (n < n1) {
                const long ey = n / ex, exx = n - ey * ex;
                const long base = (ey * We + exx) * C;
                if (bi * 64 + c < D) va = (double)Z[base + koffA[c]] - muA[c];
                if (bj * 64 + c < D) vb = (double)Z[base + koffB[c]] - muB[c];
            }
            sA[t][c] = va;
            sB[t][c] = vb;
        }
        __syncthreads();
#pragma unroll 4
        for (int t = 0; t < 16; ++t) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[t][ti * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sB[t][tj * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double *P = part + (size_t)blockIdx.y * D * D;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gi = bi * 64 + ti * 4 + i;
        if (gi >= D) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gj = bj * 64 + tj * 4 + j;
            if (gj < D) P[(size_t)gi * D + gj] = acc[i][j];
        }
    }
}

__global__ void k_cov_reduce(const double *__restrict__ part, int ns, int D, long N,
                             double *__restrict__ C) {
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)D * D) return;
    const int i = (int)(idx / D), j = (int)(idx % D);
    if (i / 64 > j / 64) return;
    double s = 0.0;
    for (int t = 0; t < ns; ++t) s += part[(size_t)t * D * D + idx];
    s /= (double)N;
    C[(size_t)i * D + j] = s;
    C[(size_t)j * D + i] = s;
}

// C[M x N] = op(A) op(B), row-major; op(A)[i][k] = TA ? A[k*lda+i] : A[i*lda+k]
template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
    k_dgemm(int M, int N, int K, const double *__restrict__ A, int lda, const double *__restrict__ B,
            int ldb, double *__restrict__ C, int ldc) {
    __shared__ double sA[16][64 + 1];
    __shared__ double sB[16][64 + 1];
    const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int idx = tid; idx < 16 * 64; idx += 256) {
            const int t = idx >> 6, c = idx & 63;
            const int k = k0 + t;
            const int i = i0 + c, j = j0 + c;
            sA[t][c] = (k < K && i < M) ? (TA ? A[(size_t)k * lda + i] : A[(size_t)i * lda + k]) : 0.0;
            sB[t][c] = (k < K && j < N) ? (TB ? B[(size_t)j * ldb + k] : B[(size_t)k * ldb + j]) : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int t = 0; t < 16; ++t) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[t][ti * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sB[t][tj * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gi = i0 + ti * 4 + i;
        if (gi >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gj = j0 + tj * 4 + j;
            if (gj < N) C[(size_t)gi * ldc + gj] = acc[i][j];
        }
    }
}

// Cholesky G = L L^T of an m x m SPD matrix, one CTA, in place (lower part).
__global__ void __launch_bounds__(512) k_chol(double *__restrict__ G, int m, int in_global,
                                              int *__restrict__ status) {
    extern __shared__ double sG_dyn[];
    double *sG = in_global ? G : sG_dyn;
    const int tid = threadIdx.x;
    if (!in_global)
        for (int i = tid; i < m * m; i += blockDim.x) sG[i] = G[i];
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        if (tid == 0) {
            double piv = sG[k * m + k];
            if (!(piv > 0.0)) {
                atomicOr(status, kDevErrNumeric);
                piv = 1e-300;
            }
            sG[k * m + k] = sqrt(piv);
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < m; i += blockDim.x) sG[i * m + k] /= sG[k * m + k];
        __syncthreads();
        const int r = m - k - 1;
        for (int idx = tid; idx < r * r; idx += blockDim.x) {
            const int i = k + 1 + idx / r, j = k + 1 + idx % r;
            if (j <= i) sG[i * m + j] -= sG[i * m + k] * sG[j * m + k];
        }
        __syncthreads();
    }
    for (int i = tid; i < m * m; i += blockDim.x) {
        const int r = i / m, c = i % m;
        G[i] = (c <= r) ? sG[i] : 0.0;
    }
}

// rows of V (rows x m) <- row * L^-T, i.e. solve L x^T = row^T
__global__ void k_trsm_rows(double *__restrict__ V, int rows, int m, const double *__restrict__ L) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    double *v = V + (size_t)r * m;
    for (int j = 0; j < m; ++j) {
        double s = v[j];
        for (int i = 0; i < j; ++i) s -= L[j * m + i] * v[i];
        v[j] = s / L[j * m + j];
    }
}

// Jacobi eigen-decomposition of a small symmetric matrix in one CTA, same
// rotation, ordering and thresholds as the classical method (Golub & Van
// Loan section 8.5).  evals descending; Vout[k*m + j] = component k of
// eigenvector j.
__global__ void __launch_bounds__(512)
    k_jacobi_small(const double *__restrict__ Hin, int m, double *__restrict__ evals,
                   double *__restrict__ Vout, double *__restrict__ work, int *__restrict__ status) {
    extern __shared__ double sm_j[];
    // work != NULL: H and V live in that global scratch (2 m^2 doubles) instead
    double *sH = work ? work : sm_j;
    double *sV = sH + m * m;
    __shared__ int pp[kMaxMBig / 2 + 1], qq[kMaxMBig / 2 + 1], act[kMaxMBig / 2 + 1];
    __shared__ double cc[kMaxMBig / 2 + 1], ss[kMaxMBig / 2 + 1];
    __shared__ int nrot, np_sh;
    __shared__ double fro_sh;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < m * m; i += nt) {
        const int r = i / m, c = i % m;
        sH[i] = 0.5 * (Hin[r * m + c] + Hin[c * m + r]);
        sV[i] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        double f = 0.0;
        for (int i = 0; i < m * m; ++i) f += sH[i] * sH[i];
        fro_sh = sqrt(f);
    }
    __syncthreads();
    const double floor_abs = 1e-18 * fro_sh;
    const int mm = (m % 2) ? m + 1 : m;
    bool converged = false;
    for (int sweep = 0; sweep < 60 && !converged; ++sweep) {
        if (tid == 0) nrot = 0;
        __syncthreads();
        for (int r = 0; r < mm - 1; ++r) {
            if (tid == 0) {
                int np = 0;
                for (int k = 0; k < mm / 2; ++k) {
                    int a, b;
                    if (k == 0) {
                        a = mm - 1;
                        b = r;
                    } else {
                        a = (r + k) % (mm - 1);
                        b = (r - k + (mm - 1)) % (mm - 1);
                    }
                    if (a >= m || b >= m) continue;
                    pp[np] = a < b ? a : b;
                    qq[np] = a < b ? b : a;
                    ++np;
                }
                np_sh = np;
            }
            __syncthreads();
            const int np = np_sh;
            if (tid < np) {
                const int p = pp[tid], q = qq[tid];
                const double apq = sH[p * m + q], app = sH[p * m + p], aqq = sH[q * m + q];
                act[tid] = 0;
                if (!(fabs(apq) <= floor_abs || fabs(apq) <= 1e-16 * sqrt(fabs(app * aqq)))) {
                    const double tau = (aqq - app) / (2.0 * apq);
                    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    cc[tid] = 1.0 / sqrt(1.0 + t * t);
                    ss[tid] = t * cc[tid];
                    act[tid] = 1;
                    atomicAdd(&nrot, 1);
                }
            }
            __syncthreads();
            for (int idx = tid; idx < np * m; idx += nt) {  // rows: H <- J^T H
                const int k = idx / m, j = idx % m;
                if (!act[k]) continue;
                const int p = pp[k], q = qq[k];
                const double ap = sH[p * m + j], aq = sH[q * m + j];
                sH[p * m + j] = cc[k] * ap - ss[k] * aq;
                sH[q * m + j] = ss[k] * ap + cc[k] * aq;
            }
            __syncthreads();
            for (int idx = tid; idx < np * m; idx += nt) {  // columns: H <- H J, V <- V J
                const int k = idx / m, i = idx % m;
                if (!act[k]) continue;
                const int p = pp[k], q = qq[k];
                const double ap = sH[i * m + p], aq = sH[i * m + q];
                sH[i * m + p] = cc[k] * ap - ss[k] * aq;
                sH[i * m + q] = ss[k] * ap + cc[k] * aq;
                const double vp = sV[i * m + p], vq = sV[i * m + q];
                sV[i * m + p] = cc[k] * vp - ss[k] * vq;
                sV[i * m + q] = ss[k] * vp + cc[k] * vq;
            }
            __syncthreads();
            if (tid < np && act[tid]) {
                sH[pp[tid] * m + qq[tid]] = 0.0;
                sH[qq[tid] * m + pp[tid]] = 0.0;
            }
            __syncthreads();
        }
        converged = (nrot == 0);
        __syncthreads();
    }
    if (!converged && tid == 0) atomicOr(status, kDevErrNumeric);
    // order by decreasing eigenvalue (thread 0 computes the permutation)
    __shared__ int ord[kMaxMBig];
    if (tid == 0) {
        for (int i = 0; i < m; ++i) ord[i] = i;
        for (int i = 0; i < m; ++i) {
            int b = i;
            for (int j = i + 1; j < m; ++j)
                if (sH[ord[j] * m + ord[j]] > sH[ord[b] * m + ord[b]]) b = j;
            const int t = ord[i];
            ord[i] = ord[b];
            ord[b] = t;
        }
    }
    __syncthreads();
    for (int j = tid; j < m; j += nt) evals[j] = sH[ord[j] * m + ord[j]];
    for (int idx = tid; idx < m * m; idx += nt) {
        const int k = idx / m, j = idx % m;
        Vout[k * m + j] = sV[k * m + ord[j]];
    }
}

// res[j] = || Yr[:, j] - theta_j Vr[:, j] ||  (columns of D x m row-major)
__global__ void k_ritz_residual(const double *__restrict__ Yr, const double *__restrict__ Vr,
                                const double *__restrict__ th, int D, int m, int d,
                                double *__restrict__ res) {
    __shared__ double red[256];
    const int j = blockIdx.x;
    if (j >= d) return;
    double acc = 0.0;
    for (int k = threadIdx.x; k < D; k += 256) {
        const double r = Yr[(size_t)k * m + j] - th[j] * Vr[(size_t)k * m + j];
        acc += r * r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) res[j] = sqrt(red[0]);
}

__global__ void k_init_subspace(double *__restrict__ V, long count) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1) + 12345ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        V[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
}

__global__ void k_diag(const double *__restrict__ C, int D, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < D) out[i] = C[(size_t)i * D + i];
}

__global__ void k_export_basis(const double *__restrict__ Vr, int D, int m, int d,
                               const double *__restrict__ mu64, float *__restrict__ basis,
                               float *__restrict__ mean) {
    const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx < (long)d * D) {
        const int j = (int)(idx / D), k = (int)(idx % D);
        basis[idx] = (float)Vr[(size_t)k * m + j];
    }
    if (mean && idx < D) mean[idx] = (float)mu64[idx];
}

template <bool TA, bool TB>
void dgemm(int M, int N, int K, const double *A, int lda, const double *B, int ldb, double *C,
           int ldc, cudaStream_t st) {
    dim3 grid(ceil_div(N, 64), ceil_div(M, 64));
    count_launches(1);
    k_dgemm<TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc);
}

struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch() {
        for (void *p : ptrs) dev_free(p);
    }
    template <typename T>
    pts_status get(T **p, size_t n, const char *what) {
        void *q = nullptr;
        *p = nullptr;
        PTS_TRY(dev_alloc(&q, std::max<size_t>(n, 1) * sizeof(T), what));
        *p = static_cast<T *>(q);
        ptrs.push_back(q);
        return PTS_OK;
    }
};

}  // namespace

pts_status pca_fit_device(const float *exemplar, int He, int We, int nch, int w, int d, double var_frac,
                          int max_iters, float *mean_out, float *basis_out, double *eig_out,
                          int *d_used, double *var_retained, double *eig_top, int *iters_used,
                          double *trace_out, int *status, cudaStream_t st) {
    const int D = nch * w * w;
    const int ex = We - w + 1;
    const long N = (long)(He - w + 1) * ex;
    int dd = d > 0 ? d : kMaxD;
    dd = std::min<long>(std::min(dd, D), N - 1);
    if (dd < 1) return set_error(PTS_ERR_INVALID_ARG, "pca_fit: too few exemplar windows");
    if (d > 0 && d > dd) return set_error(PTS_ERR_INVALID_ARG, "pca_fit: d exceeds min(D, N-1)");
    int m = std::min<long>(std::min<long>(D, N - 1), dd + std::max(16, dd / 2));
    m = std::min(m, kMaxMBig);
    if (max_iters <= 0) max_iters = 200;

    Scratch sc;
    double *mu64, *C, *part, *V, *Y, *Vr, *Yr, *G, *S, *th, *res, *diag;
    const int T = ceil_div(D, 64);
    const int npairs = T * (T + 1) / 2;
    int ns = std::max(1, std::min(64, ceil_div(304, npairs)));
    ns = std::min<long>(ns, std::max(1L, N / 64));
    const long slice_len = (N + ns - 1) / ns;
    PTS_TRY(sc.get(&mu64, D, "pca mean"));
    PTS_TRY(sc.get(&C, (size_t)D * D, "pca covariance"));
    PTS_TRY(sc.get(&part, (size_t)ns * D * D, "pca covariance slices"));
    PTS_TRY(sc.get(&V, (size_t)D * m, "pca V"));
    PTS_TRY(sc.get(&Y, (size_t)D * m, "pca Y"));
    PTS_TRY(sc.get(&Vr, (size_t)D * m, "pca Vr"));
    PTS_TRY(sc.get(&Yr, (size_t)D * m, "pca Yr"));
    PTS_TRY(sc.get(&G, (size_t)m * m, "pca G"));
    PTS_TRY(sc.get(&S, (size_t)m * m, "pca S"));
    PTS_TRY(sc.get(&th, m, "pca theta"));
    PTS_TRY(sc.get(&res, m, "pca residual"));
    PTS_TRY(sc.get(&diag, D, "pca diag"));
    const bool big = m > kMaxM;
    double *jwork = nullptr;
    if (big) PTS_TRY(sc.get(&jwork, (size_t)2 * m * m, "pca jacobi scratch"));

    const size_t jac_smem = big ? 0 : sizeof(double) * 2 * m * m;
    const size_t chol_smem = big ? 0 : sizeof(double) * m * m;
    set_smem_attr(reinterpret_cast<const void *>(k_jacobi_small), (int)(sizeof(double) * 2 * kMaxM * kMaxM));
    set_smem_attr(reinterpret_cast<const void *>(k_chol), (int)(sizeof(double) * kMaxM * kMaxM));

    count_launches(1);
    k_win_mean<<<D, 256, 0, st>>>(exemplar, We, nch, w, ex, N, mu64);
    count_launches(1);
    k_cov<<<dim3(npairs, ns), 256, 0, st>>>(exemplar, We, nch, w, ex, N, mu64, D, T, slice_len, part);
    count_launches(1);
    k_cov_reduce<<<ceil_div((long)D * D, 256), 256, 0, st>>>(part, ns, D, N, C);
    count_launches(1);
    k_diag<<<ceil_div(D, 256), 256, 0, st>>>(C, D, diag);
    std::vector<double> hdiag(D);
    PTS_CUDA_TRY(cudaMemcpyAsync(hdiag.data(), diag, sizeof(double) * D, cudaMemcpyDeviceToHost, st));

    auto orth = [&](double *Vm) {
        for (int rep = 0; rep < 2; ++rep) {
            dgemm<true, false>(m, m, D, Vm, m, Vm, m, G, m, st);
            count_launches(1);
            k_chol<<<1, 512, chol_smem, st>>>(G, m, big ? 1 : 0, status);
            count_launches(1);
            k_trsm_rows<<<ceil_div(D, 128), 128, 0, st>>>(Vm, D, m, G);
        }
    };
    count_launches(1);
    k_init_subspace<<<64, 256, 0, st>>>(V, (long)D * m);
    orth(V);

    std::vector<double> hth(m), hres(dd);
    int it = 0;
    for (it = 1; it <= max_iters; ++it) {
        dgemm<false, false>(D, m, D, C, D, V, m, Y, m, st);  // Y = Sigma V
        // Rayleigh-Ritz (and the convergence test) every kRitzEvery-th step and at the cap: the
        // steps between are plain power steps on the orthonormalised block, which span the same
        // subspace the Ritz vectors would (rotating inside it changes nothing), so only the test
        // is less frequent while the eigen-solve, which dominates a step, runs a quarter as often.
        // The first step always solves it: when the block is the whole space (m = D) that is the
        // exact answer, and no power step on a rank-deficient covariance is needed
        if (it != 1 && it % kRitzEvery != 0 && it != max_iters) {
            std::swap(V, Y);
            orth(V);
            continue;
        }
        dgemm<true, false>(m, m, D, V, m, Y, m, G, m, st);   // H = V^T Y
        count_launches(1);
        k_jacobi_small<<<1, 512, jac_smem, st>>>(G, m, th, S, jwork, status);
        dgemm<false, false>(D, m, m, V, m, S, m, Vr, m, st);  // Ritz vectors
        dgemm<false, false>(D, m, m, Y, m, S, m, Yr, m, st);  // Sigma * Ritz vectors
        count_launches(1);
        k_ritz_residual<<<dd, 256, 0, st>>>(Yr, Vr, th, D, m, dd, res);
        PTS_CUDA_TRY(cudaMemcpyAsync(hth.data(), th, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
        PTS_CUDA_TRY(cudaMemcpyAsync(hres.data(), res, sizeof(double) * dd, cudaMemcpyDeviceToHost, st));
        PTS_CUDA_TRY(cudaStreamSynchronize(st));
        double worst = 0.0;
        for (int j = 0; j < dd; ++j) worst = std::max(worst, hres[j]);
        if (worst <= 1e-12 * std::fabs(hth[0]) || it == max_iters) break;
        std::swap(V, Yr);  // power step on the Ritz vectors
        orth(V);
    }
    double trace = 0.0;
    for (int k = 0; k < D; ++k) trace += hdiag[k];
    int dfin = dd;
    if (d <= 0) {
        double acc = 0.0;
        dfin = dd;
        for (int j = 0; j < dd; ++j) {
            acc += hth[j];
            if (acc >= var_frac * trace) {
                dfin = j + 1;
                break;
            }
        }
    }
    double kept = 0.0;
    for (int j = 0; j < dfin; ++j) kept += hth[j];
    count_launches(1);
    k_export_basis<<<ceil_div((long)std::max(dfin * D, D), 256), 256, 0, st>>>(Vr, D, m, dfin, mu64,
                                                                               basis_out, mean_out);
    if (eig_out)
        PTS_CUDA_TRY(cudaMemcpyAsync(eig_out, th, sizeof(double) * dfin, cudaMemcpyDeviceToDevice, st));
    PTS_CUDA_TRY(cudaStreamSynchronize(st));
    PTS_CUDA_TRY(cudaGetLastError());
    if (d_used) *d_used = dfin;
    if (trace_out) *trace_out = trace;
    if (var_retained) *var_retained = trace > 0 ? kept / trace : 0.0;
    if (eig_top) *eig_top = hth[0];
    if (iters_used) *iters_used = std::min(it, max_iters);
    return PTS_OK;
}

}  // namespace pts
