/*
 * pts_oracle.c -- plain FP64 CPU oracle for perspective texture synthesis by
 * energy optimisation (Bashir & Ghouri, arXiv:2006.11851).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * library never does.  It shares no code, header or table with the CUDA path.
 *
 * Conventions (shared with the CUDA path only through the written contract):
 *   images      H x W x C, row-major, channel fastest ("HWC"), double here;
 *               C = 3 (RGB), or 4 (RGBS: the scale map of section 1 as a
 *               fourth channel beside R, G and B, as section 3 builds its
 *               neighbourhood vectors);
 *   window      the w x w block whose top-left pixel is (y0, x0);
 *   vector      element (dy, dx, c) of a window sits at (dy*w + dx)*C + c;
 *   exemplar    windows at every stride-1 origin fully inside the exemplar,
 *               index n = y*(We - w + 1) + x;
 *   queries     windows of the output at origins on the stride grid
 *               y0 in {0, s, ..., Ho - w}, index q = (y0/s)*((Wo-w)/s+1) + x0/s;
 *   PCA basis   basis[j*D + k] = element k of eigenvector j (j < d), eigen-
 *               vectors ordered by decreasing eigenvalue.
 *
 * Each function cites the passage of the paper it follows.  Loops run in
 * the order the definitions are written; OpenMP only splits independent
 * outer iterations (queries, rows) across threads and never changes the
 * order of any floating-point sum.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EXPORT __attribute__((visibility("default")))

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

OR_EXPORT int or_max_threads(int nthreads) { return set_threads(nthreads); }

/* ---------------------------------------------------------------------------
 * E-step (Energy Optimization, Eq. 4): z_p is the exemplar neighbourhood most
 * similar to x_p under the Euclidean norm.  Brute force over every exemplar
 * window in the full dimension D = C w^2; ties go to the smallest index n
 * (strict '<').  qlist selects the query indices to evaluate (NULL = all Q,
 * then nq must be Q).  Outputs nn[i], d2[i] for i < nq.
 * ------------------------------------------------------------------------ */
OR_EXPORT void or_nn_bruteforce(const double *X, int Ho, int Wo, const double *Z, int He, int We,
                                int w, int C, int stride, const int32_t *qlist, int nq, int32_t *nn,
                                double *d2, int nthreads) {
    set_threads(nthreads);
    const int qx = (Wo - w) / stride + 1;
    const int ex = We - w + 1;
    const long N = (long)(He - w + 1) * ex;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < nq; ++i) {
        const int q = qlist ? qlist[i] : i;
        const int y0 = (q / qx) * stride, x0 = (q % qx) * stride;
        double best = INFINITY;
        long best_n = -1;
        for (long n = 0; n < N; ++n) {
            const int ey = (int)(n / ex), exx = (int)(n % ex);
            double s = 0.0;
            for (int dy = 0; dy < w; ++dy)
                for (int dx = 0; dx < w; ++dx)
                    for (int c = 0; c < C; ++c) {
                        const double a = X[((long)(y0 + dy) * Wo + (x0 + dx)) * C + c];
                        const double b = Z[((long)(ey + dy) * We + (exx + dx)) * C + c];
                        s += (a - b) * (a - b);
                    }
            if (s < best) {
                best = s;
                best_n = n;
            }
        }
        nn[i] = (int32_t)best_n;
        d2[i] = best;
    }
}

/* Full-dimension squared distance between query q of X and exemplar window n
 * (Eq. 4 term).  Used to score candidate lists. */
OR_EXPORT void or_pair_dist2(const double *X, int Ho, int Wo, const double *Z, int He, int We,
                             int w, int C, int stride, const int32_t *q, const int32_t *n, int count,
                             double *d2) {
    (void)Ho;
    (void)He;
    const int qx = (Wo - w) / stride + 1;
    const int ex = We - w + 1;
    for (int i = 0; i < count; ++i) {
        const int y0 = (q[i] / qx) * stride, x0 = (q[i] % qx) * stride;
        const int ey = n[i] / ex, exx = n[i] % ex;
        double s = 0.0;
        for (int dy = 0; dy < w; ++dy)
            for (int dx = 0; dx < w; ++dx)
                for (int c = 0; c < C; ++c) {
                    const double a = X[((long)(y0 + dy) * Wo + (x0 + dx)) * C + c];
                    const double b = Z[((long)(ey + dy) * We + (exx + dx)) * C + c];
                    s += (a - b) * (a - b);
                }
        d2[i] = s;
    }
}

/* ---------------------------------------------------------------------------
 * PCA of the exemplar neighbourhood vectors (Energy Optimization Improvement,
 * section 2.2: dimensions are reduced by PCA before the search).
 *   mu    = (1/N) sum_n v_n
 *   Sigma = (1/N) sum_n (v_n - mu)(v_n - mu)^T
 * ------------------------------------------------------------------------ */
OR_EXPORT void or_window_mean(const double *Z, int He, int We, int w, int C, double *mu) {
    const int D = C * w * w;
    const int ex = We - w + 1;
    const long N = (long)(He - w + 1) * ex;
    for (int k = 0; k < D; ++k) mu[k] = 0.0;
    for (long n = 0; n < N; ++n) {
        const int ey = (int)(n / ex), exx = (int)(n % ex);
        for (int dy = 0; dy < w; ++dy)
            for (int dx = 0; dx < w; ++dx)
                for (int c = 0; c < C; ++c)
                    mu[(dy * w + dx) * C + c] += Z[((long)(ey + dy) * We + (exx + dx)) * C + c];
    }
    for (int k = 0; k < D; ++k) mu[k] /= (double)N;
}

/* Centered window vectors u_n = v_n - mu for n in [n0, n0 + cnt), row-major cnt x D. */
static void centered_windows(const double *Z, int We, int w, int C, const double *mu, long n0, long cnt,
                             double *U) {
    const int D = C * w * w;
    const int ex = We - w + 1;
    for (long i = 0; i < cnt; ++i) {
        const long n = n0 + i;
        const int ey = (int)(n / ex), exx = (int)(n % ex);
        for (int dy = 0; dy < w; ++dy)
            for (int dx = 0; dx < w; ++dx)
                for (int c = 0; c < C; ++c) {
                    const int k = (dy * w + dx) * C + c;
                    U[i * D + k] = Z[((long)(ey + dy) * We + (exx + dx)) * C + c] - mu[k];
                }
    }
}

/* Sigma (D x D, full symmetric) = (1/N) sum_n u_n u_n^T; each entry is the
 * sum over n in increasing order. */
OR_EXPORT void or_window_cov(const double *Z, int He, int We, int w, int C, const double *mu, double *cov,
                             int nthreads) {
    set_threads(nthreads);
    const int D = C * w * w;
    const int ex = We - w + 1;
    const long N = (long)(He - w + 1) * ex;
    const long chunk = 512;
    double *U = (double *)malloc(sizeof(double) * chunk * D);
    memset(cov, 0, sizeof(double) * (size_t)D * D);
    for (long n0 = 0; n0 < N; n0 += chunk) {
        const long cnt = (N - n0 < chunk) ? (N - n0) : chunk;
        centered_windows(Z, We, w, C, mu, n0, cnt, U);
#pragma omp parallel for schedule(dynamic, 8)
        for (int i = 0; i < D; ++i)
            for (long t = 0; t < cnt; ++t) {
                const double ui = U[t * D + i];
                for (int j = i; j < D; ++j) cov[(long)i * D + j] += ui * U[t * D + j];
            }
    }
    free(U);
    for (int i = 0; i < D; ++i)
        for (int j = i; j < D; ++j) {
            cov[(long)i * D + j] /= (double)N;
            cov[(long)j * D + i] = cov[(long)i * D + j];
        }
}

/* Gram matrix G (N x N) = (1/N) U U^T of the centered windows; used when
 * N < D, where Sigma = (1/N) U^T U shares its nonzero eigenvalues with G and
 * its eigenvectors are U^T g / sqrt(N lambda) (singular value decomposition
 * of U). */
static void window_gram(const double *Z, int He, int We, int w, int C, const double *mu, double *G,
                        double *U) {
    const int D = C * w * w;
    const int ex = We - w + 1;
    const long N = (long)(He - w + 1) * ex;
    centered_windows(Z, We, w, C, mu, 0, N, U);
#pragma omp parallel for schedule(dynamic, 8)
    for (long a = 0; a < N; ++a)
        for (long b = a; b < N; ++b) {
            double s = 0.0;
            for (int k = 0; k < D; ++k) s += U[a * D + k] * U[b * D + k];
            G[a * N + b] = s / (double)N;
            G[b * N + a] = s / (double)N;
        }
}

/* ---------------------------------------------------------------------------
 * Symmetric eigen-decomposition by Jacobi's method (Golub & Van Loan,
 * "Matrix Computations", section 8.5: the 2x2 symmetric Schur step and the
 * parallel round-robin ordering).  Each round applies n/2 rotations on
 * disjoint index pairs; such rotations commute, so a round equals applying
 * them one after another.  A rotation is skipped when
 * |a_pq| <= 1e-16 sqrt(|a_pp a_qq|) (relative threshold) or
 * |a_pq| <= 1e-18 ||A||_F (absolute floor, so rounding noise next to a zero
 * eigenvalue cannot keep the sweeps going); sweeps stop when a sweep performs
 * no rotation.  On return evals is sorted descending and
 * column j of V (V[k*n + j]) is the eigenvector of evals[j].  A is destroyed.
 * Returns the number of sweeps, or -1 if 100 sweeps did not converge.
 * ------------------------------------------------------------------------ */
OR_EXPORT int or_jacobi_eigh(double *A, int n, double *evals, double *V, int nthreads) {
    set_threads(nthreads);
    const int m = (n % 2) ? n + 1 : n; /* pad with a dummy index n when odd */
    int *pp = (int *)malloc(sizeof(int) * (m / 2));
    int *qq = (int *)malloc(sizeof(int) * (m / 2));
    double *cc = (double *)malloc(sizeof(double) * (m / 2));
    double *ss = (double *)malloc(sizeof(double) * (m / 2));
    int *active = (int *)malloc(sizeof(int) * (m / 2));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[(long)i * n + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (long i = 0; i < (long)n * n; ++i) fro += A[i] * A[i];
    const double floor_abs = 1e-18 * sqrt(fro);
    int sweeps = 0, converged = 0;
    for (sweeps = 1; sweeps <= 100 && !converged; ++sweeps) {
        long rotations = 0;
        for (int r = 0; r < m - 1; ++r) {
            /* circle method: index m-1 fixed, the others rotate */
            int np = 0;
            for (int k = 0; k < m / 2; ++k) {
                int a, b;
                if (k == 0) {
                    a = m - 1;
                    b = r;
                } else {
                    a = (r + k) % (m - 1);
                    b = (r - k + (m - 1)) % (m - 1);
                }
                if (a >= n || b >= n) continue; /* pairs with the dummy index */
                pp[np] = a < b ? a : b;
                qq[np] = a < b ? b : a;
                ++np;
            }
            int nact = 0;
            for (int k = 0; k < np; ++k) {
                const int p = pp[k], q = qq[k];
                const double apq = A[(long)p * n + q], app = A[(long)p * n + p],
                             aqq = A[(long)q * n + q];
                active[k] = 0;
                if (fabs(apq) <= floor_abs || fabs(apq) <= 1e-16 * sqrt(fabs(app * aqq))) continue;
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                cc[k] = 1.0 / sqrt(1.0 + t * t);
                ss[k] = t * cc[k];
                active[k] = 1;
                ++nact;
            }
            if (!nact) continue;
            rotations += nact;
            /* rows: A <- J^T A */
#pragma omp parallel for schedule(static)
            for (int k = 0; k < np; ++k) {
                if (!active[k]) continue;
                const int p = pp[k], q = qq[k];
                const double c = cc[k], s = ss[k];
                for (int j = 0; j < n; ++j) {
                    const double ap = A[(long)p * n + j], aq = A[(long)q * n + j];
                    A[(long)p * n + j] = c * ap - s * aq;
                    A[(long)q * n + j] = s * ap + c * aq;
                }
            }
            /* columns: A <- A J and V <- V J */
#pragma omp parallel for schedule(static)
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < np; ++k) {
                    if (!active[k]) continue;
                    const int p = pp[k], q = qq[k];
                    const double c = cc[k], s = ss[k];
                    const double ap = A[(long)i * n + p], aq = A[(long)i * n + q];
                    A[(long)i * n + p] = c * ap - s * aq;
                    A[(long)i * n + q] = s * ap + c * aq;
                    const double vp = V[(long)i * n + p], vq = V[(long)i * n + q];
                    V[(long)i * n + p] = c * vp - s * vq;
                    V[(long)i * n + q] = s * vp + c * vq;
                }
            for (int k = 0; k < np; ++k)
                if (active[k]) {
                    A[(long)pp[k] * n + qq[k]] = 0.0;
                    A[(long)qq[k] * n + pp[k]] = 0.0;
                }
        }
        if (rotations == 0) converged = 1;
    }
    /* sort descending (selection sort on indices; n is small) */
    int *ord = (int *)malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    for (int i = 0; i < n; ++i) {
        int best = i;
        for (int j = i + 1; j < n; ++j)
            if (A[(long)ord[j] * n + ord[j]] > A[(long)ord[best] * n + ord[best]]) best = j;
        const int tmp = ord[i];
        ord[i] = ord[best];
        ord[best] = tmp;
    }
    double *Vs = (double *)malloc(sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; ++j) {
        evals[j] = A[(long)ord[j] * n + ord[j]];
        for (int i = 0; i < n; ++i) Vs[(long)i * n + j] = V[(long)i * n + ord[j]];
    }
    memcpy(V, Vs, sizeof(double) * (size_t)n * n);
    free(Vs);
    free(ord);
    free(pp);
    free(qq);
    free(cc);
    free(ss);
    free(active);
    return converged ? sweeps - 1 : -1;
}

/* PCA fit (section 2.2): mean mu (D), top-d eigenvectors basis[j*D + k] and
 * all eigenvalues evals_all (min(N, D) entries, descending) of Sigma.
 * Uses the Gram matrix when N < D (see window_gram).  Returns Jacobi sweeps. */
OR_EXPORT int or_pca_fit(const double *Z, int He, int We, int w, int C, int d, double *mu, double *basis,
                         double *evals_all, int nthreads) {
    set_threads(nthreads);
    const int D = C * w * w;
    const long N = (long)(He - w + 1) * (We - w + 1);
    or_window_mean(Z, He, We, w, C, mu);
    int sweeps;
    if (N >= D) {
        double *cov = (double *)malloc(sizeof(double) * (size_t)D * D);
        double *V = (double *)malloc(sizeof(double) * (size_t)D * D);
        or_window_cov(Z, He, We, w, C, mu, cov, nthreads);
        sweeps = or_jacobi_eigh(cov, D, evals_all, V, nthreads);
        for (int j = 0; j < d; ++j)
            for (int k = 0; k < D; ++k) basis[(long)j * D + k] = V[(long)k * D + j];
        free(cov);
        free(V);
    } else {
        double *U = (double *)malloc(sizeof(double) * (size_t)N * D);
        double *G = (double *)malloc(sizeof(double) * (size_t)N * N);
        double *V = (double *)malloc(sizeof(double) * (size_t)N * N);
        window_gram(Z, He, We, w, C, mu, G, U);
        sweeps = or_jacobi_eigh(G, (int)N, evals_all, V, nthreads);
        for (int j = 0; j < d; ++j) {
            /* eigenvector of Sigma: U^T g_j, normalised */
            double nrm = 0.0;
            for (int k = 0; k < D; ++k) {
                double s = 0.0;
                for (long a = 0; a < N; ++a) s += U[a * D + k] * V[a * N + j];
                basis[(long)j * D + k] = s;
                nrm += s * s;
            }
            nrm = sqrt(nrm);
            for (int k = 0; k < D; ++k) basis[(long)j * D + k] /= nrm;
        }
        free(U);
        free(G);
        free(V);
    }
    return sweeps;
}

/* Projection onto the PCA basis (section 2.2): for each listed window,
 * y = B^T (v - mu) (d values), unorm2 = ||v - mu||^2 and the residual norm
 * resid = ||(v - mu) - B y|| of the part PCA discards.  Windows sit on the
 * stride grid of the image (stride 1 for the exemplar, the patch stride for
 * queries). */
OR_EXPORT void or_project(const double *img, int H, int W, int w, int C, int stride, const double *mu,
                          const double *basis, int d, const int32_t *list, int count, double *y,
                          double *unorm2, double *resid) {
    (void)H;
    const int D = C * w * w;
    const int qx = (W - w) / stride + 1;
#pragma omp parallel
    {
        double *u = (double *)malloc(sizeof(double) * D);
#pragma omp for schedule(static)
        for (int i = 0; i < count; ++i) {
            const int q = list ? list[i] : i;
            const int y0 = (q / qx) * stride, x0 = (q % qx) * stride;
            double un = 0.0;
            for (int dy = 0; dy < w; ++dy)
                for (int dx = 0; dx < w; ++dx)
                    for (int c = 0; c < C; ++c) {
                        const int k = (dy * w + dx) * C + c;
                        u[k] = img[((long)(y0 + dy) * W + (x0 + dx)) * C + c] - mu[k];
                        un += u[k] * u[k];
                    }
            for (int j = 0; j < d; ++j) {
                double s = 0.0;
                for (int k = 0; k < D; ++k) s += basis[(long)j * D + k] * u[k];
                y[(long)i * d + j] = s;
            }
            double r2 = 0.0;
            for (int k = 0; k < D; ++k) {
                double rk = u[k];
                for (int j = 0; j < d; ++j) rk -= basis[(long)j * D + k] * y[(long)i * d + j];
                r2 += rk * rk;
            }
            unorm2[i] = un;
            resid[i] = sqrt(r2);
        }
        free(u);
    }
}

/* ---------------------------------------------------------------------------
 * Robust energy and IRLS weights (Eqs. 5-8).  With d_p = sqrt(d2_p):
 *   W_p = max(d_p, delta)^(r - 2)        (Eq. 7; delta > 0 keeps W finite
 *                                          when d_p = 0, which Eq. 7 leaves open)
 *   E_r = sum_p d_p^r                     (Eq. 5; Eq. 4 when r = 2)
 *   E_delta = sum_p rho(d_p^2), rho(t) = t^(r/2) for t >= delta^2 and
 *             delta^r + (r/2) delta^(r-2) (t - delta^2) below: the concave
 *             function whose majorize-minimize step is exactly the weighted
 *             least squares of Eq. 8 with the weights above.
 * For r = 2 all weights are 1 and E_r = E_delta = sum d2.
 * ------------------------------------------------------------------------ */
OR_EXPORT void or_irls(const double *d2, int Q, double r, double delta, double *W, double *E_r,
                       double *E_delta) {
    double er = 0.0, ed = 0.0;
    for (int p = 0; p < Q; ++p) {
        const double t = d2[p] > 0.0 ? d2[p] : 0.0;
        const double dp = sqrt(t);
        if (r == 2.0) {
            if (W) W[p] = 1.0;
            er += t;
            ed += t;
            continue;
        }
        if (W) W[p] = pow(dp > delta ? dp : delta, r - 2.0);
        er += pow(dp, r);
        if (dp >= delta)
            ed += pow(dp, r);
        else
            ed += pow(delta, r) + 0.5 * r * pow(delta, r - 2.0) * (t - delta * delta);
    }
    *E_r = er;
    *E_delta = ed;
}

/* ---------------------------------------------------------------------------
 * M-step (optimization phase, Eq. 8 minimised over x): every output pixel i
 * becomes the weighted mean of the co-located pixels of the matched windows
 * that cover it,
 *   x_i = sum_{p covers i} W_p z_{nn(p)}[i - p] / sum_{p covers i} W_p.
 * With the patch stride s, all pixels of an s x s patch share one covering
 * set (section 2.2, 2x2 patch processing).  Sums run over p in increasing
 * query order.  Wt == NULL means W_p = 1.  Pixels covered by no window keep
 * their value from X (never happens when (Ho-w) and (Wo-w) are multiples of s).
 * ------------------------------------------------------------------------ */
OR_EXPORT void or_m_step(const int32_t *nn, const double *Wt, const double *Z, int He, int We,
                         int w, int C, int Ho, int Wo, int stride, double *X) {
    (void)He;
    const int qy = (Ho - w) / stride + 1, qx = (Wo - w) / stride + 1;
    const int ex = We - w + 1;
    double *num = (double *)calloc((size_t)Ho * Wo * C, sizeof(double));
    double *den = (double *)calloc((size_t)Ho * Wo, sizeof(double));
    for (int p = 0; p < qy * qx; ++p) {
        const int y0 = (p / qx) * stride, x0 = (p % qx) * stride;
        const int ey = nn[p] / ex, exx = nn[p] % ex;
        const double wp = Wt ? Wt[p] : 1.0;
        for (int dy = 0; dy < w; ++dy)
            for (int dx = 0; dx < w; ++dx) {
                const long o = (long)(y0 + dy) * Wo + (x0 + dx);
                den[o] += wp;
                for (int c = 0; c < C; ++c)
                    num[o * C + c] += wp * Z[((long)(ey + dy) * We + (exx + dx)) * C + c];
            }
    }
    for (long o = 0; o < (long)Ho * Wo; ++o)
        if (den[o] > 0.0)
            for (int c = 0; c < C; ++c) X[o * C + c] = num[o * C + c] / den[o];
    free(num);
    free(den);
}

/* ---------------------------------------------------------------------------
 * Coarse-to-fine synthesis (Energy Optimization Method, section 2.1: a coarse
 * result is up-sampled by interpolation to initialise the next level).
 * The paper names no filters; these are the readings used throughout:
 *   down-sampling: separable 5-tap binomial [1 4 6 4 1]/16, mirror border
 *                  without edge repeat (index -1 -> 1, H -> H-2), keep even
 *                  samples: out(y, x) = sum_ab k_a k_b img(2y+a-2, 2x+b-2);
 *   up-sampling:   bilinear x2 with half-pixel centres, source coordinate
 *                  (Y + 0.5)/2 - 0.5 clamped to [0, H-1].
 * ------------------------------------------------------------------------ */
static int mirror(int i, int n) {
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * (n - 1) - i;
    }
    return i;
}

OR_EXPORT void or_downsample2(const double *img, int H, int W, int C, double *out) {
    static const double k[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    for (int y = 0; y < Ho; ++y)
        for (int x = 0; x < Wo; ++x)
            for (int c = 0; c < C; ++c) {
                double s = 0.0;
                for (int a = 0; a < 5; ++a)
                    for (int b = 0; b < 5; ++b) {
                        const int yy = mirror(2 * y + a - 2, H), xx = mirror(2 * x + b - 2, W);
                        s += k[a] * k[b] * img[((long)yy * W + xx) * C + c];
                    }
                out[((long)y * Wo + x) * C + c] = s;
            }
}

OR_EXPORT void or_upsample2(const double *img, int H, int W, int C, double *out) {
    const int Ho = 2 * H, Wo = 2 * W;
    for (int Y = 0; Y < Ho; ++Y)
        for (int Xc = 0; Xc < Wo; ++Xc) {
            double sy = (Y + 0.5) / 2.0 - 0.5, sx = (Xc + 0.5) / 2.0 - 0.5;
            if (sy < 0) sy = 0;
            if (sx < 0) sx = 0;
            if (sy > H - 1) sy = H - 1;
            if (sx > W - 1) sx = W - 1;
            const int y0 = (int)floor(sy), x0 = (int)floor(sx);
            const int y1 = y0 + 1 < H ? y0 + 1 : H - 1, x1 = x0 + 1 < W ? x0 + 1 : W - 1;
            const double fy = sy - y0, fx = sx - x0;
            for (int c = 0; c < C; ++c) {
                const double v00 = img[((long)y0 * W + x0) * C + c];
                const double v01 = img[((long)y0 * W + x1) * C + c];
                const double v10 = img[((long)y1 * W + x0) * C + c];
                const double v11 = img[((long)y1 * W + x1) * C + c];
                out[((long)Y * Wo + Xc) * C + c] =
                    (1 - fy) * ((1 - fx) * v00 + fx * v01) + fy * ((1 - fx) * v10 + fx * v11);
            }
        }
}
