/*
 * pts_oracle_learn.c -- FP64 CPU oracle for the learned cluster proposal that
 * replaces the paper's k-means search tree (section 2.2 builds a k-means tree
 * over PCA-reduced neighbourhood vectors to accelerate the search; here a
 * flat k-means partition plus a small network that ranks its clusters).
 *
 * TEST INFRASTRUCTURE ONLY (see pts_oracle.c).  Plain loops in the order the
 * definitions are written.
 *
 *   k-means++ seeding (Arthur & Vassilvitskii, 2007) with caller-supplied
 *   uniforms; Lloyd iterations (assignment to the nearest centroid, smallest
 *   id on ties; update to the mean of the members; an empty cluster takes the
 *   point of largest assignment cost, smallest index on ties).
 *
 *   MLP  h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2), z = W3 h2 + b3, with
 *   gelu(a) = a * Phi(a) (exact form, Phi the standard normal CDF via erf),
 *   loss = mean over the batch of -log softmax(z)[label].
 *   Weights are row-major [out][in].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EXPORT __attribute__((visibility("default")))

/* squared distance between rows */
static double d2row(const double *a, const double *b, int d) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += (a[k] - b[k]) * (a[k] - b[k]);
    return s;
}

/* k-means++: idx_out[0] = floor(u[0] n); center i is the first point j whose
 * running sum of D^2 (index order) reaches u[i] * total (D^2 = squared
 * distance to the nearest chosen center); if total == 0, floor(u[i] n). */
OR_EXPORT void or_kmeans_pp(const double *Y, int n, int d, int k, const double *u, double *C,
                            int32_t *idx_out) {
    double *D2 = (double *)malloc(sizeof(double) * n);
    int first = (int)(u[0] * n);
    if (first >= n) first = n - 1;
    idx_out[0] = first;
    memcpy(C, Y + (long)first * d, sizeof(double) * d);
    for (int j = 0; j < n; ++j) D2[j] = d2row(Y + (long)j * d, C, d);
    for (int i = 1; i < k; ++i) {
        double total = 0.0;
        for (int j = 0; j < n; ++j) total += D2[j];
        int pick = n - 1;
        if (total > 0.0) {
            const double target = u[i] * total;
            double run = 0.0;
            for (int j = 0; j < n; ++j) {
                run += D2[j];
                if (run >= target && D2[j] > 0.0) {
                    pick = j;
                    break;
                }
            }
        } else {
            pick = (int)(u[i] * n);
            if (pick >= n) pick = n - 1;
        }
        idx_out[i] = pick;
        memcpy(C + (long)i * d, Y + (long)pick * d, sizeof(double) * d);
        for (int j = 0; j < n; ++j) {
            const double t = d2row(Y + (long)j * d, C + (long)i * d, d);
            if (t < D2[j]) D2[j] = t;
        }
    }
    free(D2);
}

/* nearest centroid (smallest id on ties) and its squared distance */
OR_EXPORT void or_kmeans_assign(const double *Y, int n, int d, const double *C, int k,
                                int32_t *assign, double *cost) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j) {
        double best = INFINITY;
        int bi = 0;
        for (int c = 0; c < k; ++c) {
            const double t = d2row(Y + (long)j * d, C + (long)c * d, d);
            if (t < best) {
                best = t;
                bi = c;
            }
        }
        assign[j] = bi;
        if (cost) cost[j] = best;
    }
}

/* centroid c = mean of its members (sums in point order); an empty cluster
 * takes the point of largest cost (smallest index on ties), which is then
 * excluded from further re-seeding in this update.  counts_out may be NULL. */
OR_EXPORT void or_kmeans_update(const double *Y, int n, int d, const int32_t *assign, int k,
                                double *C, int32_t *counts_out, const double *cost) {
    double *S = (double *)calloc((size_t)k * d, sizeof(double));
    int32_t *cnt = (int32_t *)calloc(k, sizeof(int32_t));
    for (int j = 0; j < n; ++j) {
        const int c = assign[j];
        cnt[c] += 1;
        for (int t = 0; t < d; ++t) S[(long)c * d + t] += Y[(long)j * d + t];
    }
    unsigned char *used = (unsigned char *)calloc(n, 1);
    for (int c = 0; c < k; ++c) {
        if (cnt[c] > 0) {
            for (int t = 0; t < d; ++t) C[(long)c * d + t] = S[(long)c * d + t] / cnt[c];
        } else if (cost) {
            int far = -1;
            for (int j = 0; j < n; ++j)
                if (!used[j] && (far < 0 || cost[j] > cost[far])) far = j;
            if (far >= 0) {
                used[far] = 1;
                memcpy(C + (long)c * d, Y + (long)far * d, sizeof(double) * d);
            }
        }
    }
    if (counts_out) memcpy(counts_out, cnt, sizeof(int32_t) * k);
    free(S);
    free(cnt);
    free(used);
}

static double gelu(double a) { return 0.5 * a * (1.0 + erf(a / sqrt(2.0))); }
static double gelu_grad(double a) {
    const double Phi = 0.5 * (1.0 + erf(a / sqrt(2.0)));
    const double phi = exp(-0.5 * a * a) / sqrt(2.0 * 3.14159265358979323846);
    return Phi + a * phi;
}

/* y[B][o] = x[B][i] W^T + b */
static void linear(const double *x, int B, int in, int out, const double *W, const double *b,
                   double *y) {
#pragma omp parallel for schedule(static)
    for (int r = 0; r < B; ++r)
        for (int o = 0; o < out; ++o) {
            double s = b ? b[o] : 0.0;
            for (int i = 0; i < in; ++i) s += x[(long)r * in + i] * W[(long)o * in + i];
            y[(long)r * out + o] = s;
        }
}

/* forward: keeps pre-activations A1, A2, activations H1, H2 and logits Z */
OR_EXPORT void or_mlp_forward(const double *X, int B, int in, int h1, int h2, int out,
                              const double *W1, const double *b1, const double *W2,
                              const double *b2, const double *W3, const double *b3, double *A1,
                              double *H1, double *A2, double *H2, double *Z) {
    linear(X, B, in, h1, W1, b1, A1);
    for (long t = 0; t < (long)B * h1; ++t) H1[t] = gelu(A1[t]);
    linear(H1, B, h1, h2, W2, b2, A2);
    for (long t = 0; t < (long)B * h2; ++t) H2[t] = gelu(A2[t]);
    linear(H2, B, h2, out, W3, b3, Z);
}

/* mean cross-entropy of logits Z [B][C] against labels; P receives softmax(Z) */
OR_EXPORT double or_ce_loss(const double *Z, int B, int C, const int32_t *labels, double *P) {
    double loss = 0.0;
    for (int r = 0; r < B; ++r) {
        double m = -INFINITY;
        for (int c = 0; c < C; ++c) m = Z[(long)r * C + c] > m ? Z[(long)r * C + c] : m;
        double s = 0.0;
        for (int c = 0; c < C; ++c) s += exp(Z[(long)r * C + c] - m);
        for (int c = 0; c < C; ++c) P[(long)r * C + c] = exp(Z[(long)r * C + c] - m) / s;
        loss += -(Z[(long)r * C + labels[r]] - m - log(s));
    }
    return loss / B;
}

/* backward of the mean cross-entropy through the MLP (inputs from forward) */
OR_EXPORT void or_mlp_backward(const double *X, int B, int in, int h1, int h2, int out,
                               const double *W1, const double *b1, const double *W2,
                               const double *b2, const double *W3, const double *b3,
                               const double *A1, const double *H1, const double *A2,
                               const double *H2, const double *P, const int32_t *labels,
                               double *dW1, double *db1, double *dW2, double *db2, double *dW3,
                               double *db3) {
    (void)b1;
    (void)b2;
    (void)b3;
    double *dZ = (double *)malloc(sizeof(double) * (size_t)B * out);
    double *dA2 = (double *)malloc(sizeof(double) * (size_t)B * h2);
    double *dA1 = (double *)malloc(sizeof(double) * (size_t)B * h1);
    for (int r = 0; r < B; ++r)
        for (int c = 0; c < out; ++c)
            dZ[(long)r * out + c] = (P[(long)r * out + c] - (c == labels[r] ? 1.0 : 0.0)) / B;
    /* layer 3 */
    for (int o = 0; o < out; ++o) {
        double sb = 0.0;
        for (int r = 0; r < B; ++r) sb += dZ[(long)r * out + o];
        db3[o] = sb;
        for (int i = 0; i < h2; ++i) {
            double s = 0.0;
            for (int r = 0; r < B; ++r) s += dZ[(long)r * out + o] * H2[(long)r * h2 + i];
            dW3[(long)o * h2 + i] = s;
        }
    }
    for (int r = 0; r < B; ++r)
        for (int i = 0; i < h2; ++i) {
            double s = 0.0;
            for (int o = 0; o < out; ++o) s += dZ[(long)r * out + o] * W3[(long)o * h2 + i];
            dA2[(long)r * h2 + i] = s * gelu_grad(A2[(long)r * h2 + i]);
        }
    /* layer 2 */
    for (int o = 0; o < h2; ++o) {
        double sb = 0.0;
        for (int r = 0; r < B; ++r) sb += dA2[(long)r * h2 + o];
        db2[o] = sb;
        for (int i = 0; i < h1; ++i) {
            double s = 0.0;
            for (int r = 0; r < B; ++r) s += dA2[(long)r * h2 + o] * H1[(long)r * h1 + i];
            dW2[(long)o * h1 + i] = s;
        }
    }
    for (int r = 0; r < B; ++r)
        for (int i = 0; i < h1; ++i) {
            double s = 0.0;
            for (int o = 0; o < h2; ++o) s += dA2[(long)r * h2 + o] * W2[(long)o * h1 + i];
            dA1[(long)r * h1 + i] = s * gelu_grad(A1[(long)r * h1 + i]);
        }
    /* layer 1 */
    for (int o = 0; o < h1; ++o) {
        double sb = 0.0;
        for (int r = 0; r < B; ++r) sb += dA1[(long)r * h1 + o];
        db1[o] = sb;
        for (int i = 0; i < in; ++i) {
            double s = 0.0;
            for (int r = 0; r < B; ++r) s += dA1[(long)r * h1 + o] * X[(long)r * in + i];
            dW1[(long)o * in + i] = s;
        }
    }
    free(dZ);
    free(dA2);
    free(dA1);
}
