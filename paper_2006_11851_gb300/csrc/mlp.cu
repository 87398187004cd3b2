// mlp.cu -- the cluster-proposal network: training (forward, softmax cross-entropy, backward,
// AdamW) and inference, on the BF16 tensor-core GEMM of gemm_tc.cu with FP32 master weights.
//
//   h1 = gelu(W1 x + b1)   (64 -> 256)
//   h2 = gelu(W2 h1 + b2)  (256 -> 256)
//   z  = W3 h2 + b3        (256 -> C, C = number of clusters)
//   loss = mean over the batch of -log softmax(z)[label]
// gelu(a) = a Phi(a) with Phi from erff.  Weights row-major [out][in]; every GEMM is written as
// C = A B^T with K contiguous in both operands, so the backward pass uses transposed BF16
// copies (W^T for dX = dY W, activations^T for dW = dY^T X).
#include <math.h>

#include <algorithm>
#include <vector>

#include "pts_internal.cuh"

namespace pts {

void launch_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                      const float *bias, int gelu, float *Cf, __nv_bfloat16 *Cb, float *Cpre, int ldc, int *status,
                      cudaStream_t st);
void launch_transpose_bf16(const __nv_bfloat16 *in, int rows, int cols, __nv_bfloat16 *out, cudaStream_t st);
void launch_f32_to_bf16(const float *in, long n, __nv_bfloat16 *out, cudaStream_t st);

namespace {

__device__ __forceinline__ float gelu_grad_f(float a) {
    const float Phi = 0.5f * (1.0f + erff(a * 0.70710678118654752f));
    const float phi = 0.39894228040143268f * expf(-0.5f * a * a);
    return Phi + a * phi;
}

// softmax cross-entropy per row; dZ = (softmax - onehot) / B in BF16, loss[row]
__global__ void k_softmax_ce(const float *__restrict__ Z, int B, int C, const int *__restrict__ labels,
                             __nv_bfloat16 *__restrict__ dZ, float *__restrict__ loss) {
    const int r = blockIdx.x;
    if (r >= B) return;
    __shared__ float red[256];
    const float *z = Z + (size_t)r * C;
    float m = -INFINITY;
    for (int c = threadIdx.x; c < C; c += blockDim.x) m = fmaxf(m, z[c]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    m = red[0];
    __syncthreads();
    float s = 0.0f;
    for (int c = threadIdx.x; c < C; c += blockDim.x) s += expf(z[c] - m);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    s = red[0];
    const int y = labels[r];
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const float p = expf(z[c] - m) / s;
        dZ[(size_t)r * C + c] = __float2bfloat16_rn((p - (c == y ? 1.0f : 0.0f)) / (float)B);
    }
    if (threadIdx.x == 0) loss[r] = -(z[y] - m - logf(s));
}

// dA = dH * gelu'(A), stored BF16
__global__ void k_gelu_back(const float *__restrict__ dH, const float *__restrict__ A, long n,
                            __nv_bfloat16 *__restrict__ dA) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dA[i] = __float2bfloat16_rn(dH[i] * gelu_grad_f(A[i]));
}

// db[c] = sum_r dY[r][c] (rows in order, one thread per column)
__global__ void k_colsum(const __nv_bfloat16 *__restrict__ dY, int rows, int cols, float *__restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += __bfloat162float(dY[(size_t)r * cols + c]);
    db[c] = s;
}

__global__ void k_adamw(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                        float *__restrict__ v, long n, float lr, float b1, float b2, float eps, float wd,
                        float bc1, float bc2, int decay) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        float pi = p[i];
        if (decay) pi -= lr * wd * pi;
        pi -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        p[i] = pi;
    }
}

// X rows of a batch (zero-padded to 64 inputs) gathered through perm, in BF16; labels too
__global__ void k_gather_batch(const float *__restrict__ Y, int d, int ldy, const int *__restrict__ perm, int off,
                               int B, const int *__restrict__ lab_all, __nv_bfloat16 *__restrict__ Xb,
                               int *__restrict__ lab) {
    const long n = (long)B * 64;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / 64), k = (int)(i % 64);
        const int src = perm ? perm[off + r] : off + r;
        Xb[i] = __float2bfloat16_rn(k < d ? Y[(size_t)src * ldy + k] : 0.0f);
        if (k == 0 && lab) lab[r] = lab_all[src];
    }
}

}  // namespace

// parameter packing (floats): W1 [H x 64], b1 [H], W2 [H x H], b2 [H], W3 [C x H], b3 [C]
long mlp_param_count(int C) { return (long)kMlpH * 64 + kMlpH + (long)kMlpH * kMlpH + kMlpH + (long)C * kMlpH + C; }

struct MlpView {
    float *W1, *b1, *W2, *b2, *W3, *b3;
};
static MlpView view(float *p, int C) {
    MlpView v;
    v.W1 = p;
    v.b1 = v.W1 + kMlpH * 64;
    v.W2 = v.b1 + kMlpH;
    v.b2 = v.W2 + kMlpH * kMlpH;
    v.W3 = v.b2 + kMlpH;
    v.b3 = v.W3 + (long)C * kMlpH;
    return v;
}

pts_status MlpState::ensure(int C_, int Bmax, cudaStream_t st) {
    (void)st;
    if (C_ != C) bmax = 0;  // activation buffers depend on C
    C = C_;
    const long np = mlp_param_count(C);
    PTS_TRY(params.ensure(np, "mlp params"));
    PTS_TRY(grads.ensure(np, "mlp grads"));
    PTS_TRY(adam_m.ensure(np, "adam m"));
    PTS_TRY(adam_v.ensure(np, "adam v"));
    PTS_TRY(wb.ensure(np, "bf16 weights"));
    PTS_TRY(wt.ensure(np, "bf16 transposed weights"));
    if (Bmax > bmax) {
        bmax = Bmax;
        PTS_TRY(xb.ensure((size_t)Bmax * 64, "mlp x"));
        PTS_TRY(xt.ensure((size_t)Bmax * 64, "mlp x^T"));
        PTS_TRY(a1.ensure((size_t)Bmax * kMlpH, "mlp a1"));
        PTS_TRY(h1b.ensure((size_t)Bmax * kMlpH, "mlp h1"));
        PTS_TRY(h1t.ensure((size_t)Bmax * kMlpH, "mlp h1^T"));
        PTS_TRY(a2.ensure((size_t)Bmax * kMlpH, "mlp a2"));
        PTS_TRY(h2b.ensure((size_t)Bmax * kMlpH, "mlp h2"));
        PTS_TRY(h2t.ensure((size_t)Bmax * kMlpH, "mlp h2^T"));
        PTS_TRY(z.ensure((size_t)Bmax * C, "mlp logits"));
        PTS_TRY(dzb.ensure((size_t)Bmax * C, "mlp dz"));
        PTS_TRY(dzt.ensure((size_t)Bmax * C, "mlp dz^T"));
        PTS_TRY(dh.ensure((size_t)Bmax * kMlpH, "mlp dh"));
        PTS_TRY(dab.ensure((size_t)Bmax * kMlpH, "mlp da"));
        PTS_TRY(dat.ensure((size_t)Bmax * kMlpH, "mlp da^T"));
        PTS_TRY(labels.ensure(Bmax, "mlp labels"));
        PTS_TRY(loss.ensure(Bmax, "mlp loss"));
    }
    return PTS_OK;
}

// BF16 weight copies (row-major) and their transposes, from the FP32 master weights
void mlp_refresh_bf16(MlpState &s, cudaStream_t st) {
    const int C = s.C;
    launch_f32_to_bf16(s.params.ptr, mlp_param_count(C), s.wb.ptr, st);
    MlpView p = view(s.params.ptr, C);
    __nv_bfloat16 *base = s.wb.ptr, *tb = s.wt.ptr;
    auto off = [&](float *q) { return (long)(q - s.params.ptr); };
    launch_transpose_bf16(base + off(p.W1), kMlpH, 64, tb + off(p.W1), st);
    launch_transpose_bf16(base + off(p.W2), kMlpH, kMlpH, tb + off(p.W2), st);
    launch_transpose_bf16(base + off(p.W3), C, kMlpH, tb + off(p.W3), st);
}

// forward on s.xb (B x 64 BF16); logits in s.z; keeps pre-activations when train != 0
void mlp_forward(MlpState &s, int B, int train, int *status, cudaStream_t st) {
    const int C = s.C;
    MlpView p = view(s.params.ptr, C);
    auto wb = [&](float *q) { return s.wb.ptr + (q - s.params.ptr); };
    launch_gemm_bf16(B, kMlpH, 64, s.xb.ptr, 64, wb(p.W1), 64, p.b1, 1, nullptr, s.h1b.ptr, train ? s.a1.ptr : nullptr,
                     kMlpH, status, st);
    launch_gemm_bf16(B, kMlpH, kMlpH, s.h1b.ptr, kMlpH, wb(p.W2), kMlpH, p.b2, 1, nullptr, s.h2b.ptr,
                     train ? s.a2.ptr : nullptr, kMlpH, status, st);
    launch_gemm_bf16(B, C, kMlpH, s.h2b.ptr, kMlpH, wb(p.W3), kMlpH, p.b3, 0, s.z.ptr, nullptr, nullptr, C, status,
                     st);
}

// cross-entropy and backward: gradients into s.grads (same packing as params)
void mlp_backward(MlpState &s, int B, const int *labels, int *status, cudaStream_t st) {
    const int C = s.C;
    MlpView p = view(s.params.ptr, C);
    MlpView g = view(s.grads.ptr, C);
    auto wt = [&](float *q) { return s.wt.ptr + (q - s.params.ptr); };
    count_launches(1);
    k_softmax_ce<<<B, 256, 0, st>>>(s.z.ptr, B, C, labels, s.dzb.ptr, s.loss.ptr);
    // layer 3: dW3 = dZ^T H2, db3 = colsum dZ, dH2 = dZ W3
    launch_transpose_bf16(s.dzb.ptr, B, C, s.dzt.ptr, st);
    launch_transpose_bf16(s.h2b.ptr, B, kMlpH, s.h2t.ptr, st);
    launch_gemm_bf16(C, kMlpH, B, s.dzt.ptr, B, s.h2t.ptr, B, nullptr, 0, g.W3, nullptr, nullptr, kMlpH, status, st);
    count_launches(1);
    k_colsum<<<ceil_div(C, 256), 256, 0, st>>>(s.dzb.ptr, B, C, g.b3);
    launch_gemm_bf16(B, kMlpH, C, s.dzb.ptr, C, wt(p.W3), C, nullptr, 0, s.dh.ptr, nullptr, nullptr, kMlpH, status, st);
    count_launches(1);
    k_gelu_back<<<152 * 4, 256, 0, st>>>(s.dh.ptr, s.a2.ptr, (long)B * kMlpH, s.dab.ptr);
    // layer 2
    launch_transpose_bf16(s.dab.ptr, B, kMlpH, s.dat.ptr, st);
    launch_transpose_bf16(s.h1b.ptr, B, kMlpH, s.h1t.ptr, st);
    launch_gemm_bf16(kMlpH, kMlpH, B, s.dat.ptr, B, s.h1t.ptr, B, nullptr, 0, g.W2, nullptr, nullptr, kMlpH, status,
                     st);
    count_launches(1);
    k_colsum<<<ceil_div(kMlpH, 256), 256, 0, st>>>(s.dab.ptr, B, kMlpH, g.b2);
    launch_gemm_bf16(B, kMlpH, kMlpH, s.dab.ptr, kMlpH, wt(p.W2), kMlpH, nullptr, 0, s.dh.ptr, nullptr, nullptr, kMlpH,
                     status, st);
    count_launches(1);
    k_gelu_back<<<152 * 4, 256, 0, st>>>(s.dh.ptr, s.a1.ptr, (long)B * kMlpH, s.dab.ptr);
    // layer 1
    launch_transpose_bf16(s.dab.ptr, B, kMlpH, s.dat.ptr, st);
    launch_transpose_bf16(s.xb.ptr, B, 64, s.xt.ptr, st);
    launch_gemm_bf16(kMlpH, 64, B, s.dat.ptr, B, s.xt.ptr, B, nullptr, 0, g.W1, nullptr, nullptr, 64, status, st);
    count_launches(1);
    k_colsum<<<ceil_div(kMlpH, 256), 256, 0, st>>>(s.dab.ptr, B, kMlpH, g.b1);
}

void mlp_adamw(MlpState &s, float lr, float wd, int step, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
    const int C = s.C;
    MlpView p = view(s.params.ptr, C);
    // decay weights, not biases
    struct Seg {
        float *p;
        long n;
        int decay;
    } segs[6] = {{p.W1, (long)kMlpH * 64, 1}, {p.b1, kMlpH, 0}, {p.W2, (long)kMlpH * kMlpH, 1},
                 {p.b2, kMlpH, 0},         {p.W3, (long)C * kMlpH, 1}, {p.b3, C, 0}};
    for (auto &g : segs) {
        const long o = g.p - s.params.ptr;
        count_launches(1);
        k_adamw<<<152, 256, 0, st>>>(g.p, s.grads.ptr + o, s.adam_m.ptr + o, s.adam_v.ptr + o, g.n, lr, b1, b2, 1e-8f,
                                     wd, bc1, bc2, g.decay);
    }
}

void mlp_gather(MlpState &s, const float *Y, int d, int ldy, const int *perm, int off, int B, const int *lab_all,
                cudaStream_t st) {
    count_launches(1);
    k_gather_batch<<<152 * 2, 256, 0, st>>>(Y, d, ldy, perm, off, B, lab_all, s.xb.ptr, lab_all ? s.labels.ptr : nullptr);
}

}  // namespace pts
