// lb_mlp.cu -- the learned warm start: a three-layer perceptron (n_in -> H -> H -> n_out, tanh on the
// hidden layers) trained and evaluated by this library's own kernels.  It maps channel parameters
// (width, body force, nlM parameters) to resampled steady profiles, which then initialise the
// lattice-Boltzmann run (lb_set_fields); the LB scheme stays the judge of the result.
//
// Numerics: the weights used by the forward and backward products are BF16 copies of FP32 master
// weights; every product accumulates in FP32; activations and gradients are FP32; Adam updates the
// FP32 masters and refreshes the BF16 copies.
//
// Layout: W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], W3 [n_out][H], b3 [n_out], flattened in this
// order (lb_mlp_get_params / set_params / gradients use the same order).  Activations are row-major
// [batch][features].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include "lbnlm.h"

namespace lbk {
void set_last_error(const char* msg);
}

namespace {

lb_status mfail(lb_status s, const char* what) {
    lbk::set_last_error(what);
    return s;
}
#define MLP_CK(call)                                                         \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) {                                             \
            char m_[256];                                                    \
            std::snprintf(m_, sizeof m_, "%s: %s", #call, cudaGetErrorString(e_)); \
            return mfail(e_ == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, m_); \
        }                                                                    \
    } while (0)

constexpr int TB = 16;  // tile edge of the product kernels

// Y[b][o] = act( sum_i X[b][i] W[o][i] + bias[o] ), W in BF16, FP32 accumulation.
// act: 0 = identity, 1 = tanh.  Tiled: a 16x16 output tile per CTA, 16-wide slabs of X and W in
// shared memory.
__global__ void k_linear_fwd(const float* __restrict__ X, const __nv_bfloat16* __restrict__ W,
                             const float* __restrict__ bias, float* __restrict__ Y, int B, int I, int O, int act) {
    __shared__ float xs[TB][TB + 1], ws[TB][TB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int b = blockIdx.y * TB + ty, o = blockIdx.x * TB + tx;
    float acc = 0.f;
    for (int i0 = 0; i0 < I; i0 += TB) {
        const int xb = blockIdx.y * TB + ty, xi = i0 + tx;
        xs[ty][tx] = (xb < B && xi < I) ? X[(long long)xb * I + xi] : 0.f;
        const int wo = blockIdx.x * TB + ty, wi = i0 + tx;
        ws[ty][tx] = (wo < O && wi < I) ? __bfloat162float(W[(long long)wo * I + wi]) : 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TB; ++k) acc = fmaf(xs[ty][k], ws[tx][k], acc);
        __syncthreads();
    }
    if (b < B && o < O) {
        float v = acc + bias[o];
        if (act == 1) v = tanhf(v);
        Y[(long long)b * O + o] = v;
    }
}

// dX[b][i] = sum_o dY[b][o] W[o][i]   (optionally times tanh'(A[b][i]) = 1 - A^2 of the input A)
__global__ void k_linear_bwd_x(const float* __restrict__ dY, const __nv_bfloat16* __restrict__ W,
                               const float* __restrict__ A, float* __restrict__ dX, int B, int I, int O) {
    __shared__ float gs[TB][TB + 1], ws[TB][TB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int b = blockIdx.y * TB + ty, i = blockIdx.x * TB + tx;
    float acc = 0.f;
    for (int o0 = 0; o0 < O; o0 += TB) {
        const int gb = blockIdx.y * TB + ty, go = o0 + tx;
        gs[ty][tx] = (gb < B && go < O) ? dY[(long long)gb * O + go] : 0.f;
        const int wo = o0 + ty, wi = blockIdx.x * TB + tx;
        ws[ty][tx] = (wo < O && wi < I) ? __bfloat162float(W[(long long)wo * I + wi]) : 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TB; ++k) acc = fmaf(gs[ty][k], ws[k][tx], acc);
        __syncthreads();
    }
    if (b < B && i < I) {
        if (A) {
            const float a = A[(long long)b * I + i];
            acc *= (1.f - a * a);
        }
        dX[(long long)b * I + i] = acc;
    }
}

// dW[o][i] = sum_b dY[b][o] X[b][i];  dbias[o] = sum_b dY[b][o] (computed by the blockIdx.x == 0 column)
__global__ void k_linear_bwd_w(const float* __restrict__ dY, const float* __restrict__ X, float* __restrict__ dW,
                               float* __restrict__ db, int B, int I, int O) {
    __shared__ float gs[TB][TB + 1], xs[TB][TB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int o = blockIdx.y * TB + ty, i = blockIdx.x * TB + tx;
    float acc = 0.f, accb = 0.f;
    for (int b0 = 0; b0 < B; b0 += TB) {
        const int gb = b0 + tx, go = blockIdx.y * TB + ty;
        gs[ty][tx] = (gb < B && go < O) ? dY[(long long)gb * O + go] : 0.f;  // gs[o][b]
        const int xb = b0 + ty, xi = blockIdx.x * TB + tx;
        xs[ty][tx] = (xb < B && xi < I) ? X[(long long)xb * I + xi] : 0.f;   // xs[b][i]
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TB; ++k) {
            acc = fmaf(gs[ty][k], xs[k][tx], acc);
            accb += gs[ty][k];
        }
        __syncthreads();
    }
    if (o < O && i < I) dW[(long long)o * I + i] = acc;
    if (o < O && blockIdx.x == 0 && tx == 0) db[o] = accb;
}

// loss = mean (Y - T)^2 over B*O values; dY = 2 (Y - T)/(B*O).  One CTA per row block, partial
// sums combined by the host in a fixed order.
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                      double* __restrict__ partial, long long n, float scale) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float d = Y[k] - T[k];
        dY[k] = 2.f * d * scale;
        s += (double)d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Adam (Kingma & Ba 2015) on the FP32 masters, then the BF16 working copy.
__global__ void k_adam(float* __restrict__ p, __nv_bfloat16* __restrict__ pb, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        const float upd = lr * (mk / c1) / (sqrtf(vk / c2) + eps);
        const float pk = p[k] - upd;
        p[k] = pk;
        pb[k] = __float2bfloat16_rn(pk);
    }
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        pb[k] = __float2bfloat16_rn(p[k]);
}

// Deterministic initialisation (uniform in +-1/sqrt(fan_in), SplitMix64 bits), biases zero.
__global__ void k_init_params(float* __restrict__ p, long long off, long long n, int fan_in, unsigned long long seed) {
    const float a = rsqrtf((float)fan_in);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)(off + k + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const float u = (float)((double)(z >> 11) * 0x1p-53) * 2.f - 1.f;
        p[off + k] = a * u;
    }
}

int nblocks(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 2048 ? 2048 : b));
}

}  // namespace

struct lb_mlp {
    int n_in = 0, H = 0, n_out = 0, max_batch = 0;
    cudaStream_t stream = nullptr;
    long long n_par = 0, o_w1 = 0, o_b1 = 0, o_w2 = 0, o_b2 = 0, o_w3 = 0, o_b3 = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // masters, gradients, Adam moments
    __nv_bfloat16* pb = nullptr;                                    // BF16 working weights
    float *a1 = nullptr, *a2 = nullptr, *y = nullptr;              // activations [max_batch][..]
    float *d1 = nullptr, *d2 = nullptr, *dy = nullptr;             // their gradients
    double* partial = nullptr;                                      // loss partial sums
    long long t = 0;                                                // Adam step
};

namespace {

void mlp_free(lb_mlp* m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void* q : {(void*)m->p, (void*)m->g, (void*)m->m, (void*)m->v, (void*)m->pb, (void*)m->a1, (void*)m->a2,
                    (void*)m->y, (void*)m->d1, (void*)m->d2, (void*)m->dy, (void*)m->partial})
        if (q) cudaFree(q);
    delete m;
}

lb_status forward(lb_mlp* m, const float* x, int B) {
    const dim3 blk(TB, TB);
    k_linear_fwd<<<dim3((m->H + TB - 1) / TB, (B + TB - 1) / TB), blk, 0, m->stream>>>(x, m->pb + m->o_w1, m->p + m->o_b1, m->a1, B, m->n_in, m->H, 1);
    k_linear_fwd<<<dim3((m->H + TB - 1) / TB, (B + TB - 1) / TB), blk, 0, m->stream>>>(m->a1, m->pb + m->o_w2, m->p + m->o_b2, m->a2, B, m->H, m->H, 1);
    k_linear_fwd<<<dim3((m->n_out + TB - 1) / TB, (B + TB - 1) / TB), blk, 0, m->stream>>>(m->a2, m->pb + m->o_w3, m->p + m->o_b3, m->y, B, m->H, m->n_out, 0);
    MLP_CK(cudaGetLastError());
    return LB_OK;
}

// Forward, loss and the full gradient into m->g; the loss (host) if requested.
lb_status backward(lb_mlp* m, const float* x, const float* target, int B, double* loss) {
    lb_status st = forward(m, x, B);
    if (st != LB_OK) return st;
    const long long n = (long long)B * m->n_out;
    const int nb = 64;
    k_mse<<<nb, 256, 0, m->stream>>>(m->y, target, m->dy, m->partial, n, 1.f / (float)n);
    const dim3 blk(TB, TB);
    // layer 3
    k_linear_bwd_w<<<dim3((m->H + TB - 1) / TB, (m->n_out + TB - 1) / TB), blk, 0, m->stream>>>(m->dy, m->a2, m->g + m->o_w3, m->g + m->o_b3, B, m->H, m->n_out);
    k_linear_bwd_x<<<dim3((m->H + TB - 1) / TB, (B + TB - 1) / TB), blk, 0, m->stream>>>(m->dy, m->pb + m->o_w3, m->a2, m->d2, B, m->H, m->n_out);
    // layer 2
    k_linear_bwd_w<<<dim3((m->H + TB - 1) / TB, (m->H + TB - 1) / TB), blk, 0, m->stream>>>(m->d2, m->a1, m->g + m->o_w2, m->g + m->o_b2, B, m->H, m->H);
    k_linear_bwd_x<<<dim3((m->H + TB - 1) / TB, (B + TB - 1) / TB), blk, 0, m->stream>>>(m->d2, m->pb + m->o_w2, m->a1, m->d1, B, m->H, m->H);
    // layer 1
    k_linear_bwd_w<<<dim3((m->n_in + TB - 1) / TB, (m->H + TB - 1) / TB), blk, 0, m->stream>>>(m->d1, x, m->g + m->o_w1, m->g + m->o_b1, B, m->n_in, m->H);
    MLP_CK(cudaGetLastError());
    if (loss) {
        std::vector<double> part(nb);
        MLP_CK(cudaMemcpyAsync(part.data(), m->partial, sizeof(double) * nb, cudaMemcpyDeviceToHost, m->stream));
        MLP_CK(cudaStreamSynchronize(m->stream));
        double s = 0.0;
        for (double q : part) s += q;
        *loss = s / (double)n;
    }
    return LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_mlp_create(int n_in, int width, int n_out, int max_batch, uint64_t seed, void* cuda_stream, lb_mlp** out) {
    if (!out) return mfail(LB_EINVAL, "lb_mlp_create: out is null");
    *out = nullptr;
    if (n_in < 1 || width < 1 || n_out < 1 || max_batch < 1) return mfail(LB_EINVAL, "lb_mlp_create: sizes must be >= 1");
    lb_mlp* m = new (std::nothrow) lb_mlp();
    if (!m) return mfail(LB_ENOMEM, "lb_mlp_create: host allocation");
    m->n_in = n_in; m->H = width; m->n_out = n_out; m->max_batch = max_batch;
    m->stream = (cudaStream_t)cuda_stream;
    m->o_w1 = 0; m->o_b1 = m->o_w1 + (long long)width * n_in;
    m->o_w2 = m->o_b1 + width; m->o_b2 = m->o_w2 + (long long)width * width;
    m->o_w3 = m->o_b2 + width; m->o_b3 = m->o_w3 + (long long)n_out * width;
    m->n_par = m->o_b3 + n_out;
    const long long P = m->n_par, B = max_batch;
    cudaError_t e = cudaSuccess;
    auto al = [&](void** q, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(q, bytes); };
    al((void**)&m->p, P * 4); al((void**)&m->g, P * 4); al((void**)&m->m, P * 4); al((void**)&m->v, P * 4);
    al((void**)&m->pb, P * 2);
    al((void**)&m->a1, B * width * 4); al((void**)&m->a2, B * width * 4); al((void**)&m->y, B * n_out * 4);
    al((void**)&m->d1, B * width * 4); al((void**)&m->d2, B * width * 4); al((void**)&m->dy, B * n_out * 4);
    al((void**)&m->partial, 64 * sizeof(double));
    if (e != cudaSuccess) { mlp_free(m); return mfail(LB_ENOMEM, "lb_mlp_create: cudaMalloc"); }
    e = cudaMemsetAsync(m->p, 0, P * 4, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, P * 4, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, P * 4, m->stream);
    if (e != cudaSuccess) { mlp_free(m); return mfail(LB_ECUDA, "lb_mlp_create: memset"); }
    k_init_params<<<nblocks(m->o_b1), 256, 0, m->stream>>>(m->p, m->o_w1, m->o_b1 - m->o_w1, n_in, seed);
    k_init_params<<<nblocks(m->o_b2 - m->o_w2), 256, 0, m->stream>>>(m->p, m->o_w2, m->o_b2 - m->o_w2, width, seed ^ 0x5bd1e995ull);
    k_init_params<<<nblocks(m->o_b3 - m->o_w3), 256, 0, m->stream>>>(m->p, m->o_w3, m->o_b3 - m->o_w3, width, seed ^ 0x27d4eb2full);
    k_to_bf16<<<nblocks(P), 256, 0, m->stream>>>(m->p, m->pb, P);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) { mlp_free(m); return mfail(LB_ECUDA, "lb_mlp_create: init kernels"); }
    *out = m;
    return LB_OK;
}

void lb_mlp_destroy(lb_mlp* m) { mlp_free(m); }

long long lb_mlp_num_params(const lb_mlp* m) { return m ? m->n_par : 0; }

lb_status lb_mlp_forward(lb_mlp* m, const float* x, int batch, float* y) {
    if (!m || !x || !y || batch < 1 || batch > m->max_batch) return mfail(LB_EINVAL, "lb_mlp_forward: bad argument");
    lb_status st = forward(m, x, batch);
    if (st != LB_OK) return st;
    MLP_CK(cudaMemcpyAsync(y, m->y, sizeof(float) * batch * m->n_out, cudaMemcpyDeviceToDevice, m->stream));
    return LB_OK;
}

lb_status lb_mlp_gradients(lb_mlp* m, const float* x, const float* target, int batch, float* grads, double* loss) {
    if (!m || !x || !target || batch < 1 || batch > m->max_batch) return mfail(LB_EINVAL, "lb_mlp_gradients: bad argument");
    lb_status st = backward(m, x, target, batch, loss);
    if (st != LB_OK) return st;
    if (grads) MLP_CK(cudaMemcpyAsync(grads, m->g, sizeof(float) * m->n_par, cudaMemcpyDeviceToDevice, m->stream));
    return LB_OK;
}

lb_status lb_mlp_train_step(lb_mlp* m, const float* x, const float* target, int batch, float lr, double* loss) {
    if (!m || !x || !target || batch < 1 || batch > m->max_batch || !(lr > 0.f))
        return mfail(LB_EINVAL, "lb_mlp_train_step: bad argument");
    lb_status st = backward(m, x, target, batch, loss);
    if (st != LB_OK) return st;
    m->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->t), c2 = 1.f - powf(b2, (float)m->t);
    k_adam<<<nblocks(m->n_par), 256, 0, m->stream>>>(m->p, m->pb, m->g, m->m, m->v, m->n_par, lr, b1, b2, 1e-8f, c1, c2);
    MLP_CK(cudaGetLastError());
    return LB_OK;
}

lb_status lb_mlp_get_params(lb_mlp* m, float* host) {
    if (!m || !host) return mfail(LB_EINVAL, "lb_mlp_get_params: null argument");
    MLP_CK(cudaMemcpyAsync(host, m->p, sizeof(float) * m->n_par, cudaMemcpyDeviceToHost, m->stream));
    MLP_CK(cudaStreamSynchronize(m->stream));
    return LB_OK;
}

lb_status lb_mlp_set_params(lb_mlp* m, const float* host) {
    if (!m || !host) return mfail(LB_EINVAL, "lb_mlp_set_params: null argument");
    MLP_CK(cudaMemcpyAsync(m->p, host, sizeof(float) * m->n_par, cudaMemcpyHostToDevice, m->stream));
    k_to_bf16<<<nblocks(m->n_par), 256, 0, m->stream>>>(m->p, m->pb, m->n_par);
    MLP_CK(cudaGetLastError());
    MLP_CK(cudaStreamSynchronize(m->stream));
    return LB_OK;
}

}  // extern "C"
