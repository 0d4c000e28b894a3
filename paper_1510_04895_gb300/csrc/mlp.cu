// Parameter-predicting MLP (a learned choice of the filter parameters; the
// paper's nearest passage is the adaptive choice of N_p and N_S from the DOS,
// Sec. 6):
// features of (H, window) -> tanh(W1 x + b1) -> tanh(W2 h1 + b2) -> W3 h2 + b3
// with outputs (log N_p, log n_s, kernel logit).  FP32 training and inference
// on the GPU with the kernels below (forward, loss, backward, Adam); every sum
// runs in a fixed order, so results are deterministic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

struct chebfd_mlp {
    int n_in = 0, n_h = 0, n_out = 0;
    int64_t count = 0;       // number of parameters
    float* params = nullptr; // W1, b1, W2, b2, W3, b3 (row-major W: out x in)
    float* grads = nullptr;
    float* m = nullptr;      // Adam moments
    float* v = nullptr;
    int t = 0;               // Adam step
    float* work = nullptr;   // activations and their gradients
    int64_t work_cap = 0;    // capacity in samples
};

namespace chebfd {

namespace {

struct Layout {
    int64_t W1, b1, W2, b2, W3, b3, total;
};

Layout layout_of(int n_in, int n_h, int n_out) {
    Layout L;
    L.W1 = 0;
    L.b1 = L.W1 + (int64_t)n_h * n_in;
    L.W2 = L.b1 + n_h;
    L.b2 = L.W2 + (int64_t)n_h * n_h;
    L.W3 = L.b2 + n_h;
    L.b3 = L.W3 + (int64_t)n_out * n_h;
    L.total = L.b3 + n_out;
    return L;
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

// Y[b, m] = act(sum_k X[b, k] W[m, k] + bias[m])
__global__ void linear_fwd(const float* X, const float* W, const float* bias, int B, int K, int M,
                           int act_tanh, float* Y) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)B * M;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / M), m = (int)(t % M);
        float s = bias[m];
        for (int k = 0; k < K; ++k) s = fmaf(X[(int64_t)b * K + k], W[(int64_t)m * K + k], s);
        Y[t] = act_tanh ? tanhf(s) : s;
    }
}

// per-sample loss and dL/dz for z (B x 3), targets T (B x 3)
__global__ void loss_fwd_bwd(const float* Z, const float* T, int B, float* per, float* dZ) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const float z0 = Z[3 * b], z1 = Z[3 * b + 1], z2 = Z[3 * b + 2];
        const float t0 = T[3 * b], t1 = T[3 * b + 1], t2 = T[3 * b + 2];
        const float sp = fmaxf(z2, 0.f) + log1pf(expf(-fabsf(z2)));  // softplus(z2)
        per[b] = (z0 - t0) * (z0 - t0) + (z1 - t1) * (z1 - t1) + sp - t2 * z2;
        const float inv = 1.f / (float)B;
        dZ[3 * b] = 2.f * (z0 - t0) * inv;
        dZ[3 * b + 1] = 2.f * (z1 - t1) * inv;
        dZ[3 * b + 2] = (1.f / (1.f + expf(-z2)) - t2) * inv;
    }
}

__global__ void sum_kernel(const float* x, int n, float* out) {
    __shared__ float s[256];
    float acc = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0] / (float)n;
}

// dW[m, k] = sum_b dA[b, m] X[b, k] ; db[m] = sum_b dA[b, m]
__global__ void linear_bwd_w(const float* dA, const float* X, int B, int K, int M, float* dW,
                             float* db) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)M * (K + 1);
         t += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(t / (K + 1)), k = (int)(t % (K + 1));
        float s = 0.f;
        if (k < K) {
            for (int b = 0; b < B; ++b) s = fmaf(dA[(int64_t)b * M + m], X[(int64_t)b * K + k], s);
            dW[(int64_t)m * K + k] = s;
        } else {
            for (int b = 0; b < B; ++b) s += dA[(int64_t)b * M + m];
            db[m] = s;
        }
    }
}

// dA_prev[b, k] = (sum_m dA[b, m] W[m, k]) * (1 - H[b, k]^2)   (through tanh)
__global__ void linear_bwd_x_tanh(const float* dA, const float* W, const float* Hprev, int B,
                                  int K, int M, float* dAprev) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)B * K;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / K), k = (int)(t % K);
        float s = 0.f;
        for (int m = 0; m < M; ++m) s = fmaf(dA[(int64_t)b * M + m], W[(int64_t)m * K + k], s);
        const float h = Hprev[t];
        dAprev[t] = s * (1.f - h * h);
    }
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

void ensure_work(chebfd_mlp* N, int B) {
    if (B <= N->work_cap) return;
    cudaFree(N->work);
    N->work = nullptr;
    N->work_cap = 0;
    // h1, h2, z, dz, da2, da1, per, loss
    const size_t floats = (size_t)B * (2 * N->n_h + 2 * N->n_out + 2 * N->n_h + 1) + 8;
    CHEBFD_CHECK_CUDA(cudaMalloc(&N->work, floats * sizeof(float)));
    N->work_cap = B;
}

struct Acts {
    float *h1, *h2, *z, *dz, *da2, *da1, *per, *loss;
};

Acts acts_of(chebfd_mlp* N, int B) {
    Acts a;
    float* p = N->work;
    a.h1 = p;
    p += (size_t)B * N->n_h;
    a.h2 = p;
    p += (size_t)B * N->n_h;
    a.z = p;
    p += (size_t)B * N->n_out;
    a.dz = p;
    p += (size_t)B * N->n_out;
    a.da2 = p;
    p += (size_t)B * N->n_h;
    a.da1 = p;
    p += (size_t)B * N->n_h;
    a.per = p;
    p += B;
    a.loss = p;
    return a;
}

void forward(chebfd_mlp* N, const float* X, int B, const Acts& a, cudaStream_t s) {
    const Layout L = layout_of(N->n_in, N->n_h, N->n_out);
    const float* P = N->params;
    linear_fwd<<<blocks_for((int64_t)B * N->n_h), 256, 0, s>>>(X, P + L.W1, P + L.b1, B, N->n_in,
                                                               N->n_h, 1, a.h1);
    linear_fwd<<<blocks_for((int64_t)B * N->n_h), 256, 0, s>>>(a.h1, P + L.W2, P + L.b2, B,
                                                               N->n_h, N->n_h, 1, a.h2);
    linear_fwd<<<blocks_for((int64_t)B * N->n_out), 256, 0, s>>>(a.h2, P + L.W3, P + L.b3, B,
                                                                 N->n_h, N->n_out, 0, a.z);
    CHEBFD_CHECK_CUDA(cudaGetLastError());
}

}  // namespace

}  // namespace chebfd

using namespace chebfd;

extern "C" {

chebfd_status chebfd_mlp_create(int n_in, int n_hidden, int n_out, chebfd_mlp** out) {
    chebfd_mlp* N = nullptr;
    chebfd_status st = guarded([&] {
        CHEBFD_REQUIRE(out, CHEBFD_EINVAL, "null output");
        CHEBFD_REQUIRE(n_in >= 1 && n_hidden >= 1 && n_out == 3, CHEBFD_EINVAL,
                       "need n_in >= 1, n_hidden >= 1 and n_out == 3");
        N = new chebfd_mlp();
        N->n_in = n_in;
        N->n_h = n_hidden;
        N->n_out = n_out;
        N->count = layout_of(n_in, n_hidden, n_out).total;
        const size_t bytes = (size_t)N->count * sizeof(float);
        CHEBFD_CHECK_CUDA(cudaMalloc(&N->params, bytes));
        CHEBFD_CHECK_CUDA(cudaMalloc(&N->grads, bytes));
        CHEBFD_CHECK_CUDA(cudaMalloc(&N->m, bytes));
        CHEBFD_CHECK_CUDA(cudaMalloc(&N->v, bytes));
        CHEBFD_CHECK_CUDA(cudaMemset(N->params, 0, bytes));
        CHEBFD_CHECK_CUDA(cudaMemset(N->grads, 0, bytes));
        CHEBFD_CHECK_CUDA(cudaMemset(N->m, 0, bytes));
        CHEBFD_CHECK_CUDA(cudaMemset(N->v, 0, bytes));
    });
    if (st != CHEBFD_OK) {
        if (N) {
            cudaFree(N->params);
            cudaFree(N->grads);
            cudaFree(N->m);
            cudaFree(N->v);
            delete N;
        }
        return st;
    }
    *out = N;
    return CHEBFD_OK;
}

chebfd_status chebfd_mlp_num_params(const chebfd_mlp* N, int64_t* count) {
    return guarded([&] {
        CHEBFD_REQUIRE(N && count, CHEBFD_EINVAL, "null argument");
        *count = N->count;
    });
}

chebfd_status chebfd_mlp_set_params(chebfd_mlp* N, const float* host, int64_t count) {
    return guarded([&] {
        CHEBFD_REQUIRE(N && host && count == N->count, CHEBFD_EINVAL, "bad parameter array");
        CHEBFD_CHECK_CUDA(
            cudaMemcpy(N->params, host, count * sizeof(float), cudaMemcpyHostToDevice));
        CHEBFD_CHECK_CUDA(cudaMemset(N->m, 0, count * sizeof(float)));
        CHEBFD_CHECK_CUDA(cudaMemset(N->v, 0, count * sizeof(float)));
        N->t = 0;
    });
}

chebfd_status chebfd_mlp_get_params(const chebfd_mlp* N, float* host, float* host_grads,
                                    int64_t count) {
    return guarded([&] {
        CHEBFD_REQUIRE(N && count == N->count, CHEBFD_EINVAL, "bad parameter array");
        if (host)
            CHEBFD_CHECK_CUDA(
                cudaMemcpy(host, N->params, count * sizeof(float), cudaMemcpyDeviceToHost));
        if (host_grads)
            CHEBFD_CHECK_CUDA(
                cudaMemcpy(host_grads, N->grads, count * sizeof(float), cudaMemcpyDeviceToHost));
    });
}

chebfd_status chebfd_mlp_forward(chebfd_mlp* N, const float* X, int B, float* Z, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(N && X && Z && B >= 1, CHEBFD_EINVAL, "bad forward arguments");
        cudaStream_t s = as_stream(stream);
        ensure_work(N, B);
        const Acts a = acts_of(N, B);
        forward(N, X, B, a, s);
        CHEBFD_CHECK_CUDA(cudaMemcpyAsync(Z, a.z, (size_t)B * N->n_out * sizeof(float),
                                          cudaMemcpyDeviceToDevice, s));
    });
}

chebfd_status chebfd_mlp_loss_grad(chebfd_mlp* N, const float* X, const float* T, int B,
                                   float* loss, void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(N && X && T && B >= 1, CHEBFD_EINVAL, "bad training arguments");
        cudaStream_t s = as_stream(stream);
        ensure_work(N, B);
        const Acts a = acts_of(N, B);
        const Layout L = layout_of(N->n_in, N->n_h, N->n_out);
        forward(N, X, B, a, s);
        loss_fwd_bwd<<<blocks_for(B), 256, 0, s>>>(a.z, T, B, a.per, a.dz);
        sum_kernel<<<1, 256, 0, s>>>(a.per, B, a.loss);
        float* G = N->grads;
        const float* P = N->params;
        linear_bwd_w<<<blocks_for((int64_t)N->n_out * (N->n_h + 1)), 256, 0, s>>>(
            a.dz, a.h2, B, N->n_h, N->n_out, G + L.W3, G + L.b3);
        linear_bwd_x_tanh<<<blocks_for((int64_t)B * N->n_h), 256, 0, s>>>(
            a.dz, P + L.W3, a.h2, B, N->n_h, N->n_out, a.da2);
        linear_bwd_w<<<blocks_for((int64_t)N->n_h * (N->n_h + 1)), 256, 0, s>>>(
            a.da2, a.h1, B, N->n_h, N->n_h, G + L.W2, G + L.b2);
        linear_bwd_x_tanh<<<blocks_for((int64_t)B * N->n_h), 256, 0, s>>>(
            a.da2, P + L.W2, a.h1, B, N->n_h, N->n_h, a.da1);
        linear_bwd_w<<<blocks_for((int64_t)N->n_h * (N->n_in + 1)), 256, 0, s>>>(
            a.da1, X, B, N->n_in, N->n_h, G + L.W1, G + L.b1);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
        if (loss) {
            CHEBFD_CHECK_CUDA(
                cudaMemcpyAsync(loss, a.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
            CHEBFD_CHECK_CUDA(cudaStreamSynchronize(s));
        }
    });
}

chebfd_status chebfd_mlp_adam(chebfd_mlp* N, float lr, float beta1, float beta2, float eps,
                              void* stream) {
    return guarded([&] {
        CHEBFD_REQUIRE(N && lr > 0.f, CHEBFD_EINVAL, "bad Adam arguments");
        N->t += 1;
        const float c1 = 1.f - std::pow(beta1, (float)N->t);
        const float c2 = 1.f - std::pow(beta2, (float)N->t);
        adam_kernel<<<blocks_for(N->count), 256, 0, as_stream(stream)>>>(
            N->params, N->grads, N->m, N->v, N->count, lr, beta1, beta2, eps, c1, c2);
        CHEBFD_CHECK_CUDA(cudaGetLastError());
    });
}

chebfd_status chebfd_mlp_destroy(chebfd_mlp* N) {
    return guarded([&] {
        if (!N) return;
        cudaFree(N->params);
        cudaFree(N->grads);
        cudaFree(N->m);
        cudaFree(N->v);
        cudaFree(N->work);
        delete N;
    });
}

}  // extern "C"
