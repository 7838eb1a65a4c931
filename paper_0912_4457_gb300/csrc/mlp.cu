// Learned subspace sizes: a 16 -> 64 -> 64 -> 2 multilayer perceptron (tanh,
// tanh, linear; FP32) that maps features of an operator and source to
// (log2 k, log2 l), the outer and inner Krylov sizes that reach a requested
// tolerance.  The paper fixes k and l by hand; this predictor and its
// training are the library's.  Forward pass, backward pass and the Adam
// update are hand-written kernels; the whole batch (at most kMlpMaxBatch
// samples) is processed by one CTA, which is ample for this size.
//
// Loss: mean over the batch of the squared error of the standardised outputs,
//   L = (1/n) sum_s sum_o (z_so - t_so)^2 / 2,  t = (y - y_mean) / y_std.
// Inputs are standardised the same way with the training set's statistics.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nksign.h"

namespace {

constexpr int kIn = NK_MLP_IN, kH = NK_MLP_HIDDEN, kOut = NK_MLP_OUT;
constexpr int kMlpMaxBatch = 256;
// parameter layout (flattened): W1[kH][kIn], b1[kH], W2[kH][kH], b2[kH], W3[kOut][kH], b3[kOut]
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kOut * kH, kParams = ob3 + kOut;
static_assert(kParams == NK_MLP_PARAMS, "parameter count");

struct MlpDev {
    float* w;    // parameters
    float* g;    // gradient
    float* m;    // Adam first moment
    float* v;    // Adam second moment
    float* x;    // standardised inputs [batch][kIn]
    float* t;    // standardised targets [batch][kOut]
    float* z;    // outputs [batch][kOut]
    float* loss; // [1]
    float* h1;   // tanh activations of layer 1 [batch][kH]
    float* h2;   // layer 2
    float* d1;   // dL/d(pre-activation) of layer 1 [batch][kH]
    float* d2;   // layer 2
};

// forward of one sample; h1, h2 are the tanh activations
__device__ void fwd_sample(const float* __restrict__ w, const float* __restrict__ x, float* h1, float* h2,
                           float* z) {
    for (int i = 0; i < kH; ++i) {
        float a = w[ob1 + i];
        for (int j = 0; j < kIn; ++j) a = fmaf(w[oW1 + i * kIn + j], x[j], a);
        h1[i] = tanhf(a);
    }
    for (int i = 0; i < kH; ++i) {
        float a = w[ob2 + i];
        for (int j = 0; j < kH; ++j) a = fmaf(w[oW2 + i * kH + j], h1[j], a);
        h2[i] = tanhf(a);
    }
    for (int o = 0; o < kOut; ++o) {
        float a = w[ob3 + o];
        for (int j = 0; j < kH; ++j) a = fmaf(w[oW3 + o * kH + j], h2[j], a);
        z[o] = a;
    }
}

// Forward for the batch (one thread per sample), then, if t != nullptr, the
// loss and the gradient: per-sample backward passes write their activations
// and deltas to per-sample rows of global scratch; each parameter gradient is
// then summed over the samples in fixed order (deterministic).
__global__ void __launch_bounds__(kMlpMaxBatch) k_mlp_fwd_bwd(MlpDev d, int n, int want_grad) {
    __shared__ float dzs[kMlpMaxBatch][kOut];
    float (*h1s)[kH] = reinterpret_cast<float (*)[kH]>(d.h1);
    float (*h2s)[kH] = reinterpret_cast<float (*)[kH]>(d.h2);
    float (*d1s)[kH] = reinterpret_cast<float (*)[kH]>(d.d1);
    float (*d2s)[kH] = reinterpret_cast<float (*)[kH]>(d.d2);
    const int s = threadIdx.x;
    if (s < n) {
        float z[kOut];
        fwd_sample(d.w, d.x + (size_t)s * kIn, h1s[s], h2s[s], z);
        for (int o = 0; o < kOut; ++o) {
            d.z[(size_t)s * kOut + o] = z[o];
            dzs[s][o] = want_grad ? (z[o] - d.t[(size_t)s * kOut + o]) / (float)n : 0.0f;
        }
        if (want_grad) {
            for (int j = 0; j < kH; ++j) {
                float g = 0.0f;
                for (int o = 0; o < kOut; ++o) g = fmaf(d.w[oW3 + o * kH + j], dzs[s][o], g);
                d2s[s][j] = g * (1.0f - h2s[s][j] * h2s[s][j]);
            }
            for (int j = 0; j < kH; ++j) {
                float g = 0.0f;
                for (int i = 0; i < kH; ++i) g = fmaf(d.w[oW2 + i * kH + j], d2s[s][i], g);
                d1s[s][j] = g * (1.0f - h1s[s][j] * h1s[s][j]);
            }
        }
    }
    __syncthreads();
    if (!want_grad) return;
    // loss (fixed order)
    if (threadIdx.x == 0) {
        float L = 0.0f;
        for (int q = 0; q < n; ++q)
            for (int o = 0; o < kOut; ++o) {
                const float e = d.z[(size_t)q * kOut + o] - d.t[(size_t)q * kOut + o];
                L = fmaf(0.5f * e, e, L);
            }
        d.loss[0] = L / (float)n;
    }
    // parameter gradients: each thread owns parameters, sums over samples in order
    for (int pi = threadIdx.x; pi < kParams; pi += blockDim.x) {
        float g = 0.0f;
        if (pi < ob1) {
            const int i = pi / kIn, j = pi % kIn;
            for (int q = 0; q < n; ++q) g = fmaf(d1s[q][i], d.x[(size_t)q * kIn + j], g);
        } else if (pi < oW2) {
            const int i = pi - ob1;
            for (int q = 0; q < n; ++q) g += d1s[q][i];
        } else if (pi < ob2) {
            const int i = (pi - oW2) / kH, j = (pi - oW2) % kH;
            for (int q = 0; q < n; ++q) g = fmaf(d2s[q][i], h1s[q][j], g);
        } else if (pi < oW3) {
            const int i = pi - ob2;
            for (int q = 0; q < n; ++q) g += d2s[q][i];
        } else if (pi < ob3) {
            const int o = (pi - oW3) / kH, j = (pi - oW3) % kH;
            for (int q = 0; q < n; ++q) g = fmaf(dzs[q][o], h2s[q][j], g);
        } else {
            const int o = pi - ob3;
            for (int q = 0; q < n; ++q) g += dzs[q][o];
        }
        d.g[pi] = g;
    }
}

// Adam (Kingma & Ba) with bias correction, step number t (1-based), and
// decoupled weight decay wd (Loshchilov & Hutter: w -= lr wd w; 0 = plain Adam)
__global__ void k_adam(MlpDev d, float lr, float b1, float b2, float eps, float wd, int t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float g = d.g[i];
    const float m = b1 * d.m[i] + (1.0f - b1) * g;
    const float v = b2 * d.v[i] + (1.0f - b2) * g * g;
    d.m[i] = m;
    d.v[i] = v;
    const float mh = m / (1.0f - powf(b1, (float)t));
    const float vh = v / (1.0f - powf(b2, (float)t));
    d.w[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * d.w[i]);
}

}  // namespace

struct nk_mlp {
    MlpDev d;
    float xmu[kIn], xsd[kIn], ymu[kOut], ysd[kOut];
    int step = 0;
    float wd = 0.0f;
    std::string err = "no error";
};

static int mlp_fail(nk_mlp* m, int code, const char* msg) {
    if (m) m->err = msg;
    return code;
}

#define MLP_CUDA(m, call)                                                   \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return mlp_fail(m, NK_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

// splitmix64: deterministic initial weights from a seed
static uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static int upload_batch(nk_mlp* m, const float* X, const float* Y, int n) {
    std::vector<float> xs((size_t)n * kIn), ts((size_t)n * kOut);
    for (int s = 0; s < n; ++s) {
        for (int j = 0; j < kIn; ++j) xs[(size_t)s * kIn + j] = (X[(size_t)s * kIn + j] - m->xmu[j]) / m->xsd[j];
        for (int o = 0; Y && o < kOut; ++o)
            ts[(size_t)s * kOut + o] = (Y[(size_t)s * kOut + o] - m->ymu[o]) / m->ysd[o];
    }
    MLP_CUDA(m, cudaMemcpy(m->d.x, xs.data(), sizeof(float) * xs.size(), cudaMemcpyHostToDevice));
    if (Y) MLP_CUDA(m, cudaMemcpy(m->d.t, ts.data(), sizeof(float) * ts.size(), cudaMemcpyHostToDevice));
    return NK_OK;
}

extern "C" {

int nk_mlp_create(unsigned long long seed, nk_mlp** out) {
    if (!out) return NK_EINVAL;
    nk_mlp* m = new nk_mlp();
    float* base = nullptr;
    const size_t nfl = 4 * (size_t)kParams + (size_t)kMlpMaxBatch * (kIn + 2 * kOut + 4 * kH) + 1;
    if (cudaMalloc(&base, sizeof(float) * nfl) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return NK_ENOMEM;
    }
    m->d.w = base;
    m->d.g = base + kParams;
    m->d.m = base + 2 * kParams;
    m->d.v = base + 3 * kParams;
    m->d.x = base + 4 * kParams;
    m->d.t = m->d.x + (size_t)kMlpMaxBatch * kIn;
    m->d.z = m->d.t + (size_t)kMlpMaxBatch * kOut;
    m->d.loss = m->d.z + (size_t)kMlpMaxBatch * kOut;
    m->d.h1 = m->d.loss + 1;
    m->d.h2 = m->d.h1 + (size_t)kMlpMaxBatch * kH;
    m->d.d1 = m->d.h2 + (size_t)kMlpMaxBatch * kH;
    m->d.d2 = m->d.d1 + (size_t)kMlpMaxBatch * kH;
    // Glorot-uniform weights, zero biases
    std::vector<float> w(kParams, 0.0f);
    uint64_t st = seed;
    auto uni = [&](float a) { return (float)(((splitmix(st) >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0) * a; };
    for (int i = 0; i < kH * kIn; ++i) w[oW1 + i] = uni(std::sqrt(6.0f / (kIn + kH)));
    for (int i = 0; i < kH * kH; ++i) w[oW2 + i] = uni(std::sqrt(6.0f / (kH + kH)));
    for (int i = 0; i < kOut * kH; ++i) w[oW3 + i] = uni(std::sqrt(6.0f / (kH + kOut)));
    cudaMemcpy(m->d.w, w.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice);
    cudaMemset(m->d.m, 0, sizeof(float) * 2 * kParams);
    for (int j = 0; j < kIn; ++j) { m->xmu[j] = 0.0f; m->xsd[j] = 1.0f; }
    for (int o = 0; o < kOut; ++o) { m->ymu[o] = 0.0f; m->ysd[o] = 1.0f; }
    if (cudaGetLastError() != cudaSuccess) {
        cudaFree(base);
        delete m;
        return NK_ECUDA;
    }
    *out = m;
    return NK_OK;
}

int nk_mlp_set_norm(nk_mlp* m, const float* xmu, const float* xsd, const float* ymu, const float* ysd) {
    if (!m || !xmu || !xsd || !ymu || !ysd) return NK_EINVAL;
    for (int j = 0; j < kIn; ++j) {
        if (!(xsd[j] > 0.0f)) return mlp_fail(m, NK_EINVAL, "input scales must be positive");
        m->xmu[j] = xmu[j];
        m->xsd[j] = xsd[j];
    }
    for (int o = 0; o < kOut; ++o) {
        if (!(ysd[o] > 0.0f)) return mlp_fail(m, NK_EINVAL, "output scales must be positive");
        m->ymu[o] = ymu[o];
        m->ysd[o] = ysd[o];
    }
    return NK_OK;
}

int nk_mlp_set_weight_decay(nk_mlp* m, float wd) {
    if (!m) return NK_EINVAL;
    if (!(wd >= 0.0f) || !(wd < 1.0f)) return mlp_fail(m, NK_EINVAL, "weight decay must be in [0, 1)");
    m->wd = wd;
    return NK_OK;
}

int nk_mlp_get_params(nk_mlp* m, float* params) {
    if (!m || !params) return NK_EINVAL;
    MLP_CUDA(m, cudaMemcpy(params, m->d.w, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    return NK_OK;
}

int nk_mlp_set_params(nk_mlp* m, const float* params) {
    if (!m || !params) return NK_EINVAL;
    MLP_CUDA(m, cudaMemcpy(m->d.w, params, sizeof(float) * kParams, cudaMemcpyHostToDevice));
    MLP_CUDA(m, cudaMemset(m->d.m, 0, sizeof(float) * 2 * kParams));
    m->step = 0;
    return NK_OK;
}

int nk_mlp_loss_grad(nk_mlp* m, const float* X, const float* Y, int n, float* loss, float* grad) {
    if (!m || !X || !Y || n < 1 || n > kMlpMaxBatch) return mlp_fail(m, NK_EINVAL, "need 1 <= n <= 256");
    int rc = upload_batch(m, X, Y, n);
    if (rc) return rc;
    k_mlp_fwd_bwd<<<1, kMlpMaxBatch>>>(m->d, n, 1);
    MLP_CUDA(m, cudaGetLastError());
    if (loss) MLP_CUDA(m, cudaMemcpy(loss, m->d.loss, sizeof(float), cudaMemcpyDeviceToHost));
    if (grad) MLP_CUDA(m, cudaMemcpy(grad, m->d.g, sizeof(float) * kParams, cudaMemcpyDeviceToHost));
    MLP_CUDA(m, cudaDeviceSynchronize());
    return NK_OK;
}

int nk_mlp_train(nk_mlp* m, const float* X, const float* Y, int n, int epochs, float lr, float* loss_hist) {
    if (!m || !X || !Y || n < 1 || n > kMlpMaxBatch || epochs < 1 || !(lr > 0.0f))
        return mlp_fail(m, NK_EINVAL, "need 1 <= n <= 256, epochs >= 1, lr > 0");
    int rc = upload_batch(m, X, Y, n);
    if (rc) return rc;
    for (int e = 0; e < epochs; ++e) {
        k_mlp_fwd_bwd<<<1, kMlpMaxBatch>>>(m->d, n, 1);
        ++m->step;
        k_adam<<<(kParams + 255) / 256, 256>>>(m->d, lr, 0.9f, 0.999f, 1e-8f, m->wd, m->step);
        if (loss_hist) MLP_CUDA(m, cudaMemcpyAsync(loss_hist + e, m->d.loss, sizeof(float), cudaMemcpyDeviceToHost, 0));
    }
    MLP_CUDA(m, cudaGetLastError());
    MLP_CUDA(m, cudaDeviceSynchronize());
    return NK_OK;
}

int nk_mlp_forward(nk_mlp* m, const float* X, int n, float* Yout) {
    if (!m || !X || !Yout || n < 1 || n > kMlpMaxBatch) return mlp_fail(m, NK_EINVAL, "need 1 <= n <= 256");
    int rc = upload_batch(m, X, nullptr, n);
    if (rc) return rc;
    k_mlp_fwd_bwd<<<1, kMlpMaxBatch>>>(m->d, n, 0);
    std::vector<float> z((size_t)n * kOut);
    MLP_CUDA(m, cudaMemcpy(z.data(), m->d.z, sizeof(float) * z.size(), cudaMemcpyDeviceToHost));
    for (int s = 0; s < n; ++s)
        for (int o = 0; o < kOut; ++o) Yout[(size_t)s * kOut + o] = z[(size_t)s * kOut + o] * m->ysd[o] + m->ymu[o];
    return NK_OK;
}

const char* nk_mlp_last_error(const nk_mlp* m) { return m ? m->err.c_str() : "null predictor"; }

void nk_mlp_destroy(nk_mlp* m) {
    if (!m) return;
    cudaFree(m->d.w);
    delete m;
}

}  // extern "C"
