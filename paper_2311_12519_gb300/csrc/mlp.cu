// The learned cost model's network: a perceptron F -> 64 -> 64 -> 1 with ReLU,
// fp32, trained with Adam on the mean squared error of standardised targets.
// It has no counterpart in the paper, which picks its parameters by the noise
// analysis of Sec. 3.2.1; here the network ranks kernel schedules and layouts
// by predicted latency.
//
// Kernels:
//   k_colstats   mean and standard deviation of every feature column and of y
//   k_mlp_grad   forward + backward of a mini-batch, one partial gradient per block
//   k_mlp_adam   sums the partial gradients in a fixed order and takes one Adam step
//   k_mlp_fwd    predictions (destandardised)
// A block of 64 threads owns one hidden unit per thread; a sample's activations
// live in shared memory.  Partial gradients are reduced in block order, so a
// training run is deterministic for a given seed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "../../include/hyena_costmodel.h"
#include "internal.h"

namespace {
using hy::fail;
using u32 = uint32_t;
using u64 = uint64_t;

constexpr int H = 64;        // hidden width
constexpr int FMAX = 64;     // most features
constexpr int GRAD_BLOCKS = 64;

#define MLP_CUDA(x)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ == cudaErrorMemoryAllocation) {                                             \
            cudaGetLastError();                                                            \
            fail(HE_ENOMEM, std::string(#x ": ") + cudaGetErrorString(e_));                \
        }                                                                                  \
        if (e_ != cudaSuccess) fail(HE_ECUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
    } while (0)

// parameter offsets inside the flat vector: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3
struct Off {
    u32 F, W1, b1, W2, b2, w3, b3, n;
    __host__ __device__ explicit Off(u32 f) : F(f) {
        W1 = 0, b1 = H * F, W2 = b1 + H, b2 = W2 + H * H, w3 = b2 + H, b3 = w3 + H, n = b3 + 1;
    }
};

__device__ __forceinline__ u64 splitmix(u64 z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// column c < F of X, or y for c == F: mean and standard deviation (population, floor 1e-6)
__global__ void k_colstats(const float* __restrict__ X, const float* __restrict__ y, u32 n, u32 F,
                           float* __restrict__ mean, float* __restrict__ stdv) {
    __shared__ double s1[256], s2[256];
    const u32 c = blockIdx.x;
    double a = 0, b = 0;
    for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = c < F ? X[(size_t)i * F + c] : y[i];
        a += v, b += v * v;
    }
    s1[threadIdx.x] = a, s2[threadIdx.x] = b;
    __syncthreads();
    for (u32 h = blockDim.x / 2; h; h >>= 1) {
        if (threadIdx.x < h) s1[threadIdx.x] += s1[threadIdx.x + h], s2[threadIdx.x] += s2[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = s1[0] / n, var = s2[0] / n - m * m;
        mean[c] = (float)m;
        stdv[c] = (float)fmax(sqrt(fmax(var, 0.0)), 1e-6);
    }
}

struct Net {
    const float* p;           // parameters
    const float* xm;          // feature means [F]
    const float* xs;          // feature standard deviations [F]
    u32 F;
};

// forward pass of one sample by 64 threads; x (standardised) in xs_sm, returns y on every thread
__device__ float forward(const Net& net, const Off& o, const float* xsm, float* h1, float* h2, float* red) {
    const u32 j = threadIdx.x;
    float a = net.p[o.b1 + j];
    for (u32 i = 0; i < net.F; i++) a += net.p[o.W1 + j * net.F + i] * xsm[i];
    h1[j] = fmaxf(a, 0.f);
    __syncthreads();
    float b = net.p[o.b2 + j];
#pragma unroll 8
    for (u32 k = 0; k < H; k++) b += net.p[o.W2 + j * H + k] * h1[k];
    h2[j] = fmaxf(b, 0.f);
    // y = w3 . h2 + b3: warp sums, then the two warps' sums in a fixed order
    float v = net.p[o.w3 + j] * h2[j];
    for (int d = 16; d; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((j & 31) == 0) red[j >> 5] = v;
    __syncthreads();
    const float y = red[0] + red[1] + net.p[o.b3];
    __syncthreads();
    return y;
}

__device__ void load_x(const Net& net, const float* X, u32 i, float* xsm) {
    for (u32 c = threadIdx.x; c < net.F; c += blockDim.x)
        xsm[c] = (X[(size_t)i * net.F + c] - net.xm[c]) / net.xs[c];
    __syncthreads();
}

// one mini-batch of `batch` samples drawn with replacement by a counter-based generator
// (index = SplitMix64(seed, step, slot) mod n); block b takes slots b, b + gridDim.x, ...
// Writes its gradient of mean squared error (of standardised y) to part[b][0..n) and its
// sum of squared errors to part[b][n].
__global__ void __launch_bounds__(H) k_mlp_grad(Net net, const float* __restrict__ X, const float* __restrict__ y,
                                                 u32 n, float ym, float ys, u32 batch, u64 seed, u64 step,
                                                 float* __restrict__ part) {
    __shared__ float xsm[FMAX], h1[H], h2[H], d2[H], red[2];
    const Off o(net.F);
    const u32 j = threadIdx.x;
    float gW1[FMAX], gW2[H];
#pragma unroll
    for (int i = 0; i < FMAX; i++) gW1[i] = 0;
#pragma unroll
    for (int i = 0; i < H; i++) gW2[i] = 0;
    float gb1 = 0, gb2 = 0, gw3 = 0, gb3 = 0, sse = 0;
    for (u32 slot = blockIdx.x; slot < batch; slot += gridDim.x) {
        const u32 i = (u32)(splitmix(seed ^ splitmix(step * 0x100000001ull + slot)) % n);
        load_x(net, X, i, xsm);
        const float out = forward(net, o, xsm, h1, h2, red);
        const float err = out - (y[i] - ym) / ys;
        sse += err * err;
        const float dy = 2.f * err / (float)batch;
        // layer 3
        gw3 += dy * h2[j];
        gb3 += dy;
        // layer 2: delta of hidden unit j
        const float dj2 = h2[j] > 0.f ? dy * net.p[o.w3 + j] : 0.f;
        d2[j] = dj2;
#pragma unroll
        for (int k = 0; k < H; k++) gW2[k] += dj2 * h1[k];
        gb2 += dj2;
        __syncthreads();
        // layer 1: delta of hidden unit j sums over the units of layer 2
        float dj1 = 0.f;
        if (h1[j] > 0.f)
            for (u32 k = 0; k < H; k++) dj1 += net.p[o.W2 + k * H + j] * d2[k];
#pragma unroll
        for (int c = 0; c < FMAX; c++)
            if (c < (int)net.F) gW1[c] += dj1 * xsm[c];
        gb1 += dj1;
        __syncthreads();
    }
    float* g = part + (size_t)blockIdx.x * (o.n + 1);
#pragma unroll
    for (int c = 0; c < FMAX; c++)
        if (c < (int)net.F) g[o.W1 + j * net.F + c] = gW1[c];
    g[o.b1 + j] = gb1;
#pragma unroll
    for (int k = 0; k < H; k++) g[o.W2 + j * H + k] = gW2[k];
    g[o.b2 + j] = gb2;
    g[o.w3 + j] = gw3;
    if (j == 0) {
        g[o.b3] = gb3;
        g[o.n] = sse;
    }
}

// Adam (Kingma and Ba, 2015) on the summed partial gradients; t = step number from 1
__global__ void k_mlp_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ part, u32 n_par, u32 n_part, float lr, float b1, float b2,
                           float eps, u32 t) {
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_par) return;
    float g = 0.f;
    for (u32 b = 0; b < n_part; b++) g += part[(size_t)b * (n_par + 1) + i];
    const float mi = b1 * m[i] + (1.f - b1) * g, vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi, v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t)), vh = vi / (1.f - powf(b2, (float)t));
    p[i] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void __launch_bounds__(H) k_mlp_fwd(Net net, const float* __restrict__ X, u32 n, float ym, float ys,
                                               float* __restrict__ out) {
    __shared__ float xsm[FMAX], h1[H], h2[H], red[2];
    const Off o(net.F);
    for (u32 i = blockIdx.x; i < n; i += gridDim.x) {
        load_x(net, X, i, xsm);
        const float y = forward(net, o, xsm, h1, h2, red);
        if (threadIdx.x == 0) out[i] = y * ys + ym;
        __syncthreads();
    }
}
}  // namespace

struct he_mlp {
    u32 F = 0, n_par = 0, t = 0;
    int device = 0;
    float *p = nullptr, *m = nullptr, *v = nullptr, *stats = nullptr, *part = nullptr;  // stats: mean[F+1], std[F+1]
    float ym = 0.f, ys = 1.f;  // host copy of the target's standardisation
    ~he_mlp() {
        cudaFree(p), cudaFree(m), cudaFree(v), cudaFree(stats), cudaFree(part);
    }
    Net net() const { return Net{p, stats, stats + F + 1, F}; }
    void read_target_stats() {
        MLP_CUDA(cudaMemcpy(&ym, stats + F, sizeof(float), cudaMemcpyDeviceToHost));
        MLP_CUDA(cudaMemcpy(&ys, stats + 2 * F + 1, sizeof(float), cudaMemcpyDeviceToHost));
    }
};

static u64 host_splitmix(u64 z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" int he_mlp_create(uint32_t n_features, uint64_t seed, he_mlp** out) {
    return hy::guard([&] {
        if (!out || n_features == 0 || n_features > (u32)FMAX) fail(HE_EINVAL, "1 <= n_features <= 64");
        auto M = std::make_unique<he_mlp>();
        M->F = n_features;
        const Off o(n_features);
        M->n_par = o.n;
        MLP_CUDA(cudaGetDevice(&M->device));
        MLP_CUDA(cudaMalloc(&M->p, o.n * sizeof(float)));
        MLP_CUDA(cudaMalloc(&M->m, o.n * sizeof(float)));
        MLP_CUDA(cudaMalloc(&M->v, o.n * sizeof(float)));
        MLP_CUDA(cudaMalloc(&M->stats, 2 * (n_features + 1) * sizeof(float)));
        MLP_CUDA(cudaMalloc(&M->part, (size_t)GRAD_BLOCKS * (o.n + 1) * sizeof(float)));
        // He-uniform weights (bound sqrt(6 / fan_in)), zero biases; identity standardisation
        std::vector<float> h(o.n, 0.f);
        u64 st = seed;
        auto uni = [&](float bound) {
            st = host_splitmix(st);
            return (float)(((double)(st >> 11) / 9007199254740992.0) * 2.0 - 1.0) * bound;
        };
        for (u32 i = 0; i < H * n_features; i++) h[o.W1 + i] = uni(std::sqrt(6.f / n_features));
        for (u32 i = 0; i < H * H; i++) h[o.W2 + i] = uni(std::sqrt(6.f / H));
        for (u32 i = 0; i < H; i++) h[o.w3 + i] = uni(std::sqrt(6.f / H));
        MLP_CUDA(cudaMemcpy(M->p, h.data(), o.n * sizeof(float), cudaMemcpyHostToDevice));
        MLP_CUDA(cudaMemset(M->m, 0, o.n * sizeof(float)));
        MLP_CUDA(cudaMemset(M->v, 0, o.n * sizeof(float)));
        std::vector<float> s(2 * (n_features + 1), 0.f);
        for (u32 i = 0; i <= n_features; i++) s[n_features + 1 + i] = 1.f;
        MLP_CUDA(cudaMemcpy(M->stats, s.data(), s.size() * sizeof(float), cudaMemcpyHostToDevice));
        *out = M.release();
    });
}

extern "C" int he_mlp_param_count(const he_mlp* m, uint32_t* count) {
    return hy::guard([&] {
        if (!m || !count) fail(HE_EINVAL, "null argument");
        *count = m->n_par + 2 * (m->F + 1);
    });
}

extern "C" int he_mlp_get_params(const he_mlp* m, float* h) {
    return hy::guard([&] {
        if (!m || !h) fail(HE_EINVAL, "null argument");
        MLP_CUDA(cudaMemcpy(h, m->p, m->n_par * sizeof(float), cudaMemcpyDeviceToHost));
        MLP_CUDA(cudaMemcpy(h + m->n_par, m->stats, 2 * (m->F + 1) * sizeof(float), cudaMemcpyDeviceToHost));
    });
}

extern "C" int he_mlp_set_params(he_mlp* m, const float* h) {
    return hy::guard([&] {
        if (!m || !h) fail(HE_EINVAL, "null argument");
        for (u32 i = 0; i <= m->F; i++)
            if (!(h[m->n_par + m->F + 1 + i] > 0.f)) fail(HE_EINVAL, "standard deviations must be positive");
        MLP_CUDA(cudaMemcpy(m->p, h, m->n_par * sizeof(float), cudaMemcpyHostToDevice));
        MLP_CUDA(cudaMemcpy(m->stats, h + m->n_par, 2 * (m->F + 1) * sizeof(float), cudaMemcpyHostToDevice));
        MLP_CUDA(cudaMemset(m->m, 0, m->n_par * sizeof(float)));
        MLP_CUDA(cudaMemset(m->v, 0, m->n_par * sizeof(float)));
        m->t = 0;
        m->read_target_stats();
    });
}

extern "C" int he_mlp_fit_scaling(he_mlp* m, const float* d_X, const float* d_y, uint32_t n, void* stream) {
    return hy::guard([&] {
        if (!m || !d_X || !d_y || n < 2) fail(HE_EINVAL, "bad argument");
        k_colstats<<<m->F + 1, 256, 0, (cudaStream_t)stream>>>(d_X, d_y, n, m->F, m->stats, m->stats + m->F + 1);
        MLP_CUDA(cudaGetLastError());
        MLP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        m->read_target_stats();
    });
}

extern "C" int he_mlp_step(he_mlp* m, const float* d_X, const float* d_y, uint32_t n, uint32_t batch, float lr,
                           uint64_t seed, void* stream, float* loss) {
    return hy::guard([&] {
        if (!m || !d_X || !d_y || !n || !batch) fail(HE_EINVAL, "bad argument");
        cudaStream_t s = (cudaStream_t)stream;
        const u32 blocks = std::min<u32>(GRAD_BLOCKS, batch);
        k_mlp_grad<<<blocks, H, 0, s>>>(m->net(), d_X, d_y, n, m->ym, m->ys, batch, seed, m->t, m->part);
        MLP_CUDA(cudaGetLastError());
        m->t++;
        k_mlp_adam<<<(m->n_par + 255) / 256, 256, 0, s>>>(m->p, m->m, m->v, m->part, m->n_par, blocks, lr, 0.9f,
                                                          0.999f, 1e-8f, m->t);
        MLP_CUDA(cudaGetLastError());
        if (loss) {
            std::vector<float> sse(blocks);
            for (u32 b = 0; b < blocks; b++)
                MLP_CUDA(cudaMemcpyAsync(&sse[b], m->part + (size_t)b * (m->n_par + 1) + m->n_par, sizeof(float),
                                         cudaMemcpyDeviceToHost, s));
            MLP_CUDA(cudaStreamSynchronize(s));
            double t = 0;
            for (float x : sse) t += x;
            *loss = (float)(t / batch);
        }
    });
}

extern "C" int he_mlp_train(he_mlp* m, const float* d_X, const float* d_y, uint32_t n, uint32_t steps,
                            uint32_t batch, float lr, uint64_t seed, void* stream, float* final_loss) {
    return hy::guard([&] {
        if (!m || !d_X || !d_y || n < 2 || !steps || !batch) fail(HE_EINVAL, "bad argument");
        if (he_mlp_fit_scaling(m, d_X, d_y, n, stream) != HE_OK) fail(HE_ECUDA, "feature scaling failed");
        for (u32 i = 0; i < steps; i++) {
            // cosine decay of the step size to a tenth
            const float f = 0.55f + 0.45f * std::cos(3.14159265f * (float)i / (float)steps);
            float* lp = (i + 1 == steps) ? final_loss : nullptr;
            const int rc = he_mlp_step(m, d_X, d_y, n, batch, lr * f, seed, stream, lp);
            if (rc != HE_OK) fail(rc, "training step failed");
        }
    });
}

extern "C" int he_mlp_predict(const he_mlp* m, const float* d_X, uint32_t n, float* d_y, void* stream) {
    return hy::guard([&] {
        if (!m || !d_X || !d_y) fail(HE_EINVAL, "null argument");
        if (!n) return;
        k_mlp_fwd<<<std::min<u32>(n, 4096), H, 0, (cudaStream_t)stream>>>(m->net(), d_X, n, m->ym, m->ys, d_y);
        MLP_CUDA(cudaGetLastError());
    });
}

extern "C" void he_mlp_destroy(he_mlp* m) { delete m; }
