// Learned SC/PC mode selector: an MLP 8 -> 32 -> 32 -> 1 (ReLU, FP32) that
// predicts y = log(t_PC / t_SC) for one partition in one iteration and stands
// in for the traffic model of Sec. 3.2 (the paper has no learned selector).
// Training is full-batch Adam on the mean squared error, with the library's
// own forward/backward/reduction/update kernels; every reduction runs in a
// fixed order, so training is deterministic for a given input and seed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "gpop_internal.cuh"

namespace gpop {

namespace {

constexpr int F = GPOP_SELECTOR_FEATURES;  // 8
constexpr int H = GPOP_SELECTOR_HIDDEN;    // 32
constexpr int NW = GPOP_SELECTOR_WEIGHTS;  // 1377
constexpr int NP = GPOP_SELECTOR_PARAMS;   // weights + mean, std, fmin, fmax
constexpr int S = 64;                      // samples per gradient block (static smem < 48 KB)
constexpr int T = 256;                     // threads per gradient block

// offsets of the parameter groups in the flat layout W1[32][8] b1 W2[32][32] b2 W3[32] b3
constexpr int oW1 = 0, ob1 = oW1 + H * F, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + H;
static_assert(ob3 + 1 == NW, "selector layout");

std::mutex g_mu;
float *g_dparams = nullptr;    // installed parameters (device), NP floats
float *g_dparams_t = nullptr;  // the same with W1 and W2 transposed (engine inference)

// Forward pass, loss gradient and parameter gradients for samples
// [blockIdx.x*S, +S); writes this block's gradient sums to part[blockIdx.x].
__global__ void __launch_bounds__(T) k_mlp_grad(const float *__restrict__ w, const float *__restrict__ x,
                                                const float *__restrict__ y, uint32_t n, float inv_n,
                                                float *__restrict__ part, float *__restrict__ loss_part,
                                                float *__restrict__ pred) {
    __shared__ float sw[NW];
    __shared__ float sx[S][F];
    __shared__ float h1[S][H], h2[S][H], d1[S][H], d2[S][H];
    __shared__ float e[S], sq[S];
    const uint32_t s0 = blockIdx.x * S;
    for (int i = threadIdx.x; i < NW; i += T) sw[i] = w[i];
    for (int i = threadIdx.x; i < S * F; i += T) {
        uint32_t s = s0 + i / F;
        sx[i / F][i % F] = s < n ? x[(uint64_t)s * F + i % F] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < S * H; i += T) {  // layer 1
        int s = i / H, j = i % H;
        float a = sw[ob1 + j];
        for (int k = 0; k < F; ++k) a = fmaf(sw[oW1 + j * F + k], sx[s][k], a);
        h1[s][j] = fmaxf(a, 0.f);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < S * H; i += T) {  // layer 2
        int s = i / H, j = i % H;
        float a = sw[ob2 + j];
        for (int k = 0; k < H; ++k) a = fmaf(sw[oW2 + j * H + k], h1[s][k], a);
        h2[s][j] = fmaxf(a, 0.f);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < S; s += T) {  // output and dL/dy_hat of the mean squared error
        float a = sw[ob3];
        for (int k = 0; k < H; ++k) a = fmaf(sw[oW3 + k], h2[s][k], a);
        bool ok = s0 + s < n;
        float r = ok ? a - y[s0 + s] : 0.f;
        e[s] = 2.f * r * inv_n;
        sq[s] = r * r * inv_n;
        if (ok && pred) pred[s0 + s] = a;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < S * H; i += T) {  // back through layer 3
        int s = i / H, j = i % H;
        d2[s][j] = h2[s][j] > 0.f ? e[s] * sw[oW3 + j] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < S * H; i += T) {  // back through layer 2
        int s = i / H, k = i % H;
        float a = 0.f;
        for (int j = 0; j < H; ++j) a = fmaf(d2[s][j], sw[oW2 + j * H + k], a);
        d1[s][k] = h1[s][k] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // parameter gradients, each a sum over the block's samples in index order
    float *out = part + (uint64_t)blockIdx.x * NW;
    for (int pi = threadIdx.x; pi < NW; pi += T) {
        float g = 0.f;
        if (pi < ob1) {
            int j = pi / F, k = pi % F;
            for (int s = 0; s < S; ++s) g = fmaf(d1[s][j], sx[s][k], g);
        } else if (pi < oW2) {
            int j = pi - ob1;
            for (int s = 0; s < S; ++s) g += d1[s][j];
        } else if (pi < ob2) {
            int j = (pi - oW2) / H, k = (pi - oW2) % H;
            for (int s = 0; s < S; ++s) g = fmaf(d2[s][j], h1[s][k], g);
        } else if (pi < oW3) {
            int j = pi - ob2;
            for (int s = 0; s < S; ++s) g += d2[s][j];
        } else if (pi < ob3) {
            int j = pi - oW3;
            for (int s = 0; s < S; ++s) g = fmaf(e[s], h2[s][j], g);
        } else {
            for (int s = 0; s < S; ++s) g += e[s];
        }
        out[pi] = g;
    }
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int s = 0; s < S; ++s) l += sq[s];
        loss_part[blockIdx.x] = l;
    }
}

// sums the per-block gradients (and loss) in block order
__global__ void k_mlp_reduce(const float *part, const float *loss_part, uint32_t nblk, float *grad, float *loss) {
    for (int pi = blockIdx.x * blockDim.x + threadIdx.x; pi <= NW; pi += gridDim.x * blockDim.x) {
        float g = 0.f;
        if (pi < NW) {
            for (uint32_t b = 0; b < nblk; ++b) g += part[(uint64_t)b * NW + pi];
            grad[pi] = g;
        } else {
            for (uint32_t b = 0; b < nblk; ++b) g += loss_part[b];
            *loss = g;
        }
    }
}

// Adam (Kingma & Ba 2015) with bias correction
__global__ void k_adam(float *w, const float *grad, float *m, float *v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NW; i += gridDim.x * blockDim.x) {
        float g = grad[i];
        float mi = b1 * m[i] + (1.f - b1) * g;
        float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

uint64_t sm64(uint64_t seed, uint64_t n) {  // splitmix64, counter form
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

struct DevBuf {
    std::vector<void *> p;
    template <typename Tp>
    cudaError_t alloc(Tp **q, size_t n) {
        cudaError_t e = cudaMalloc((void **)q, sizeof(Tp) * (n ? n : 1));
        if (e == cudaSuccess) p.push_back(*q);
        return e;
    }
    ~DevBuf() {
        for (void *q : p) cudaFree(q);
    }
};

}  // namespace

const float *selector_device_params() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_dparams;
}

const float *selector_device_params_transposed() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_dparams_t;
}

}  // namespace gpop

using namespace gpop;

extern "C" gpop_status gpop_selector_set(const float *params) {
    set_error("");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!params) {
        if (g_dparams) cudaFree(g_dparams);
        if (g_dparams_t) cudaFree(g_dparams_t);
        g_dparams = g_dparams_t = nullptr;
        return GPOP_OK;
    }
    for (int i = 0; i < NP; ++i)
        if (!std::isfinite(params[i])) return fail(GPOP_ERR_INVALID_ARG, "selector parameters must be finite");
    for (int i = 0; i < F; ++i)
        if (!(params[NW + F + i] > 0.f)) return fail(GPOP_ERR_INVALID_ARG, "feature std must be positive");
    // the engine's inference reads W1 [H][F] and W2 [H][H] column by column (lane j = hidden unit j), so it
    // gets a copy with both matrices transposed; gpop_selector_get returns the layout that was set
    std::vector<float> t(params, params + NP);
    for (int j = 0; j < H; ++j) {
        for (int i = 0; i < F; ++i) t[i * H + j] = params[j * F + i];
        for (int i = 0; i < H; ++i) t[H * F + H + i * H + j] = params[H * F + H + j * H + i];
    }
    if (!g_dparams) GPOP_CUDA_TRY(cudaMalloc((void **)&g_dparams, sizeof(float) * NP));
    if (!g_dparams_t) GPOP_CUDA_TRY(cudaMalloc((void **)&g_dparams_t, sizeof(float) * NP));
    GPOP_CUDA_TRY(cudaMemcpy(g_dparams, params, sizeof(float) * NP, cudaMemcpyHostToDevice));
    GPOP_CUDA_TRY(cudaMemcpy(g_dparams_t, t.data(), sizeof(float) * NP, cudaMemcpyHostToDevice));
    return GPOP_OK;
}

extern "C" gpop_status gpop_selector_get(float *params) {
    set_error("");
    if (!params) return fail(GPOP_ERR_INVALID_ARG, "params is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dparams) return fail(GPOP_ERR_NO_SELECTOR, "no selector installed");
    GPOP_CUDA_TRY(cudaMemcpy(params, g_dparams, sizeof(float) * NP, cudaMemcpyDeviceToHost));
    return GPOP_OK;
}

extern "C" gpop_status gpop_selector_grad(const float *params, const float *x, const float *y, uint32_t n,
                                         void *cuda_stream, float *pred_out, float *grad_out, float *loss_out) {
    set_error("");
    if (!params || !x || !y || n == 0 || !grad_out) return fail(GPOP_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint32_t nblk = (n + S - 1) / S;
    DevBuf b;
    float *dw, *dx, *dy, *dpart, *dlp, *dg, *dl, *dpred;
    GPOP_CUDA_TRY(b.alloc(&dw, NW));
    GPOP_CUDA_TRY(b.alloc(&dx, (size_t)n * F));
    GPOP_CUDA_TRY(b.alloc(&dy, n));
    GPOP_CUDA_TRY(b.alloc(&dpart, (size_t)nblk * NW));
    GPOP_CUDA_TRY(b.alloc(&dlp, nblk));
    GPOP_CUDA_TRY(b.alloc(&dg, NW));
    GPOP_CUDA_TRY(b.alloc(&dl, 1));
    GPOP_CUDA_TRY(b.alloc(&dpred, n));
    GPOP_CUDA_TRY(cudaMemcpyAsync(dw, params, sizeof(float) * NW, cudaMemcpyHostToDevice, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(dx, x, sizeof(float) * n * F, cudaMemcpyHostToDevice, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(dy, y, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    k_mlp_grad<<<nblk, T, 0, s>>>(dw, dx, dy, n, 1.f / (float)n, dpart, dlp, dpred);
    k_mlp_reduce<<<(NW + 256) / 256, 256, 0, s>>>(dpart, dlp, nblk, dg, dl);
    GPOP_CUDA_TRY(cudaGetLastError());
    GPOP_CUDA_TRY(cudaMemcpyAsync(grad_out, dg, sizeof(float) * NW, cudaMemcpyDeviceToHost, s));
    if (pred_out) GPOP_CUDA_TRY(cudaMemcpyAsync(pred_out, dpred, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    float l = 0.f;
    GPOP_CUDA_TRY(cudaMemcpyAsync(&l, dl, sizeof(float), cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    if (loss_out) *loss_out = l;
    return GPOP_OK;
}

extern "C" gpop_status gpop_selector_train(const float *features, const float *targets, uint32_t n, uint32_t epochs,
                                          float lr, uint64_t seed, void *cuda_stream, float *params_out,
                                          float *loss_out) {
    set_error("");
    if (!features || !targets || n < 2 || !params_out || !(lr > 0.f)) return fail(GPOP_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // feature statistics (host, FP64) and standardisation
    std::vector<double> mean(F, 0.0), var(F, 0.0);
    std::vector<float> fmin(F, INFINITY), fmax(F, -INFINITY);
    for (uint32_t i = 0; i < n; ++i)
        for (int k = 0; k < F; ++k) {
            float v = features[(size_t)i * F + k];
            if (!std::isfinite(v)) return fail(GPOP_ERR_INVALID_ARG, "non-finite feature");
            mean[k] += v;
            fmin[k] = std::min(fmin[k], v);
            fmax[k] = std::max(fmax[k], v);
        }
    for (int k = 0; k < F; ++k) mean[k] /= n;
    for (uint32_t i = 0; i < n; ++i)
        for (int k = 0; k < F; ++k) {
            double d = features[(size_t)i * F + k] - mean[k];
            var[k] += d * d;
        }
    std::vector<float> sd(F), xs((size_t)n * F);
    for (int k = 0; k < F; ++k) sd[k] = (float)std::max(std::sqrt(var[k] / n), 1e-6);
    for (uint32_t i = 0; i < n; ++i)
        for (int k = 0; k < F; ++k)
            xs[(size_t)i * F + k] = (float)((features[(size_t)i * F + k] - mean[k]) / sd[k]);
    // Glorot-uniform initial weights from a splitmix64 stream, zero biases
    std::vector<float> w(NW, 0.f);
    auto init = [&](int off, int fan_out, int fan_in) {
        float a = std::sqrt(6.f / (float)(fan_in + fan_out));
        for (int i = 0; i < fan_out * fan_in; ++i) {
            double u = (double)(sm64(seed, (uint64_t)(off + i)) >> 11) * (1.0 / 9007199254740992.0);
            w[off + i] = (float)((2.0 * u - 1.0) * a);
        }
    };
    init(oW1, H, F);
    init(oW2, H, H);
    init(oW3, 1, H);
    uint32_t nblk = (n + S - 1) / S;
    DevBuf b;
    float *dw, *dx, *dy, *dpart, *dlp, *dg, *dl, *dm, *dv;
    GPOP_CUDA_TRY(b.alloc(&dw, NW));
    GPOP_CUDA_TRY(b.alloc(&dx, (size_t)n * F));
    GPOP_CUDA_TRY(b.alloc(&dy, n));
    GPOP_CUDA_TRY(b.alloc(&dpart, (size_t)nblk * NW));
    GPOP_CUDA_TRY(b.alloc(&dlp, nblk));
    GPOP_CUDA_TRY(b.alloc(&dg, NW));
    GPOP_CUDA_TRY(b.alloc(&dl, 1));
    GPOP_CUDA_TRY(b.alloc(&dm, NW));
    GPOP_CUDA_TRY(b.alloc(&dv, NW));
    GPOP_CUDA_TRY(cudaMemcpyAsync(dw, w.data(), sizeof(float) * NW, cudaMemcpyHostToDevice, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(dx, xs.data(), sizeof(float) * n * F, cudaMemcpyHostToDevice, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(dy, targets, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    GPOP_CUDA_TRY(cudaMemsetAsync(dm, 0, sizeof(float) * NW, s));
    GPOP_CUDA_TRY(cudaMemsetAsync(dv, 0, sizeof(float) * NW, s));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double p1 = 1.0, p2 = 1.0;
    for (uint32_t ep = 0; ep < epochs; ++ep) {
        k_mlp_grad<<<nblk, T, 0, s>>>(dw, dx, dy, n, 1.f / (float)n, dpart, dlp, nullptr);
        k_mlp_reduce<<<(NW + 256) / 256, 256, 0, s>>>(dpart, dlp, nblk, dg, dl);
        p1 *= b1;
        p2 *= b2;
        k_adam<<<(NW + 255) / 256, 256, 0, s>>>(dw, dg, dm, dv, lr, b1, b2, eps, (float)(1.0 - p1), (float)(1.0 - p2));
    }
    // final loss at the trained weights
    k_mlp_grad<<<nblk, T, 0, s>>>(dw, dx, dy, n, 1.f / (float)n, dpart, dlp, nullptr);
    k_mlp_reduce<<<(NW + 256) / 256, 256, 0, s>>>(dpart, dlp, nblk, dg, dl);
    GPOP_CUDA_TRY(cudaGetLastError());
    float l = 0.f;
    GPOP_CUDA_TRY(cudaMemcpyAsync(params_out, dw, sizeof(float) * NW, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(&l, dl, sizeof(float), cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k < F; ++k) {
        params_out[NW + k] = (float)mean[k];
        params_out[NW + F + k] = sd[k];
        params_out[NW + 2 * F + k] = fmin[k];
        params_out[NW + 3 * F + k] = fmax[k];
    }
    if (loss_out) *loss_out = l;
    return GPOP_OK;
}

// --- allocation-free variant of gpop_selector_grad ---------------------------------------------
//
// For callers that must not allocate device memory: code that runs while a stream is being captured
// into a CUDA graph (an allocation there would break or be baked into the capture), code whose device
// memory is owned by another allocator (a framework's caching allocator, a fixed pre-sized arena), and
// latency-critical loops where cudaMalloc/cudaFree would synchronise the device.  The caller passes
// device buffers for every input and output; the per-block partial gradients live in the fixed array
// below, which every GPU that loads this library keeps until the process exits.

namespace gpop {
namespace {

constexpr uint32_t kNoAllocMaxSamples = 16384;             // largest n accepted
constexpr uint32_t kNoAllocMaxBlocks = kNoAllocMaxSamples / S;
// per-block gradient sums (kNoAllocMaxBlocks x NW), per-block loss sums, one spare loss slot
constexpr size_t kNoAllocFloats = (size_t)kNoAllocMaxBlocks * NW + kNoAllocMaxBlocks + 1;
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

std::mutex g_noalloc_mu;
float *g_noalloc_addr[256] = {};  // device address of g_noalloc_scratch per device ordinal

}  // namespace
}  // namespace gpop

extern "C" gpop_status gpop_selector_grad_noalloc(const float *params, const float *x, const float *y, uint32_t n,
                                                 void *cuda_stream, float *pred_out, float *grad_out,
                                                 float *loss_out) {
    set_error("");
    if (!params || !x || !y || !grad_out) return fail(GPOP_ERR_INVALID_ARG, "params, x, y and grad_out must be device pointers");
    if (n == 0 || n > kNoAllocMaxSamples)
        return fail(GPOP_ERR_INVALID_ARG, "gpop_selector_grad_noalloc: n must be in [1, 16384] (fixed scratch size)");
    int dev = 0;
    GPOP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(GPOP_ERR_INVALID_ARG, "device ordinal out of range");
    float *scratch;
    {
        // one-time set-up per device, with that device current: the host-side name of the array is
        // not a device address, so ask the runtime for the address this device uses
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *addr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (e != cudaSuccess || !addr)
                return fail(GPOP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_noalloc_addr[dev] = static_cast<float *>(addr);
        }
        scratch = g_noalloc_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const uint32_t nblk = (n + S - 1) / S;
    float *part = scratch;
    float *loss_part = scratch + (size_t)kNoAllocMaxBlocks * NW;
    float *loss = loss_out ? loss_out : loss_part + kNoAllocMaxBlocks;
    // every slot the reduction reads is written by k_mlp_grad first, so nothing needs clearing
    k_mlp_grad<<<nblk, T, 0, s>>>(params, x, y, n, 1.f / (float)n, part, loss_part, pred_out);
    k_mlp_reduce<<<(NW + 256) / 256, 256, 0, s>>>(part, loss_part, nblk, grad_out, loss);
    GPOP_CUDA_TRY(cudaGetLastError());
    return GPOP_OK;
}
