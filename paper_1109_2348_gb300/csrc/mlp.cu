// The learned CDF model: an FP32 MLP 8 -> 32 -> 32 -> 1 with ReLU, its
// forward pass, MSE loss gradient, Adam step, trainer and the compilation of
// the trained CDF into a sorted table of 4095 bucket splitters.
//
// Input x = the 8 prefix bytes of a rotation / 255; target t = the
// rotation's sorted rank / n, so the network approximates the CDF of 8-byte
// prefixes. Parameter layout (1,377 floats, row-major):
//   W1[32][8] | b1[32] | W2[32][32] | b2[32] | W3[32] | b3
// The loss over a batch is mean((y - t)^2); gradients are reduced in a fixed
// order (per-CTA partial sums, then CTA partials in index order), so runs are
// bit-reproducible. The MLP is FFMA work on CUDA cores: it is off the timed
// sort path (the sort only searches the compiled splitter table).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "bwt.h"
#include "plan_internal.h"

namespace bwt {

namespace {

constexpr int NP = BWT_MLP_NPARAMS;
constexpr int IN = 8, H = 32;
constexpr int OFF_W1 = 0, OFF_B1 = 256, OFF_W2 = 288, OFF_B2 = 1312, OFF_W3 = 1344, OFF_B3 = 1376;
constexpr int GS = 64;  // samples per CTA in the gradient kernel

__device__ __forceinline__ float mlp_eval(const float* __restrict__ P, const float* x, float* h1, float* h2) {
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float a = P[OFF_B1 + j];
#pragma unroll
        for (int i = 0; i < IN; ++i) a = fmaf(P[OFF_W1 + j * IN + i], x[i], a);
        h1[j] = a > 0.f ? a : 0.f;
    }
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float a = P[OFF_B2 + j];
#pragma unroll
        for (int i = 0; i < H; ++i) a = fmaf(P[OFF_W2 + j * H + i], h1[i], a);
        h2[j] = a > 0.f ? a : 0.f;
    }
    float y = P[OFF_B3];
#pragma unroll
    for (int i = 0; i < H; ++i) y = fmaf(P[OFF_W3 + i], h2[i], y);
    return y;
}

__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ params, const float* __restrict__ x,
                                                     uint32_t count, float* __restrict__ y) {
    __shared__ float P[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    float xs[IN], h1[H], h2[H];
#pragma unroll
    for (int i = 0; i < IN; ++i) xs[i] = x[(size_t)s * IN + i];
    y[s] = mlp_eval(P, xs, h1, h2);
}

// Forward + backward of GS samples per CTA; writes the CTA's gradient sum
// (already divided by the batch size B) and its summed squared error.
// Samples are x[idx[first + s]] (or x[first + s] without idx).
__global__ void __launch_bounds__(GS) k_mlp_grad(const float* __restrict__ params, const float* __restrict__ x,
                                                 const float* __restrict__ t, const uint32_t* __restrict__ idx,
                                                 uint32_t first, uint32_t B, float* __restrict__ partial,
                                                 float* __restrict__ loss_partial) {
    __shared__ float P[NP];
    __shared__ float sx[GS][IN];
    __shared__ float sh1[GS][H + 1], sh2[GS][H + 1], sd1[GS][H + 1], sd2[GS][H + 1];
    __shared__ float sdy[GS], serr[GS];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    const int s = threadIdx.x;
    const uint32_t b = blockIdx.x * GS + s;
    float xs[IN], h1[H], h2[H];
    if (b < B) {
        const uint32_t src = idx ? idx[first + b] : first + b;
#pragma unroll
        for (int i = 0; i < IN; ++i) xs[i] = x[(size_t)src * IN + i];
        const float y = mlp_eval(P, xs, h1, h2);
        const float e = y - t[src];
        const float dy = 2.f * e / (float)B;
        serr[s] = e * e;
        sdy[s] = dy;
        float d2[H];
#pragma unroll
        for (int j = 0; j < H; ++j) d2[j] = h2[j] > 0.f ? dy * P[OFF_W3 + j] : 0.f;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            float a = 0.f;
#pragma unroll
            for (int j = 0; j < H; ++j) a = fmaf(P[OFF_W2 + j * H + i], d2[j], a);
            sd1[s][i] = h1[i] > 0.f ? a : 0.f;
            sd2[s][i] = d2[i];
            sh1[s][i] = h1[i];
            sh2[s][i] = h2[i];
        }
#pragma unroll
        for (int i = 0; i < IN; ++i) sx[s][i] = xs[i];
    } else {
        serr[s] = 0.f;
        sdy[s] = 0.f;
        for (int i = 0; i < H; ++i) sd1[s][i] = sd2[s][i] = sh1[s][i] = sh2[s][i] = 0.f;
        for (int i = 0; i < IN; ++i) sx[s][i] = 0.f;
    }
    __syncthreads();
    float* out = partial + (size_t)blockIdx.x * NP;
    for (int e = threadIdx.x; e < NP; e += blockDim.x) {
        float g = 0.f;
        if (e < OFF_B1) {
            const int j = e / IN, i = e % IN;
            for (int q = 0; q < GS; ++q) g = fmaf(sd1[q][j], sx[q][i], g);
        } else if (e < OFF_W2) {
            const int j = e - OFF_B1;
            for (int q = 0; q < GS; ++q) g += sd1[q][j];
        } else if (e < OFF_B2) {
            const int j = (e - OFF_W2) / H, i = (e - OFF_W2) % H;
            for (int q = 0; q < GS; ++q) g = fmaf(sd2[q][j], sh1[q][i], g);
        } else if (e < OFF_W3) {
            const int j = e - OFF_B2;
            for (int q = 0; q < GS; ++q) g += sd2[q][j];
        } else if (e < OFF_B3) {
            const int i = e - OFF_W3;
            for (int q = 0; q < GS; ++q) g = fmaf(sdy[q], sh2[q][i], g);
        } else {
            for (int q = 0; q < GS; ++q) g += sdy[q];
        }
        out[e] = g;
    }
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int q = 0; q < GS; ++q) l += serr[q];
        loss_partial[blockIdx.x] = l;
    }
}

// Sums the CTA partials in index order; optionally writes the gradient and
// the mean loss, and optionally applies one Adam step (Kingma and Ba 2015).
__global__ void k_mlp_reduce(const float* __restrict__ partial, const float* __restrict__ loss_partial, int nblk,
                             uint32_t B, float* __restrict__ grad_out, float* __restrict__ loss_out,
                             float* __restrict__ params, float* __restrict__ m, float* __restrict__ v, int step,
                             float lr, float beta1, float beta2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && loss_out) {
        float l = 0.f;
        for (int b = 0; b < nblk; ++b) l += loss_partial[b];
        *loss_out = l / (float)B;
    }
    if (i >= NP) return;
    float g = 0.f;
    for (int b = 0; b < nblk; ++b) g += partial[(size_t)b * NP + i];
    if (grad_out) grad_out[i] = g;
    if (params && step > 0) {
        const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
        const float mi = beta1 * m[i] + (1.f - beta1) * g;
        const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
        m[i] = mi;
        v[i] = vi;
        params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_adam(float* __restrict__ params, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int step, float lr, float beta1, float beta2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    const float mi = beta1 * m[i] + (1.f - beta1) * g[i];
    const float vi = beta2 * v[i] + (1.f - beta2) * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Bisection over the 64-bit key space, one thread per splitter: splitter j
// is the smallest key x (to 64-bit precision) with F(x) >= (j + 1) / 4096,
// where F = the MLP evaluated on x's 8 bytes mapped through norm. F need not
// be monotone; the table is sorted afterwards, and any sorted table gives
// exact results.
__global__ void __launch_bounds__(128) k_compile_splitters(const float* __restrict__ params,
                                                           const float* __restrict__ norm,
                                                           uint64_t* __restrict__ spl, uint32_t count) {
    __shared__ float P[NP];
    __shared__ float nrm[256];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) P[i] = params[i];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) nrm[i] = norm[i];
    __syncthreads();
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    const float q = (float)(j + 1) / (float)(count + 1);
    uint64_t lo = 0, hi = ~0ull;  // invariant: F(hi) >= q is assumed at the top end
    float h1[H], h2[H], xs[IN];
    for (int it = 0; it < 64 && lo < hi; ++it) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
#pragma unroll
        for (int b = 0; b < IN; ++b) xs[b] = nrm[(mid >> (56 - 8 * b)) & 0xff];
        const float f = mlp_eval(P, xs, h1, h2);
        if (f >= q) hi = mid; else lo = mid + 1;
    }
    spl[j] = hi;
}

// Sorts the table in place (count <= 4096, one CTA, bitonic in shared memory),
// then spreads every run of equal splitters evenly over the key interval up
// to the next distinct splitter. Equal splitters come from a model that is
// flat across an interval and jumps at its end (the model reads the key as
// eight separate bytes, so it jumps at byte boundaries of the key): the run's
// share of the distribution lies in that interval, and even spacing there is
// the linear reading of the model's CDF across it. The table stays sorted.
__global__ void __launch_bounds__(1024) k_sort_splitters(uint64_t* __restrict__ spl, uint32_t count) {
    __shared__ uint64_t a[4096];
    for (uint32_t i = threadIdx.x; i < 4096; i += blockDim.x) a[i] = i < count ? spl[i] : ~0ull;
    __syncthreads();
    for (uint32_t k = 2; k <= 4096; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < 4096; i += blockDim.x) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t x = a[i], y = a[ixj];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        a[i] = y;
                        a[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) {
        uint32_t i = 0;
        while (i < count) {
            uint32_t j = i;
            while (j + 1 < count && a[j + 1] == a[i]) ++j;
            const uint32_t c = j - i + 1;
            if (c > 1) {
                const uint64_t base = a[i];
                const uint64_t next = j + 1 < count ? a[j + 1] : ~0ull;
                const unsigned __int128 span = (unsigned __int128)(next - base);
                for (uint32_t r = 1; r < c; ++r) a[i + r] = base + (uint64_t)(span * r / c);
            }
            i = j + 1;
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) spl[i] = a[i];
}

struct MlpScratch {
    float* partial = nullptr;
    float* loss_partial = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    uint32_t cap_blocks = 0;
};

bwt_status ensure_scratch(MlpScratch& s, uint32_t nblk) {
    if (s.cap_blocks >= nblk) return BWT_OK;
    if (s.partial) cudaFree(s.partial);
    if (s.loss_partial) cudaFree(s.loss_partial);
    s.partial = nullptr;
    s.loss_partial = nullptr;
    if (cudaMalloc(&s.partial, sizeof(float) * NP * nblk) != cudaSuccess ||
        cudaMalloc(&s.loss_partial, sizeof(float) * nblk) != cudaSuccess) {
        cudaGetLastError();
        s.cap_blocks = 0;
        return BWT_ENOMEM;
    }
    s.cap_blocks = nblk;
    return BWT_OK;
}

void free_scratch(MlpScratch& s) {
    if (s.partial) cudaFree(s.partial);
    if (s.loss_partial) cudaFree(s.loss_partial);
    if (s.m) cudaFree(s.m);
    if (s.v) cudaFree(s.v);
    s = MlpScratch();
}

}  // namespace

}  // namespace bwt

using namespace bwt;

#define CKM(call)                                               \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return record_cuda(_e, #call);   \
    } while (0)

extern "C" bwt_status bwt_mlp_forward(const float* d_params, const float* d_x, uint32_t count, float* d_y,
                                      void* stream) {
    if (!d_params || (!d_x && count) || (!d_y && count)) return BWT_EINVAL;
    bwt::NvtxRange nvtx_range("mlp_forward");
    if (!count) return BWT_OK;
    k_mlp_forward<<<(count + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d_params, d_x, count, d_y);
    CKM(cudaGetLastError());
    return BWT_OK;
}

extern "C" bwt_status bwt_mlp_loss_grad(const float* d_params, const float* d_x, const float* d_t, uint32_t count,
                                        float* d_grad, float* d_loss, void* stream) {
    if (!d_params || !d_x || !d_t || !d_grad || count == 0) return BWT_EINVAL;
    bwt::NvtxRange nvtx_range("mlp_loss_grad");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t nblk = (count + GS - 1) / GS;
    MlpScratch s;
    bwt_status r = ensure_scratch(s, nblk);
    if (r != BWT_OK) return r;
    k_mlp_grad<<<nblk, GS, 0, st>>>(d_params, d_x, d_t, nullptr, 0, count, s.partial, s.loss_partial);
    k_mlp_reduce<<<(NP + 255) / 256, 256, 0, st>>>(s.partial, s.loss_partial, (int)nblk, count, d_grad, d_loss,
                                                   nullptr, nullptr, nullptr, 0, 0.f, 0.f, 0.f, 0.f);
    cudaError_t e = cudaGetLastError();
    cudaStreamSynchronize(st);
    free_scratch(s);
    CKM(e);
    return BWT_OK;
}

extern "C" bwt_status bwt_mlp_adam_step(float* d_params, const float* d_grad, float* d_m, float* d_v, uint32_t step,
                                        float lr, void* stream) {
    if (!d_params || !d_grad || !d_m || !d_v || step == 0) return BWT_EINVAL;
    bwt::NvtxRange nvtx_range("mlp_adam");
    k_adam<<<(NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_params, d_grad, d_m, d_v, (int)step, lr, 0.9f,
                                                               0.999f, 1e-8f);
    CKM(cudaGetLastError());
    return BWT_OK;
}

extern "C" bwt_status bwt_model_train(float* d_params, const float* d_x, const float* d_t, uint32_t count,
                                      const uint32_t* d_order, uint32_t epochs, uint32_t batch, float lr,
                                      float* d_epoch_loss, void* stream) {
    if (!d_params || !d_x || !d_t || !d_order || count == 0 || batch == 0 || epochs == 0) return BWT_EINVAL;
    bwt::NvtxRange nvtx_range("mlp_train");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t nblk = (batch + GS - 1) / GS;
    MlpScratch s;
    bwt_status r = ensure_scratch(s, nblk);
    if (r != BWT_OK) return r;
    float* batch_loss = nullptr;
    const uint32_t steps_per_epoch = (count + batch - 1) / batch;
    if (cudaMalloc(&s.m, sizeof(float) * NP) != cudaSuccess || cudaMalloc(&s.v, sizeof(float) * NP) != cudaSuccess ||
        cudaMalloc(&batch_loss, sizeof(float) * steps_per_epoch) != cudaSuccess) {
        cudaGetLastError();
        free_scratch(s);
        if (batch_loss) cudaFree(batch_loss);
        return BWT_ENOMEM;
    }
    cudaMemsetAsync(s.m, 0, sizeof(float) * NP, st);
    cudaMemsetAsync(s.v, 0, sizeof(float) * NP, st);
    int step = 0;
    std::vector<float> h_loss(steps_per_epoch);
    cudaError_t e = cudaSuccess;
    for (uint32_t ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        const uint32_t* order = d_order + (size_t)ep * count;
        for (uint32_t b0 = 0; b0 < count; b0 += batch) {
            const uint32_t B = std::min(batch, count - b0);
            const uint32_t nb = (B + GS - 1) / GS;
            ++step;
            k_mlp_grad<<<nb, GS, 0, st>>>(d_params, d_x, d_t, order, b0, B, s.partial, s.loss_partial);
            k_mlp_reduce<<<(NP + 255) / 256, 256, 0, st>>>(s.partial, s.loss_partial, (int)nb, B, nullptr,
                                                           batch_loss + b0 / batch, d_params, s.m, s.v, step, lr,
                                                           0.9f, 0.999f, 1e-8f);
        }
        e = cudaGetLastError();
        if (d_epoch_loss && e == cudaSuccess) {
            // mean of the epoch's batch losses, computed on the host from a copy
            e = cudaMemcpyAsync(h_loss.data(), batch_loss, sizeof(float) * steps_per_epoch, cudaMemcpyDeviceToHost,
                                st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            double acc = 0;
            for (float v : h_loss) acc += v;
            const float mean = (float)(acc / steps_per_epoch);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_epoch_loss + ep, &mean, sizeof(float), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
    }
    cudaStreamSynchronize(st);
    cudaFree(batch_loss);
    free_scratch(s);
    CKM(e);
    return BWT_OK;
}

extern "C" bwt_status bwt_model_compile(const float* d_params, const float* d_norm, uint64_t* d_splitters,
                                        void* stream) {
    if (!d_params || !d_norm || !d_splitters) return BWT_EINVAL;
    bwt::NvtxRange nvtx_range("mlp_compile");
    cudaStream_t st = (cudaStream_t)stream;
    k_compile_splitters<<<(BWT_SPLITTERS + 127) / 128, 128, 0, st>>>(d_params, d_norm, d_splitters, BWT_SPLITTERS);
    k_sort_splitters<<<1, 1024, 0, st>>>(d_splitters, BWT_SPLITTERS);
    CKM(cudaGetLastError());
    return BWT_OK;
}
