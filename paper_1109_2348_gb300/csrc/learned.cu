// Learned-CDF bucketing (BWT_F_LEARNED) and the model's file and sample
// plumbing.
//
// Model files hold the MLP parameters and the compiled splitter table; the
// plan keeps the splitters on the device. Training samples come from the
// plain sorter: after the plain sort, the row at sorted position k of block
// b holds rotation SA[k], so (8 prefix bytes of SA[k]) / 255 -> (k - off_b) /
// n_b samples the CDF of rotation prefixes.
#include <cstdio>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "plan_internal.h"

using namespace bwt;

#define CKL(call)                                              \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return record_cuda(_e, #call);  \
    } while (0)

static const char kModelTag[8] = {'B', 'W', 'T', 'M', 'D', 'L', '0', '1'};

extern "C" bwt_status bwt_model_save(const char* path, const float* params, const uint64_t* splitters) {
    if (!path || !params || !splitters) return BWT_EINVAL;
    FILE* f = std::fopen(path, "wb");
    if (!f) return BWT_EINVAL;
    bool ok = std::fwrite(kModelTag, 1, 8, f) == 8 &&
              std::fwrite(params, sizeof(float), BWT_MLP_NPARAMS, f) == BWT_MLP_NPARAMS &&
              std::fwrite(splitters, sizeof(uint64_t), BWT_SPLITTERS, f) == BWT_SPLITTERS;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? BWT_OK : BWT_EINVAL;
}

extern "C" bwt_status bwt_model_load(const char* path, float* params, uint64_t* splitters) {
    if (!path || !params || !splitters) return BWT_EINVAL;
    FILE* f = std::fopen(path, "rb");
    if (!f) return BWT_ENOMODEL;
    char tag[8];
    bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, kModelTag, 8) == 0 &&
              std::fread(params, sizeof(float), BWT_MLP_NPARAMS, f) == BWT_MLP_NPARAMS &&
              std::fread(splitters, sizeof(uint64_t), BWT_SPLITTERS, f) == BWT_SPLITTERS;
    std::fclose(f);
    return ok ? BWT_OK : BWT_ENOMODEL;
}

static bwt_status ensure_learned_memory(bwt_plan* p) {
    if (!p->splitters) CKL(cudaMalloc(&p->splitters, sizeof(uint64_t) * BWT_SPLITTERS));
    return BWT_OK;
}

extern "C" bwt_status bwt_plan_set_splitters(bwt_plan* p, const uint64_t* splitters) {
    if (!p || !splitters) return BWT_EINVAL;
    CKL(cudaSetDevice(p->device));
    std::vector<uint64_t> h(BWT_SPLITTERS);
    CKL(cudaMemcpy(h.data(), splitters, sizeof(uint64_t) * BWT_SPLITTERS, cudaMemcpyDefault));
    for (int i = 1; i < BWT_SPLITTERS; ++i)
        if (h[i] < h[i - 1]) return BWT_EINVAL;
    bwt_status s = ensure_learned_memory(p);
    if (s != BWT_OK) return s;
    CKL(cudaMemcpy(p->splitters, h.data(), sizeof(uint64_t) * BWT_SPLITTERS, cudaMemcpyHostToDevice));
    p->have_model = true;
    return BWT_OK;
}

bwt_status bwt::load_model(bwt_plan* p, const char* path) {
    if (!path || !*path) return BWT_ENOMODEL;
    std::vector<float> params(BWT_MLP_NPARAMS);
    std::vector<uint64_t> spl(BWT_SPLITTERS);
    bwt_status s = bwt_model_load(path, params.data(), spl.data());
    if (s != BWT_OK) return s;
    return bwt_plan_set_splitters(p, spl.data());
}

namespace {

__global__ void k_make_samples(const uint8_t* __restrict__ S, const uint32_t* __restrict__ SA,
                               const BlockInfo* __restrict__ blocks, uint32_t nb, const uint64_t* __restrict__ pos,
                               uint32_t count, float* __restrict__ x, float* __restrict__ t) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    const uint32_t k = (uint32_t)pos[s];
    uint32_t lo = 0, hi = nb;  // block b with off <= k < off + n
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (blocks[mid].off <= k) lo = mid; else hi = mid;
    }
    const BlockInfo bi = blocks[lo];
    const uint32_t i = SA[k] < bi.n ? SA[k] : 0u;
    for (int j = 0; j < 8; ++j) {
        uint32_t q = i + j;
        while (q >= bi.n) q -= bi.n;
        x[(size_t)s * 8 + j] = (float)S[bi.off + q] * (1.f / 255.f);
    }
    t[s] = (float)(k - bi.off) / (float)bi.n;
}

}  // namespace

extern "C" bwt_status bwt_model_samples(bwt_plan* p, const uint8_t* d_in, const uint64_t* offsets,
                                        uint32_t num_blocks, const uint64_t* d_pos, uint32_t count, float* d_x,
                                        float* d_t, void* stream) {
    if (!p || !d_in || !offsets || !d_pos || !d_x || !d_t) return BWT_EINVAL;
    CKL(cudaSetDevice(p->device));
    cudaStream_t st = (cudaStream_t)stream;
    std::memset(&p->stats, 0, sizeof(p->stats));
    bwt_status s = prepare_batch(p, offsets, num_blocks, st);
    if (s != BWT_OK) return s;
    if ((s = reset_ctrl(p, st)) != BWT_OK) return s;
    if ((s = enqueue_initial_sort(p, d_in, st)) != BWT_OK) return s;
    if ((s = run_doubling_host_loop(p, st)) != BWT_OK) return s;
    if (count) {
        k_make_samples<<<(count + 255) / 256, 256, 0, st>>>(d_in, p->sa, p->blocks, p->nb, d_pos, count, d_x, d_t);
        CKL(cudaGetLastError());
    }
    return finish_status(p, st);
}

bwt_status bwt::run_learned(bwt_plan* p, const uint8_t* d_in, uint8_t* d_L, int32_t* d_primary, cudaStream_t st) {
    (void)d_in; (void)d_L; (void)d_primary; (void)st;
    if (!p->have_model) return BWT_ENOMODEL;
    return BWT_ENOMODEL;
}
