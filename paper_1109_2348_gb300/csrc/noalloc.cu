// bwt_forward_block_noalloc: forward BWT of one small block without any
// device allocation.
//
// Some callers cannot allocate device memory: a host framework that owns the
// whole GPU through its own memory pool and forbids allocations outside it,
// or a latency-bound pipeline that cannot afford the implicit device
// synchronisation of cudaMalloc / cudaFree. Such a caller cannot create a
// bwt_plan (a plan allocates its scratch). This entry point needs only the
// caller's input and output buffers: its scratch is a file-scope
// __device__ array of fixed size, loaded with the library, which every GPU
// that loads the library keeps until the process exits.
//
// One CTA sorts the block by prefix doubling: rank_1[i] = S[i]; a round
// with shift h sorts all rotations by (rank_h[i], rank_h[(i + h) mod n]) with
// four stable 8-bit LSD passes (rotations enter each round in index order, so
// identical rotations stay lower-index-first), then renames every rotation to
// the sorted position of the first member of its group. It stops when all
// ranks differ or 2h >= n. Ranks stay below 2^16, so a round's key is one
// u32 and the block size is capped at BWT_NOALLOC_MAX_BYTES.
//
// Every scratch word a call reads was written earlier in the same call, so
// nothing has to be cleared between calls. Calls share the one array: two
// calls whose kernels overlap on the GPU (different streams, or different
// host threads on one device) race and corrupt each other's results.
#include <cstdint>

#include "bwt.h"
#include "plan_internal.h"

namespace {

constexpr uint32_t NA_MAX = BWT_NOALLOC_MAX_BYTES;
constexpr int NA_THREADS = 1024;
constexpr int NA_WARPS = NA_THREADS / 32;
constexpr int NA_WORDS = 5 * NA_MAX;  // rank, keys x2, values x2

static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

__device__ __forceinline__ uint32_t na_lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Block-wide inclusive max-scan of one value per thread; returns the scan
// and writes the block maximum to *total.
__device__ __forceinline__ uint32_t na_block_max_scan(uint32_t v, uint32_t* tmp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = max(x, y);
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = tmp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w = max(w, y);
        }
        tmp[lane] = w;
    }
    __syncthreads();
    const uint32_t r = warp > 0 ? max(tmp[warp - 1], x) : x;
    *total = tmp[NA_WARPS - 1];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(NA_THREADS, 1) k_bwt_block_noalloc(const uint8_t* __restrict__ S, uint32_t n,
                                                                     uint8_t* __restrict__ L,
                                                                     int32_t* __restrict__ primary,
                                                                     uint32_t* __restrict__ scratch) {
    __shared__ uint16_t whist[NA_WARPS][256];
    __shared__ uint32_t base[256], chunk_cnt[256], tmp[32];
    __shared__ uint32_t s_distinct;
    uint32_t* rank = scratch;
    uint32_t* kbuf[2] = {scratch + NA_MAX, scratch + 3 * NA_MAX};
    uint32_t* vbuf[2] = {scratch + 2 * NA_MAX, scratch + 4 * NA_MAX};
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = na_lanemask_lt();

    for (uint32_t i = tid; i < n; i += NA_THREADS) rank[i] = S[i];
    __syncthreads();
    uint32_t h = 1;
    for (int round = 0; round < 32; ++round) {
        for (uint32_t i = tid; i < n; i += NA_THREADS) {
            uint32_t j = i + h;
            while (j >= n) j -= n;
            kbuf[0][i] = (rank[i] << 16) | rank[j];
            vbuf[0][i] = i;
        }
        __syncthreads();
        // four stable LSD passes of 8 bits: buffer 0 -> 1 -> 0 -> 1 -> 0
        for (int pass = 0; pass < 4; ++pass) {
            const int shift = 8 * pass;
            const uint32_t* sk = kbuf[pass & 1];
            const uint32_t* sv = vbuf[pass & 1];
            uint32_t* dk = kbuf[(pass + 1) & 1];
            uint32_t* dv = vbuf[(pass + 1) & 1];
            if (tid < 256) base[tid] = 0;
            __syncthreads();
            for (uint32_t c0 = 0; c0 < n; c0 += NA_THREADS) {
                const uint32_t i = c0 + tid;
                const uint32_t d = i < n ? (sk[i] >> shift) & 255u : 256u;
                const uint32_t peers = bwt::match_label<9>(d);
                if (d < 256u && lane == __ffs(peers) - 1) atomicAdd(&base[d], (uint32_t)__popc(peers));
            }
            __syncthreads();
            if (warp == 0) {  // exclusive scan of the 256 digit counts
                uint32_t v[8], s = 0;
                for (int q = 0; q < 8; ++q) {
                    v[q] = base[lane * 8 + q];
                    s += v[q];
                }
                uint32_t x = s;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                uint32_t ex = x - s;
                for (int q = 0; q < 8; ++q) {
                    base[lane * 8 + q] = ex;
                    ex += v[q];
                }
            }
            __syncthreads();
            for (uint32_t c0 = 0; c0 < n; c0 += NA_THREADS) {
                for (int q = tid; q < NA_WARPS * 256 / 2; q += NA_THREADS) reinterpret_cast<uint32_t*>(whist)[q] = 0u;
                __syncthreads();
                const uint32_t i = c0 + tid;
                const bool valid = i < n;
                const uint32_t key = valid ? sk[i] : 0u;
                const uint32_t val = valid ? sv[i] : 0u;
                const uint32_t d = valid ? (key >> shift) & 255u : 256u;
                const uint32_t peers = bwt::match_label<9>(d);
                const uint32_t below = __popc(peers & lt);
                if (valid && lane == __ffs(peers) - 1) whist[warp][d] = (uint16_t)__popc(peers);
                __syncthreads();
                if (tid < 256) {  // prefix over warps, chunk total per digit
                    uint32_t s = 0;
                    for (int w = 0; w < NA_WARPS; ++w) {
                        const uint32_t c = whist[w][tid];
                        whist[w][tid] = (uint16_t)s;
                        s += c;
                    }
                    chunk_cnt[tid] = s;
                }
                __syncthreads();
                if (valid) {
                    const uint32_t pos = base[d] + whist[warp][d] + below;
                    dk[pos] = key;
                    dv[pos] = val;
                }
                __syncthreads();
                if (tid < 256) base[tid] += chunk_cnt[tid];
                __syncthreads();
            }
        }
        // rename: rank of a rotation = sorted position of its group's head
        if (tid == 0) s_distinct = 0;
        __syncthreads();
        uint32_t carry = 0;
        const uint32_t* K = kbuf[0];
        const uint32_t* SA = vbuf[0];
        for (uint32_t c0 = 0; c0 < n; c0 += NA_THREADS) {
            const uint32_t k = c0 + tid;
            const bool valid = k < n;
            const bool head = valid && (k == 0 || K[k] != K[k - 1]);
            uint32_t cmax;
            const uint32_t gs = max(carry, na_block_max_scan(head ? k : 0u, tmp, &cmax));
            if (valid) rank[SA[k]] = gs;
            const uint32_t heads = __syncthreads_count(head);
            if (tid == 0) s_distinct += heads;
            carry = max(carry, cmax);
        }
        __syncthreads();
        const bool done = s_distinct == n || 2 * h >= n;
        __syncthreads();
        if (done) break;
        h *= 2;
    }
    for (uint32_t k = tid; k < n; k += NA_THREADS) {
        const uint32_t sa = vbuf[0][k];
        L[k] = S[sa == 0 ? n - 1 : sa - 1];
        if (sa == 0) *primary = (int32_t)k;
    }
}

// Device address of the scratch array on the current device. The host-side
// symbol is only a stand-in for it, and the address belongs to the module
// loaded in the current context, so it is looked up on every call (a host-side
// query once the module is loaded): a cached address would go stale after
// cudaDeviceReset or in a new primary context.
bwt_status noalloc_scratch(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return bwt::record_cuda(e, "cudaGetSymbolAddress");
    *out = p;
    return BWT_OK;
}

// [a, a + na) and [b, b + nb) share a byte.
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

}  // namespace

extern "C" bwt_status bwt_forward_block_noalloc(const uint8_t* d_in, uint32_t n, uint8_t* d_L, int32_t* d_primary,
                                                void* stream) {
    if (!d_in || !d_L || !d_primary || n == 0) return BWT_EINVAL;
    if (n > NA_MAX) return BWT_ETOOBIG;
    if (overlaps(d_in, n, d_L, n) || overlaps(d_primary, sizeof(int32_t), d_L, n) ||
        overlaps(d_primary, sizeof(int32_t), d_in, n))
        return BWT_EINVAL;
    void* scratch = nullptr;
    bwt_status s = noalloc_scratch(&scratch);
    if (s != BWT_OK) return s;
    k_bwt_block_noalloc<<<1, NA_THREADS, 0, (cudaStream_t)stream>>>(d_in, n, d_L, d_primary,
                                                                     static_cast<uint32_t*>(scratch));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bwt::record_cuda(e, "k_bwt_block_noalloc launch");
    return BWT_OK;
}
