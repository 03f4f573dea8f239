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

static const char kModelTag[8] = {'B', 'W', 'T', 'M', 'D', 'L', '0', '2'};

extern "C" bwt_status bwt_model_save(const char* path, const float* params, const float* norm,
                                     const uint64_t* splitters) {
    if (!path || !params || !norm || !splitters) return BWT_EINVAL;
    FILE* f = std::fopen(path, "wb");
    if (!f) return BWT_EINVAL;
    bool ok = std::fwrite(kModelTag, 1, 8, f) == 8 &&
              std::fwrite(params, sizeof(float), BWT_MLP_NPARAMS, f) == BWT_MLP_NPARAMS &&
              std::fwrite(norm, sizeof(float), 256, f) == 256 &&
              std::fwrite(splitters, sizeof(uint64_t), BWT_SPLITTERS, f) == BWT_SPLITTERS;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? BWT_OK : BWT_EINVAL;
}

extern "C" bwt_status bwt_model_load(const char* path, float* params, float* norm, uint64_t* splitters) {
    if (!path || !params || !norm || !splitters) return BWT_EINVAL;
    FILE* f = std::fopen(path, "rb");
    if (!f) return BWT_ENOMODEL;
    char tag[8];
    bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, kModelTag, 8) == 0 &&
              std::fread(params, sizeof(float), BWT_MLP_NPARAMS, f) == BWT_MLP_NPARAMS &&
              std::fread(norm, sizeof(float), 256, f) == 256 &&
              std::fread(splitters, sizeof(uint64_t), BWT_SPLITTERS, f) == BWT_SPLITTERS;
    std::fclose(f);
    return ok ? BWT_OK : BWT_ENOMODEL;
}

extern "C" bwt_status bwt_plan_set_splitters(bwt_plan* p, const uint64_t* splitters) {
    if (!p || !splitters) return BWT_EINVAL;
    CKL(cudaSetDevice(p->device));
    std::vector<uint64_t> h(BWT_SPLITTERS);
    CKL(cudaMemcpy(h.data(), splitters, sizeof(uint64_t) * BWT_SPLITTERS, cudaMemcpyDefault));
    for (int i = 1; i < BWT_SPLITTERS; ++i)
        if (h[i] < h[i - 1]) return BWT_EINVAL;
    bwt_status s = ensure_learned_buffers(p);
    if (s != BWT_OK) return s;
    CKL(cudaMemcpy(p->splitters, h.data(), sizeof(uint64_t) * BWT_SPLITTERS, cudaMemcpyHostToDevice));
    p->have_model = true;
    return BWT_OK;
}

bwt_status bwt::load_model(bwt_plan* p, const char* path) {
    if (!path || !*path) return BWT_ENOMODEL;
    std::vector<float> params(BWT_MLP_NPARAMS), norm(256);
    std::vector<uint64_t> spl(BWT_SPLITTERS);
    bwt_status s = bwt_model_load(path, params.data(), norm.data(), spl.data());
    if (s != BWT_OK) return s;
    return bwt_plan_set_splitters(p, spl.data());
}

namespace {

__global__ void k_make_samples(const uint8_t* __restrict__ S, const uint32_t* __restrict__ SA,
                               const BlockInfo* __restrict__ blocks, uint32_t nb, const uint64_t* __restrict__ pos,
                               uint32_t count, const float* __restrict__ norm, float* __restrict__ x,
                               float* __restrict__ t) {
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
        x[(size_t)s * 8 + j] = norm[S[bi.off + q]];
    }
    t[s] = (float)(k - bi.off) / (float)bi.n;
}

__global__ void k_byte_hist(const uint8_t* __restrict__ S, uint64_t n, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[S[i]], 1u);
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_byte_norm(const uint32_t* __restrict__ hist, uint64_t n, float* __restrict__ norm) {
    if (threadIdx.x != 0) return;
    uint64_t below = 0;
    for (int b = 0; b < 256; ++b) {
        norm[b] = (float)(((double)below + 0.5 * (double)hist[b]) / (double)n);
        below += hist[b];
    }
}

}  // namespace

extern "C" bwt_status bwt_model_byte_norm(const uint8_t* d_in, uint64_t n, float* d_norm, void* stream) {
    if (!d_in || !d_norm || n == 0 || n >= (1ull << 32)) return BWT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* hist = nullptr;
    CKL(cudaMalloc(&hist, 256 * sizeof(uint32_t)));
    cudaError_t e = cudaMemsetAsync(hist, 0, 256 * sizeof(uint32_t), st);
    if (e == cudaSuccess) {
        k_byte_hist<<<num_sms() * 4, 256, 0, st>>>(d_in, n, hist);
        k_byte_norm<<<1, 32, 0, st>>>(hist, n, d_norm);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(hist);
    CKL(e);
    return BWT_OK;
}

extern "C" bwt_status bwt_model_samples(bwt_plan* p, const uint8_t* d_in, const uint64_t* offsets,
                                        uint32_t num_blocks, const uint64_t* d_pos, uint32_t count,
                                        const float* d_norm, float* d_x, float* d_t, void* stream) {
    if (!p || !d_in || !offsets || !d_pos || !d_norm || !d_x || !d_t) return BWT_EINVAL;
    CKL(cudaSetDevice(p->device));
    cudaStream_t st = (cudaStream_t)stream;
    std::memset(&p->stats, 0, sizeof(p->stats));
    bwt_status s = prepare_batch(p, offsets, num_blocks, st);
    if (s != BWT_OK) return s;
    if ((s = reset_ctrl(p, st)) != BWT_OK) return s;
    if ((s = enqueue_initial_sort(p, d_in, st)) != BWT_OK) return s;
    if ((s = run_doubling_host_loop(p, st)) != BWT_OK) return s;
    if (count) {
        k_make_samples<<<(count + 255) / 256, 256, 0, st>>>(d_in, p->sa, p->blocks, p->nb, d_pos, count, d_norm,
                                                            d_x, d_t);
        CKL(cudaGetLastError());
    }
    return finish_status(p, st);
}

// ---------------------------------------------------------------------------
// Learned bucketing of a batch (BWT_F_LEARNED).
//
//   count:   bucket b(i) = #{j : splitter[j] <= K_i} of every rotation, counted
//            per block (a 12-step binary search over the splitters in shared
//            memory);
//   route:   a block whose over-capacity buckets hold more than a quarter of
//            its rotations is sorted by the plain radix instead;
//   scatter: rotations go to their bucket's range (per-tile reservation of
//            each bucket's slots with one atomic per tile and bucket);
//   sort:    consecutive whole buckets are grouped into chunks of at most
//            `cap` rotations and each chunk is sorted by (K, i) in shared
//            memory -- buckets are ordered by K, so a sorted chunk sorts every
//            bucket in it;
//   overflow buckets (> cap) are sorted by the segmented radix: first by the
//            rotation index (digits taken from the value), then by K, which
//            leaves equal prefixes in index order as the doubling rounds
//            require.
// Then naming, prefix doubling and the L gather run as on the plain path.

namespace {

constexpr int NBK = BWT_BUCKETS;
constexpr int NSP = BWT_SPLITTERS;
constexpr uint32_t BUCKET_CAP = 2048;

__device__ __forceinline__ uint32_t bucket_of(const uint64_t* spl, uint64_t key) {
    uint32_t lo = 0, hi = NSP;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (spl[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint64_t pack8b(const uint8_t* b) {
    uint64_t k = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) k = (k << 8) | b[j];
    return k;
}

// bytes of rotation positions [i0, i0 + len + 7) of block bi, wrapping
__device__ __forceinline__ void load_tile_bytes(const uint8_t* S, BlockInfo bi, uint32_t i0, uint32_t len,
                                                uint8_t* sb) {
    for (uint32_t q = threadIdx.x; q < len + 7; q += blockDim.x) {
        uint32_t pos = i0 + q;
        if (pos >= bi.n) pos = bi.n >= 8 ? pos - bi.n : pos % bi.n;
        sb[q] = S[bi.off + pos];
    }
}

constexpr size_t SPL_BYTES = 4096 * 8;
constexpr size_t CNT_BYTES = 4096 * 4;
constexpr size_t TILE_BYTES = 4096 + 16;
constexpr size_t COUNT_SMEM = SPL_BYTES + CNT_BYTES + TILE_BYTES;
constexpr size_t SCATTER_SMEM = SPL_BYTES + 2 * CNT_BYTES + TILE_BYTES;

__global__ void __launch_bounds__(256) k_bucket_count(const uint8_t* __restrict__ S, const BlockInfo* __restrict__ blocks,
                                                      const TileDesc* __restrict__ tiles, uint32_t ntiles,
                                                      const uint64_t* __restrict__ splitters,
                                                      uint32_t* __restrict__ counts) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* spl = reinterpret_cast<uint64_t*>(smem);
    uint32_t* h = reinterpret_cast<uint32_t*>(smem + SPL_BYTES);
    uint8_t* sb = smem + SPL_BYTES + CNT_BYTES;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < NSP; i += blockDim.x) spl[i] = splitters[i];
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (int i = threadIdx.x; i < NBK; i += blockDim.x) h[i] = 0;
        const TileDesc td = tiles[t];
        const BlockInfo bi = blocks[td.blk];
        load_tile_bytes(S, bi, td.start - bi.off, td.len, sb);
        __syncthreads();
        for (uint32_t q0 = 0; q0 < td.len; q0 += blockDim.x) {
            const uint32_t q = q0 + threadIdx.x;
            const bool valid = q < td.len;
            const uint32_t b = valid ? bucket_of(spl, pack8b(sb + q)) : (uint32_t)NBK;
            const uint32_t peers = __match_any_sync(0xffffffffu, b);
            if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[b], (uint32_t)__popc(peers));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < NBK; i += blockDim.x) {
            const uint32_t c = h[i];
            if (c) atomicAdd(&counts[(size_t)td.blk * NBK + i], c);
        }
        __syncthreads();
    }
}

// Per block: keys in over-capacity buckets, number of such buckets, largest
// bucket, sum of squared bucket sizes, non-empty buckets (u64 each).
__global__ void __launch_bounds__(256) k_bucket_stats(const uint32_t* __restrict__ counts, uint32_t cap,
                                                      uint32_t nb, unsigned long long* __restrict__ out) {
    __shared__ unsigned long long r[5][256];
    for (uint32_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        unsigned long long ok = 0, ob = 0, mx = 0, sq = 0, ne = 0;
        for (int i = threadIdx.x; i < NBK; i += blockDim.x) {
            const unsigned long long v = counts[(size_t)blk * NBK + i];
            mx = v > mx ? v : mx;
            sq += v * v;
            ne += v > 0;
            if (v > cap) {
                ok += v;
                ++ob;
            }
        }
        r[0][threadIdx.x] = ok;
        r[1][threadIdx.x] = ob;
        r[2][threadIdx.x] = mx;
        r[3][threadIdx.x] = sq;
        r[4][threadIdx.x] = ne;
        __syncthreads();
        for (int st = 128; st > 0; st >>= 1) {
            if ((int)threadIdx.x < st) {
                r[0][threadIdx.x] += r[0][threadIdx.x + st];
                r[1][threadIdx.x] += r[1][threadIdx.x + st];
                r[2][threadIdx.x] = r[2][threadIdx.x] > r[2][threadIdx.x + st] ? r[2][threadIdx.x] : r[2][threadIdx.x + st];
                r[3][threadIdx.x] += r[3][threadIdx.x + st];
                r[4][threadIdx.x] += r[4][threadIdx.x + st];
            }
            __syncthreads();
        }
        if (threadIdx.x < 5) out[5 * blk + threadIdx.x] = r[threadIdx.x][0];
        __syncthreads();
    }
}

template <int ITEMS>
__global__ void __launch_bounds__(256) k_bucket_scatter(const uint8_t* __restrict__ S,
                                                        const BlockInfo* __restrict__ blocks,
                                                        const TileDesc* __restrict__ tiles, uint32_t ntiles,
                                                        const uint64_t* __restrict__ splitters,
                                                        const uint32_t* __restrict__ starts,
                                                        uint32_t* __restrict__ cursor, uint64_t* __restrict__ K,
                                                        uint32_t* __restrict__ I) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* spl = reinterpret_cast<uint64_t*>(smem);
    uint32_t* lcount = reinterpret_cast<uint32_t*>(smem + SPL_BYTES);
    uint32_t* gbase = reinterpret_cast<uint32_t*>(smem + SPL_BYTES + CNT_BYTES);
    uint8_t* sb = smem + SPL_BYTES + 2 * CNT_BYTES;
    const int lane = threadIdx.x & 31;
    uint32_t lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    for (int i = threadIdx.x; i < NSP; i += blockDim.x) spl[i] = splitters[i];
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (int i = threadIdx.x; i < NBK; i += blockDim.x) lcount[i] = 0;
        const TileDesc td = tiles[t];
        const BlockInfo bi = blocks[td.blk];
        const uint32_t i0 = td.start - bi.off;
        load_tile_bytes(S, bi, i0, td.len, sb);
        __syncthreads();
        uint64_t key[ITEMS];
        uint32_t bl[ITEMS];  // bucket (low 12 bits) | slot within the tile's share of the bucket << 12
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t q = j * 256 + threadIdx.x;
            const bool valid = q < td.len;
            key[j] = valid ? pack8b(sb + q) : 0ull;
            const uint32_t b = valid ? bucket_of(spl, key[j]) : (uint32_t)NBK;
            const uint32_t peers = __match_any_sync(0xffffffffu, b);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (valid && lane == leader) base = atomicAdd(&lcount[b], (uint32_t)__popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            bl[j] = valid ? (b | ((base + __popc(peers & lt)) << 12)) : 0xffffffffu;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < NBK; i += blockDim.x) {
            const uint32_t c = lcount[i];
            if (c) gbase[i] = atomicAdd(&cursor[(size_t)td.blk * NBK + i], c);
        }
        __syncthreads();
        const uint32_t* st = starts + (size_t)td.blk * NBK;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (bl[j] != 0xffffffffu) {
                const uint32_t b = bl[j] & 4095u;
                const uint32_t pos = bi.off + st[b] + gbase[b] + (bl[j] >> 12);
                K[pos] = key[j];
                I[pos] = i0 + j * 256 + threadIdx.x;
            }
        }
        __syncthreads();
    }
}

// Greedy grouping of each bucket-routed block's consecutive buckets into
// chunks of at most cap rotations; over-capacity buckets become overflow
// segments. One CTA per block; thread 0 walks the 4096 bucket sizes.
__global__ void __launch_bounds__(256) k_bucket_chunks(const uint32_t* __restrict__ starts,
                                                       const BlockInfo* __restrict__ blocks,
                                                       const uint32_t* __restrict__ route, uint32_t nb, uint32_t cap,
                                                       Bins out, uint32_t* ctrl) {
    __shared__ uint32_t st[NBK + 1];
    for (uint32_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        if (route[blk] != 0) continue;  // uniform across the CTA
        const BlockInfo bi = blocks[blk];
        for (int i = threadIdx.x; i < NBK; i += blockDim.x) st[i] = starts[(size_t)blk * NBK + i];
        if (threadIdx.x == 0) st[NBK] = bi.n;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t cstart = 0, clen = 0;
            auto push = [&](int cls, uint32_t s0, uint32_t len) {
                const uint32_t slot = atomicAdd(&out.count[cls], 1u);
                if (slot < out.cap[cls]) out.list[cls][slot] = GroupDesc{bi.off + s0, len, blk, 0u};
                else atomicOr(&ctrl[CTRL_ERR], ERR_CAPACITY);
            };
            for (int b = 0; b < NBK; ++b) {
                const uint32_t sz = st[b + 1] - st[b];
                if (sz > cap) {
                    if (clen > 1) push(0, cstart, clen);
                    push(CLS_LARGE, st[b], sz);
                    cstart = st[b + 1];
                    clen = 0;
                } else if (clen + sz > cap) {
                    if (clen > 1) push(0, cstart, clen);
                    cstart = st[b];
                    clen = sz;
                } else {
                    clen += sz;
                }
            }
            if (clen > 1) push(0, cstart, clen);
        }
        __syncthreads();
    }
}

// Sorts every chunk by (K, i) in shared memory (bitonic; len <= BUCKET_CAP).
__global__ void __launch_bounds__(256) k_chunk_sort(uint64_t* __restrict__ K, uint32_t* __restrict__ I, Bins chunks) {
    __shared__ uint64_t sk[BUCKET_CAP];
    __shared__ uint32_t si[BUCKET_CAP];
    const uint32_t n = bin_count(chunks, 0);
    for (uint32_t c = blockIdx.x; c < n; c += gridDim.x) {
        const GroupDesc g = chunks.list[0][c];
        uint32_t P = 2;
        while (P < g.len) P <<= 1;
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
            if (i < g.len) {
                sk[i] = K[g.start + i];
                si[i] = I[g.start + i];
            } else {
                sk[i] = ~0ull;
                si[i] = ~0u;
            }
        }
        __syncthreads();
        for (uint32_t kk = 2; kk <= P; kk <<= 1) {
            for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
                for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                    const uint32_t ixj = i ^ j;
                    if (ixj > i) {
                        const uint64_t a = sk[i], b = sk[ixj];
                        const uint32_t ai = si[i], bi = si[ixj];
                        const bool gt = a > b || (a == b && ai > bi);
                        const bool up = (i & kk) == 0;
                        if (gt == up) {
                            sk[i] = b;
                            sk[ixj] = a;
                            si[i] = bi;
                            si[ixj] = ai;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t i = threadIdx.x; i < g.len; i += blockDim.x) {
            K[g.start + i] = sk[i];
            I[g.start + i] = si[i];
        }
        __syncthreads();
    }
}

// Per overflow segment: digit histograms of PI index passes then PK key passes.
__global__ void __launch_bounds__(256) k_seg_hist_u64(const uint64_t* __restrict__ K, const uint32_t* __restrict__ I,
                                                      const TileDesc* __restrict__ tiles,
                                                      const uint32_t* __restrict__ num_tiles,
                                                      uint32_t* __restrict__ hist, int PI, int PK) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* h = reinterpret_cast<uint32_t*>(smem);
    const int P = PI + PK;
    const int lane = threadIdx.x & 31;
    const uint32_t nt = *num_tiles;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        for (int i = threadIdx.x; i < P * 256; i += blockDim.x) h[i] = 0;
        __syncthreads();
        const TileDesc td = tiles[t];
        for (uint32_t q0 = 0; q0 < td.len; q0 += blockDim.x) {
            const uint32_t q = q0 + threadIdx.x;
            const bool valid = q < td.len;
            const uint64_t k = valid ? K[td.start + q] : 0ull;
            const uint32_t v = valid ? I[td.start + q] : 0u;
            for (int ps = 0; ps < P; ++ps) {
                uint32_t d = 256;
                if (valid) d = ps < PI ? (v >> (8 * ps)) & 255u : (uint32_t)((k >> (8 * (ps - PI))) & 255u);
                const uint32_t peers = __match_any_sync(0xffffffffu, d);
                if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[ps * 256 + d], (uint32_t)__popc(peers));
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < P * 256; i += blockDim.x) {
            const uint32_t c = h[i];
            if (c) atomicAdd(&hist[(size_t)td.seg * P * 256 + i], c);
        }
        __syncthreads();
    }
}

__global__ void k_copy_tiles(const uint64_t* __restrict__ Ks, const uint32_t* __restrict__ Is,
                             uint64_t* __restrict__ Kd, uint32_t* __restrict__ Id, const TileDesc* __restrict__ tiles,
                             const uint32_t* __restrict__ num_tiles) {
    const uint32_t nt = *num_tiles;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const TileDesc td = tiles[t];
        for (uint32_t q = threadIdx.x; q < td.len; q += blockDim.x) {
            Kd[td.start + q] = Ks[td.start + q];
            Id[td.start + q] = Is[td.start + q];
        }
    }
}

int bits_needed(uint32_t max_value) {
    int b = 0;
    while (b < 32 && (max_value >> b) != 0) ++b;
    return b;
}

}  // namespace

bwt_status bwt::ensure_learned_buffers(bwt_plan* p) {
    const size_t nbk = (size_t)p->cap_b * NBK;
    if (!p->splitters) CKL(cudaMalloc(&p->splitters, sizeof(uint64_t) * NSP));
    if (!p->bucket_count) CKL(cudaMalloc(&p->bucket_count, sizeof(uint32_t) * nbk));
    if (!p->bucket_cursor) CKL(cudaMalloc(&p->bucket_cursor, sizeof(uint32_t) * nbk));
    if (!p->route) CKL(cudaMalloc(&p->route, sizeof(uint32_t) * p->cap_b));
    if (!p->bstats) CKL(cudaMalloc(&p->bstats, sizeof(unsigned long long) * 5 * p->cap_b));
    if (!p->tiles_aux) CKL(cudaMalloc(&p->tiles_aux, sizeof(TileDesc) * p->cap_tiles0));
    if (!p->h_route) CKL(cudaMallocHost(&p->h_route, sizeof(uint32_t) * p->cap_b));
    if (!p->h_bstats) CKL(cudaMallocHost(&p->h_bstats, sizeof(unsigned long long) * 5 * p->cap_b));
    if (!p->h_tiles_aux) CKL(cudaMallocHost(&p->h_tiles_aux, sizeof(TileDesc) * p->cap_tiles0));
    return BWT_OK;
}

bwt_status bwt::run_learned(bwt_plan* p, const uint8_t* d_in, uint8_t* d_L, int32_t* d_primary, cudaStream_t st) {
    if (!p->have_model) return BWT_ENOMODEL;
    bwt_status s;
    if ((s = ensure_learned_buffers(p)) != BWT_OK) return s;
    static bool attr = [] {
        cudaFuncSetAttribute((void*)k_bucket_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)COUNT_SMEM);
        cudaFuncSetAttribute((void*)k_bucket_scatter<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SCATTER_SMEM);
        cudaFuncSetAttribute((void*)k_bucket_scatter<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SCATTER_SMEM);
        cudaFuncSetAttribute((void*)k_bucket_scatter<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SCATTER_SMEM);
        return true;
    }();
    (void)attr;
    const uint32_t nb = p->nb, nt = p->ntiles0;
    const int sms = num_sms();
    uint32_t* ctrl = p->ctrl;
    if ((s = reset_ctrl(p, st)) != BWT_OK) return s;

    // 1. count buckets per block, 2. per-block overflow statistics
    CKL(cudaMemsetAsync(p->bucket_count, 0, sizeof(uint32_t) * NBK * nb, st));
    k_bucket_count<<<std::max(1, std::min<int>(nt, sms * 3)), 256, COUNT_SMEM, st>>>(d_in, p->blocks, p->tiles0, nt,
                                                                                     p->splitters, p->bucket_count);
    k_bucket_stats<<<std::min<uint32_t>(nb, 65535), 256, 0, st>>>(p->bucket_count, BUCKET_CAP, nb, p->bstats);
    CKL(cudaGetLastError());
    CKL(cudaMemcpyAsync(p->h_bstats, p->bstats, sizeof(unsigned long long) * 5 * nb, cudaMemcpyDeviceToHost, st));
    CKL(cudaStreamSynchronize(st));
    p->stats.kernel_launches += 3;

    // 3. route: plain radix for blocks whose overflow exceeds a quarter of the block
    uint32_t ntp = 0, ntb = 0;
    std::vector<uint32_t> plain_blocks;
    uint64_t plain_keys = 0;
    for (uint32_t b = 0; b < nb; ++b) {
        const BlockInfo bi = p->h_blocks[b];
        const unsigned long long* bs = p->h_bstats + 5 * b;
        const bool plain = bs[0] * 4 > bi.n;
        p->h_route[b] = plain ? 1u : 0u;
        if (plain) {
            plain_blocks.push_back(b);
            plain_keys += bi.n;
            p->stats.blocks_routed_plain++;
        } else {
            p->stats.buckets_overflowed += bs[1];
            p->stats.keys_overflowed += bs[0];
        }
        p->stats.max_bucket = std::max<uint32_t>(p->stats.max_bucket, (uint32_t)bs[2]);
        p->stats.bucket_sq_sum += bs[3];
        p->stats.buckets_nonempty += bs[4];
    }
    // sub-tables (first-tile indices relative to each sub-table): plain blocks first, then bucketed
    const uint32_t T = (uint32_t)p->tile;
    for (int pass = 0; pass < 2; ++pass) {
        for (uint32_t b = 0; b < nb; ++b) {
            if ((p->h_route[b] == 1u) != (pass == 0)) continue;
            const BlockInfo bi = p->h_blocks[b];
            const uint32_t base = pass == 0 ? 0 : ntp;
            const uint32_t first = (pass == 0 ? ntp : ntb) ;
            for (uint32_t o = 0; o < bi.n; o += T) {
                TileDesc td;
                td.start = bi.off + o;
                td.len = std::min(T, bi.n - o);
                td.seg = b;
                td.firstTile = first;
                td.segStart = bi.off;
                td.blk = b;
                td.pad0 = bi.n;
                td.pad1 = 0;
                p->h_tiles_aux[base + (pass == 0 ? ntp++ : ntb++)] = td;
            }
        }
    }
    CKL(cudaMemcpyAsync(p->route, p->h_route, sizeof(uint32_t) * nb, cudaMemcpyHostToDevice, st));
    CKL(cudaMemcpyAsync(p->tiles_aux, p->h_tiles_aux, sizeof(TileDesc) * (ntp + ntb), cudaMemcpyHostToDevice, st));
    p->h_aux[0] = ntp;
    p->h_aux[1] = ntb;
    CKL(cudaMemcpyAsync(ctrl + CTRL_AUX0, p->h_aux, sizeof(uint32_t) * 2, cudaMemcpyHostToDevice, st));
    const TileDesc* tilesP = p->tiles_aux;
    const TileDesc* tilesB = p->tiles_aux + ntp;

    // 4a. plain-routed blocks: the first sort of the plain path, ending in buffer 0
    const int rb = p->rbits, RADIX = 1 << rb;
    if (ntp) {
        const int P = (64 + rb - 1) / rb;
        uint32_t seg_stride;
        if (rb == 8) {
            CKL(cudaMemsetAsync(p->hist, 0, sizeof(uint32_t) * 256 * nb, st));
            CKL(launch_hist_bytes(d_in, p->blocks, tilesP, ntp, p->hist, st));
            CKL(launch_scan_rows(p->hist, 256, nullptr, 0, nb, nb, st));
            seg_stride = 256;
        } else {
            CKL(cudaMemsetAsync(p->hist, 0, sizeof(uint32_t) * 6 * 2048 * nb, st));
            CKL(launch_hist_keys11(d_in, p->blocks, tilesP, ntp, p->tile, p->hist, st));
            CKL(launch_scan_rows(p->hist, 2048, nullptr, 0, nb * 6, nb * 6, st));
            seg_stride = 6 * 2048;
        }
        p->stats.kernel_launches += 2;
        for (int ps = 0; ps < P; ++ps) {
            CKL(cudaMemsetAsync(p->status, 0, sizeof(uint32_t) * (size_t)ntp * RADIX, st));
            OneSweepParams a{};
            const int out = (P - 1 - ps) & 1, in = (P - ps) & 1;
            a.kin = ps == 0 ? nullptr : p->keys[in];
            a.vin = ps == 0 ? nullptr : p->vals[in];
            a.kout = p->keys[out];
            a.vout = p->vals[out];
            a.S = d_in;
            a.blocks = p->blocks;
            a.tiles = tilesP;
            a.num_tiles = ctrl + CTRL_AUX0;
            a.seg_base = p->hist + (rb == 8 ? 0 : ps * 2048);
            a.seg_base_stride = seg_stride;
            a.status = p->status;
            a.tile_counter = ctrl + CTRL_TILE_CTR + ps;
            a.ctrl = ctrl;
            a.shift = ps * rb;
            CKL(launch_onesweep(8, ps == 0, rb, p->tile, a, 0, st));
            p->stats.kernel_launches++;
            p->stats.radix_launches++;
            p->stats.radix_keys += plain_keys;
        }
    }

    // 4b. bucket-routed blocks: scan, scatter, chunk sort
    Bins aux = bins_of(p, 1);
    CKL(cudaMemsetAsync(aux.count, 0, sizeof(uint32_t) * NCLS, st));
    if (ntb) {
        CKL(launch_scan_rows(p->bucket_count, NBK, nullptr, 0, nb, nb, st));  // counts -> starts in place
        CKL(cudaMemsetAsync(p->bucket_cursor, 0, sizeof(uint32_t) * NBK * nb, st));
        const int g = std::max(1, std::min<int>(ntb, sms * 2));
        if (T <= 1024)
            k_bucket_scatter<4><<<g, 256, SCATTER_SMEM, st>>>(d_in, p->blocks, tilesB, ntb, p->splitters,
                                                              p->bucket_count, p->bucket_cursor, p->keys[0], p->vals[0]);
        else if (T <= 2048)
            k_bucket_scatter<8><<<g, 256, SCATTER_SMEM, st>>>(d_in, p->blocks, tilesB, ntb, p->splitters,
                                                              p->bucket_count, p->bucket_cursor, p->keys[0], p->vals[0]);
        else
            k_bucket_scatter<16><<<g, 256, SCATTER_SMEM, st>>>(d_in, p->blocks, tilesB, ntb, p->splitters,
                                                               p->bucket_count, p->bucket_cursor, p->keys[0],
                                                               p->vals[0]);
        k_bucket_chunks<<<std::min<uint32_t>(nb, 65535), 256, 0, st>>>(p->bucket_count, p->blocks, p->route, nb,
                                                                       BUCKET_CAP, aux, ctrl);
        k_chunk_sort<<<sms * 6, 256, 0, st>>>(p->keys[0], p->vals[0], aux);
        CKL(cudaGetLastError());
        p->stats.kernel_launches += 4;

        // 4c. overflow buckets: radix on the index, then on the key
        const int PI = std::max(1, (bits_needed(p->max_n - 1) + 7) / 8), PK = 8, PT = PI + PK;
        CKL(launch_build_large_tiles(aux, p->tile, p->ltiles, p->cap_ltiles, ctrl, st));
        CKL(launch_zero_by_count(p->hist, aux.count + CLS_LARGE, (uint32_t)(PT * 256),
                                 (uint32_t)std::min<uint64_t>(p->cap_hist, 0xffffffffu), st));
        k_seg_hist_u64<<<sms * 4, 256, PT * 256 * 4, st>>>(p->keys[0], p->vals[0], p->ltiles, ctrl + CTRL_NUM_LTILES,
                                                           p->hist, PI, PK);
        CKL(cudaGetLastError());
        CKL(launch_scan_rows(p->hist, 256, aux.count + CLS_LARGE, (uint32_t)PT, 0, (uint32_t)(p->cap_hist / 256),
                             st));
        p->stats.kernel_launches += 4;
        for (int ps = 0; ps < PT; ++ps) {
            CKL(launch_zero_by_count(p->status, ctrl + CTRL_NUM_LTILES, 256u,
                                     (uint32_t)std::min<uint64_t>(p->cap_status, 0xffffffffu), st));
            CKL(cudaMemsetAsync(ctrl + CTRL_TILE_CTR + 16 + ps, 0, 4, st));
            OneSweepParams a{};
            a.kin = p->keys[ps & 1];
            a.vin = p->vals[ps & 1];
            a.kout = p->keys[(ps + 1) & 1];
            a.vout = p->vals[(ps + 1) & 1];
            a.blocks = p->blocks;
            a.tiles = p->ltiles;
            a.num_tiles = ctrl + CTRL_NUM_LTILES;
            a.seg_base = p->hist + ps * 256;
            a.seg_base_stride = (uint32_t)(PT * 256);
            a.status = p->status;
            a.tile_counter = ctrl + CTRL_TILE_CTR + 16 + ps;
            a.ctrl = ctrl;
            a.shift = ps < PI ? 8 * ps : 8 * (ps - PI);
            CKL(launch_onesweep(ps < PI ? -8 : 8, false, 8, p->tile, a, 0, st));
            p->stats.kernel_launches += 2;
            p->stats.radix_launches++;
            p->stats.radix_keys += p->stats.keys_overflowed;
        }
        if (PT & 1) {
            k_copy_tiles<<<sms * 4, 256, 0, st>>>(p->keys[1], p->vals[1], p->keys[0], p->vals[0], p->ltiles,
                                                  ctrl + CTRL_NUM_LTILES);
            CKL(cudaGetLastError());
            p->stats.kernel_launches++;
        }
    }

    // 5. naming, doubling, L gather -- as on the plain path, from buffer 0
    p->sa = p->vals[0];
    p->key2 = p->vals[1];
    p->kA = reinterpret_cast<uint32_t*>(p->keys[1]);
    p->vA = p->kA + p->cap_n;
    p->kB = reinterpret_cast<uint32_t*>(p->keys[0]);
    p->vB = p->kB + p->cap_n;
    if ((s = enqueue_naming(p, p->keys[0], st)) != BWT_OK) return s;
    if ((s = run_doubling_host_loop(p, st)) != BWT_OK) return s;
    CKL(launch_gather_L(d_in, p->sa, p->blocks, p->tiles0, p->ntiles0, d_L, d_primary, st));
    p->stats.kernel_launches++;
    return BWT_OK;
}
