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
    if ((s = build_splitter_index(p)) != BWT_OK) return s;
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
    const uint32_t sa = SA[k] & ~SA_FINAL;
    const uint32_t i = sa < bi.n ? sa : 0u;
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
    bwt::NvtxRange nvtx_range("mlp_byte_norm");
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
    bwt::NvtxRange nvtx_range("mlp_samples");
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
//            per block (a search of the splitters in shared memory from an
//            index on the key's first two bytes), the bucket stored per
//            rotation;
//   route:   a block whose over-capacity buckets hold more than a quarter of
//            its rotations is counted again with equal-width buckets (the top
//            12 key bits), and sorted by the plain radix if those overflow too;
//   plan:    consecutive buckets are grouped into chunks of at most 3328
//            padded rotations (a bucket above that is an overflow bucket);
//   scatter: each tile's rotations go to their chunk's range in runs (one
//            slot reservation per tile and chunk), tagged with their bucket;
//   sort:    one CTA per chunk sorts every bucket by (K, i) with a team of
//            its threads, writes the chunk's SA and names it (a chunk is a
//            whole key range, so its groups begin and end inside it); groups
//            of one keep no stored rank (they are found on demand); an
//            overflow bucket of up to 13,312 rotations is sorted the same way
//            by one 512- or 1,024-thread CTA;
//   larger overflow buckets are sorted by the segmented radix: first by the
//            rotation index (digits taken from the value), then by K, which
//            leaves equal prefixes in index order as the doubling rounds
//            require, and named inside their own bounds.
// Then prefix doubling and the L gather run as on the plain path.

namespace {

constexpr int NBK = BWT_BUCKETS;
constexpr int NSP = BWT_SPLITTERS;

// The splitter search (bucket_of) starts from an index on the key's first
// two bytes: text keys use a few thousand of the 65,536 two-byte prefixes
// and the splitters spread over them, so a search takes one or two steps
// (five or six with an index on the top 12 bits, whose bank conflicts bound
// the counting kernel).
static_assert(NBK == LR_BUCKETS, "the lazy rank lookup indexes bucket starts by learned bucket");

// The index of a splitter table (built once when the table is installed).
__global__ void k_build_index(const uint64_t* __restrict__ spl, uint16_t* __restrict__ first) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < IDX_WORDS; c += gridDim.x * blockDim.x) {
        uint32_t lo = NSP;
        if (c < IDX_CELLS) {
            const uint64_t x = (uint64_t)c << (64 - IDX_BITS);
            uint32_t hi = NSP;
            lo = 0;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (spl[mid] < x) lo = mid + 1; else hi = mid;
            }
        }
        first[c] = (uint16_t)lo;
    }
}

// Loads the splitters and their index into shared memory.
__device__ __forceinline__ void load_splitters(const uint64_t* __restrict__ splitters,
                                               const uint16_t* __restrict__ index, uint64_t* spl, uint16_t* first) {
    for (int i = threadIdx.x; i < NSP; i += blockDim.x) spl[i] = splitters[i];
    const uint4* src = reinterpret_cast<const uint4*>(index);
    uint4* dst = reinterpret_cast<uint4*>(first);
    for (int i = threadIdx.x; i < IDX_WORDS / 8; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

constexpr size_t SPL_BYTES = 4096 * 8 + IDX_WORDS * 2;  // splitters + two-byte-prefix index
constexpr size_t CNT_BYTES = 4096 * 4;
constexpr size_t TILE_BYTES = 4096 + 48;
constexpr size_t COUNT_SMEM = SPL_BYTES + CNT_BYTES + TILE_BYTES;
constexpr int COUNT_THREADS = 1024;  // one CTA an SM: its shared memory holds the splitters and the index

// Counts every rotation's bucket. FLAT = false: the learned bucketing of
// every block, storing each rotation's learned bucket in fb (u16 per
// rotation) for the scatter; FLAT = true: the equal-width bucketing (the top
// 12 key bits) of the blocks marked in `need` only (those the learned
// buckets do not fit). Text keys crowd a few of the equal-width buckets, so
// their shared-memory atomics conflict: counting them only where the routing
// needs them keeps them off the common path. Counts gather in one shared-
// memory word per bucket (learned in the low half, equal-width in the high
// half), so a CTA counts at most 65535 rotations (`span` tiles) before it
// adds them to the block's rows: one global atomic per non-empty bucket and
// span; a span that crosses into the next block flushes at the boundary.
// counts: [2][block][4096] (learned rows, then equal-width rows).
__device__ __forceinline__ void flush_counts(uint32_t* h, uint32_t* __restrict__ counts, uint32_t nb, uint32_t blk) {
    for (int i = threadIdx.x; i < NBK; i += blockDim.x) {
        const uint32_t c = h[i];
        h[i] = 0;
        if (c & 0xffffu) atomicAdd(&counts[(size_t)blk * NBK + i], c & 0xffffu);
        if (c >> 16) atomicAdd(&counts[((size_t)nb + blk) * NBK + i], c >> 16);
    }
}

template <bool FLAT>
__global__ void __launch_bounds__(COUNT_THREADS, 1) k_bucket_count(const uint8_t* __restrict__ S,
                                                                    const BlockInfo* __restrict__ blocks,
                                                                    const TileDesc* __restrict__ tiles,
                                                                    uint32_t ntiles, uint32_t span,
                                                                    const uint64_t* __restrict__ splitters,
                                                                    const uint16_t* __restrict__ index,
                                                                    uint32_t nb, uint32_t* __restrict__ counts,
                                                                    uint16_t* __restrict__ fb,
                                                                    const uint32_t* __restrict__ need) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* spl = reinterpret_cast<uint64_t*>(smem);
    uint16_t* first = reinterpret_cast<uint16_t*>(smem + 4096 * 8);
    uint32_t* h = reinterpret_cast<uint32_t*>(smem + SPL_BYTES);
    uint8_t* sb = smem + SPL_BYTES + CNT_BYTES;
    if (!FLAT) load_splitters(splitters, index, spl, first);
    for (int i = threadIdx.x; i < NBK; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t nspan = (ntiles + span - 1) / span;
    // One CTA an SM, so nothing else hides a tile's load: the next tile's
    // bytes (one 16-byte word a thread, from the aligned addresses covering
    // them) are loaded into registers while the current tile is counted.
    auto fetch = [&](uint32_t t, uint4& w, uint32_t& shift, bool& fast) {
        const TileDesc td = tiles[t];
        const BlockInfo bi = blocks[td.blk];
        const uint32_t i0 = td.start - bi.off;
        const uintptr_t a = reinterpret_cast<uintptr_t>(S + bi.off + i0);
        const uintptr_t a0 = a & ~(uintptr_t)15;
        // the same test as stage_tile_bytes' vector path
        fast = (uint64_t)i0 + td.len + 7 + 16 <= bi.n && a0 >= reinterpret_cast<uintptr_t>(S);
        shift = (uint32_t)(a - a0);
        const uint32_t nvec = (shift + td.len + 7 + 15) >> 4;
        w = make_uint4(0, 0, 0, 0);
        if (FLAT && need[td.blk] == 0u) return;  // a tile that will be skipped: no bytes
        if (fast && threadIdx.x < nvec) w = __ldg(reinterpret_cast<const uint4*>(a0) + threadIdx.x);
    };
    static_assert((TILE_BYTES - 48) / 16 + 3 <= COUNT_THREADS, "one 16-byte word a thread covers a tile");
    __shared__ uint32_t s_any;
    for (uint32_t s = blockIdx.x; s < nspan; s += gridDim.x) {
        const uint32_t t0 = s * span, t1 = min(ntiles, t0 + span);
        if (FLAT) {  // whole spans of blocks the learned buckets fit are skipped, checked at once
            if (threadIdx.x == 0) s_any = 0u;
            __syncthreads();
            if (t0 + threadIdx.x < t1 && need[tiles[t0 + threadIdx.x].blk]) s_any = 1u;
            __syncthreads();
            const bool any = s_any != 0u;
            __syncthreads();  // every thread has read s_any before the next span resets it
            if (!any) continue;
        }
        uint32_t cur = tiles[t0].blk;
        uint4 w;
        uint32_t wshift;
        bool wfast;
        fetch(t0, w, wshift, wfast);
        for (uint32_t t = t0; t < t1; ++t) {
            const TileDesc td = tiles[t];
            if (td.blk != cur) {  // CTA-uniform; the histogram is complete (synced after the last tile)
                flush_counts(h, counts, nb, cur);
                cur = td.blk;
            }
            if (FLAT && need[td.blk] == 0u) {  // CTA-uniform: a block the learned buckets fit
                if (t + 1 < t1) fetch(t + 1, w, wshift, wfast);
                continue;
            }
            const BlockInfo bi = blocks[td.blk];
            uint32_t shift;
            if (wfast) {
                if (threadIdx.x < (wshift + td.len + 7 + 15) >> 4) reinterpret_cast<uint4*>(sb)[threadIdx.x] = w;
                shift = wshift;
            } else {
                shift = stage_tile_bytes(S, bi, td.start - bi.off, td.len, sb, threadIdx.x, blockDim.x);
            }
            __syncthreads();
            if (t + 1 < t1) fetch(t + 1, w, wshift, wfast);
            for (uint32_t q = threadIdx.x; q < td.len; q += blockDim.x) {
                const uint64_t key = pack8_smem(sb, shift + q);
                if (FLAT) {
                    atomicAdd(&h[(uint32_t)(key >> 52)], 1u << 16);
                } else {
                    const uint32_t b = bucket_of(spl, first, key);
                    fb[td.start + q] = (uint16_t)b;
                    atomicAdd(&h[b], 1u);
                }
            }
            __syncthreads();
        }
        flush_counts(h, counts, nb, cur);
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

// ---- two-level scatter -------------------------------------------------------
//
// Writing every rotation straight to its fine bucket scatters a tile over up
// to 4096 places (about one key each), so nearly every 12-byte write is a
// separate memory sector. Instead each block's consecutive fine buckets are
// grouped into chunks of at most CHUNK_CAP rotations (greedy, one warp per
// block); the scatter writes each tile's keys chunk by chunk in runs, and one
// CTA per chunk then sorts the whole chunk by (K, i) in shared memory and
// names it. A chunk is a union of whole fine buckets, and a fine bucket is a
// key interval, so a chunk holds every rotation of its key range: its first
// rotation starts a group and its last ends one, and naming needs nothing
// outside the chunk. A fine bucket larger than CHUNK_CAP is a chunk of its
// own: up to BIG_CAP rotations one CTA sorts it the same way (512 threads up
// to MID_CAP, 1,024 beyond; a
// model's over-full buckets are mostly a few thousand distinct keys), beyond
// that it goes to the overflow radix.
constexpr int MS_NT = 256;                           // threads of the chunk sort
constexpr int MS_IT = 13;                            // rotations per thread (odd: conflict-free strides)
constexpr uint32_t CHUNK_CAP = MS_NT * MS_IT;        // 3328
constexpr int BIG_NT = 1024;                         // threads of the big-chunk sort
constexpr uint32_t BIG_CAP = BIG_NT * MS_IT;         // 13312
constexpr int MID_NT = 512;                          // over-full buckets up to MID_CAP: 512 threads
constexpr uint32_t MID_CAP = MID_NT * MS_IT;         // 6656 (two such CTAs an SM)
constexpr uint32_t MAXCH = 1024;  // chunks per block (blocks above about 1.6 M rotations go plain)
constexpr uint32_t MAXB = 256;    // fine buckets per chunk (the chunk sort's bucket tables)

// A chunk is packed by padded sizes: a bucket of s rotations takes
// ceil(s / MS_IT) threads of the chunk sort (its team) and as many MS_IT-slot
// runs, so a chunk's teams fit the sort's threads.
__host__ __device__ constexpr uint32_t padded(uint32_t s) { return (s + MS_IT - 1) / MS_IT * MS_IT; }

// The scatter tags every rotation it writes into a packed chunk with the low
// 8 bits of its fine bucket (value bits 24..31; chunked blocks hold fewer
// than 2^24 rotations), and a chunk spans at most MAXB = 256 consecutive
// buckets, so the chunk sort reads each rotation's bucket in the chunk off
// its value. Over-capacity buckets, flagged CM_OWN in the chunk map, are
// written untagged.
constexpr uint16_t CM_OWN = 0x8000;
constexpr uint32_t TAG_SHIFT = 24, IDX_MASK = (1u << TAG_SHIFT) - 1u;

struct ChunkTables {
    uint16_t* cmap;        // [block][4096] chunk of each fine bucket (| CM_OWN: a bucket sorted on its own)
    uint32_t* cbase;       // [block][MAXCH] block-relative start of each chunk
    uint32_t* ccur;        // [block][MAXCH] slots taken by the scatter
};

__global__ void __launch_bounds__(256) k_chunk_plan(const uint32_t* __restrict__ starts,
                                                    const BlockInfo* __restrict__ blocks,
                                                    const uint32_t* __restrict__ route, uint32_t nb, ChunkTables ct,
                                                    Bins out, uint32_t* ctrl) {
    __shared__ uint32_t st[NBK + 1];
    __shared__ uint16_t cm[NBK];
    __shared__ uint32_t cb[MAXCH];
    __shared__ GroupDesc chunks[MAXCH];
    __shared__ uint32_t s_n[3];  // normal chunks to emit, overflow chunks to emit, chunks total
    for (uint32_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        if (route[blk] == 1u) continue;  // plain-routed (uniform across the CTA)
        const BlockInfo bi = blocks[blk];
        for (int i = threadIdx.x; i < NBK; i += blockDim.x) st[i] = starts[(size_t)blk * NBK + i];
        if (threadIdx.x == 0) st[NBK] = bi.n;
        __syncthreads();
        if (threadIdx.x < 32) {
            // Greedy packing by one warp, up to 32 buckets a step: the lanes
            // take the next 32 bucket sizes, an inclusive scan over them
            // (stopped at the first overflow bucket) shows how many still
            // fit in the open chunk, and those join it at once.
            const uint32_t lane = threadIdx.x;
            uint32_t nch = 0, nemit = 0, len = 0, plen = 0, cstart = 0, cb0 = 0, nbo = 0, b = 0;
            bool open = false;  // a chunk is open (possibly holding only empty buckets)
            auto close = [&]() {  // the open chunk, if it holds rotations, becomes chunk nch
                if (len > 0) {
                    if (lane == 0 && nch < MAXCH) {
                        cb[nch] = cstart;
                        // pad: the chunk's first fine bucket and its number of buckets
                        chunks[nemit] = GroupDesc{bi.off + cstart, len, blk, cb0 | (nbo << 16)};
                    }
                    if (nch < MAXCH) ++nemit;
                    ++nch;
                }
                open = false;
                len = plen = nbo = 0;
            };
            while (b < (uint32_t)NBK) {
                const uint32_t bb = b + lane;
                const uint32_t sz = bb < (uint32_t)NBK ? st[bb + 1] - st[bb] : 0xffffffffu;  // past the end: a stop
                const uint32_t bigm = __ballot_sync(0xffffffffu, sz > CHUNK_CAP);
                if (bigm & 1u) {  // bucket b is an overflow bucket: a chunk of its own, sorted by the radix path
                    close();
                    if (lane == 0) {
                        cm[b] = (uint16_t)(min(nch, MAXCH - 1) | CM_OWN);
                        if (nch < MAXCH) cb[nch] = st[b];
                        // the 512- or 1,024-thread sort, else the overflow radix
                        const int li = sz <= MID_CAP ? 2 : sz <= BIG_CAP ? 1 : CLS_LARGE;
                        const uint32_t slot = atomicAdd(&out.count[li], 1u);
                        if (slot < out.cap[li]) out.list[li][slot] = GroupDesc{bi.off + st[b], sz, blk, b | (1u << 16)};
                        else atomicOr(&ctrl[CTRL_ERR], ERR_CAPACITY);
                    }
                    ++nch;
                    ++b;
                    continue;
                }
                const uint32_t fb = bigm ? (uint32_t)(__ffs(bigm) - 1) : 32u;  // first stop lane (>= 1)
                uint32_t incl = lane < fb ? sz : 0u, pincl = lane < fb ? padded(sz) : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    const uint32_t py = __shfl_up_sync(0xffffffffu, pincl, o);
                    if ((int)lane >= o) {
                        incl += y;
                        pincl += py;
                    }
                }
                const bool fit = lane < fb && plen + pincl <= CHUNK_CAP && nbo + lane < MAXB;
                const uint32_t k = __popc(__ballot_sync(0xffffffffu, fit));  // fits are a prefix of the lanes
                if (k > 0) {
                    if (!open) {
                        open = true;
                        cstart = st[b];
                        cb0 = b;
                    }
                    if (lane < k) cm[b + lane] = (uint16_t)min(nch, MAXCH - 1);
                    len += __shfl_sync(0xffffffffu, incl, k - 1);
                    plen += __shfl_sync(0xffffffffu, pincl, k - 1);
                    nbo += k;
                    b += k;
                }
                // lane k stopped: an overflow bucket (handled next step) or a
                // bucket that does not fit (close, it opens the next chunk)
                if (k < 32 && b < (uint32_t)NBK && !((bigm >> k) & 1u)) close();
            }
            close();
            if (lane == 0) {
                if (nch > MAXCH) atomicOr(&ctrl[CTRL_ERR], ERR_CAPACITY);
                s_n[0] = nemit;
                s_n[1] = atomicAdd(&out.count[0], nemit);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < NBK; i += blockDim.x) ct.cmap[(size_t)blk * NBK + i] = cm[i];
        for (uint32_t i = threadIdx.x; i < MAXCH; i += blockDim.x) {
            ct.cbase[(size_t)blk * MAXCH + i] = cb[i];
            ct.ccur[(size_t)blk * MAXCH + i] = 0u;
        }
        for (uint32_t i = threadIdx.x; i < s_n[0]; i += blockDim.x) {
            const uint32_t slot = s_n[1] + i;
            if (slot < out.cap[0]) out.list[0][slot] = chunks[i];
            else atomicOr(&ctrl[CTRL_ERR], ERR_CAPACITY);
        }
        __syncthreads();
    }
}

// Scatters the tiles of bucketed blocks to their chunks. A CTA takes runs of
// consecutive tiles (up to 16, fewer when there are few tiles per CTA) (reloading the block's chunk map and chunk starts into
// shared memory when the block changes). A rotation's bucket is its stored
// learned bucket (fb) or, in blocks routed to equal-width buckets, its top 12
// key bits. Each tile is ranked by chunk in shared memory (tile-local
// positions and chunks only, 4 bytes a rotation; keys are re-packed from the
// staged bytes on the way out), so each chunk's share of the tile is written
// as one run, at a slot range reserved with one atomic per tile and chunk.
// Values written to packed chunks carry their bucket's tag (CM_OWN above).
constexpr size_t CHUNK_SCATTER_SMEM = NBK * 2 + 4 * MAXCH * 4 + TILE_BYTES + 4096 * 4;

template <int ITEMS>
__global__ void __launch_bounds__(256, 4) k_chunk_scatter(const uint8_t* __restrict__ S,
                                                       const BlockInfo* __restrict__ blocks,
                                                       const TileDesc* __restrict__ tiles,
                                                       const uint32_t* __restrict__ ntiles_dev,
                                                       const uint16_t* __restrict__ fb,
                                                       const uint32_t* __restrict__ route, ChunkTables ct,
                                                       uint64_t* __restrict__ K, uint32_t* __restrict__ I,
                                                       uint32_t* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint8_t* sb = smem;                                                  // [TILE_BYTES], 16-aligned
    uint16_t* cm = reinterpret_cast<uint16_t*>(smem + TILE_BYTES);       // [NBK] chunk of each bucket
    uint32_t* cb = reinterpret_cast<uint32_t*>(cm + NBK);                // [MAXCH] chunk starts (block-relative)
    uint32_t* lcount = cb + MAXCH;                                       // [MAXCH] tile's rotations per chunk
    uint32_t* pre = lcount + MAXCH;                                      // [MAXCH] tile-local chunk offsets
    uint32_t* dbase = pre + MAXCH;                                       // [MAXCH] destination of pre[c]
    uint32_t* stQC = dbase + MAXCH;  // [4096] by rank: tile position (low 16 bits) | fine bucket (high 16)
    __shared__ uint32_t scan_tmp[32];
    const uint32_t ntiles = *ntiles_dev;
    const uint32_t span = max(1u, min(16u, ntiles / (gridDim.x * 4u)));
    const uint32_t nspan = (ntiles + span - 1) / span;
    for (uint32_t s = blockIdx.x; s < nspan; s += gridDim.x) {
        const uint32_t t0 = s * span, t1 = min(ntiles, t0 + span);
        uint32_t cur = 0xffffffffu;
        BlockInfo bi{};     // of block cur, with its route: read once a block, so a
        bool flat = false;  // tile's loads wait only on its own descriptor
        for (uint32_t t = t0; t < t1; ++t) {
            const TileDesc td = tiles[t];
            if (td.blk != cur) {  // CTA-uniform
                cur = td.blk;
                bi = blocks[cur];
                flat = route[cur] == 2u;
                for (int i = threadIdx.x; i < NBK; i += blockDim.x) cm[i] = ct.cmap[(size_t)cur * NBK + i];
                for (int i = threadIdx.x; i < (int)MAXCH; i += blockDim.x) cb[i] = ct.cbase[(size_t)cur * MAXCH + i];
            }
            const uint32_t i0 = td.start - bi.off;
            for (int i = threadIdx.x; i < (int)MAXCH; i += blockDim.x) lcount[i] = 0;
            uint32_t bk[ITEMS];  // fine bucket of each item
            if (!flat) {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    const uint32_t q = j * 256 + threadIdx.x;
                    bk[j] = q < td.len ? (uint32_t)fb[td.start + q] : 0u;
                }
            }
            const uint32_t shift = stage_tile_bytes(S, bi, i0, td.len, sb, threadIdx.x, 256);
            __syncthreads();
            // chunk (low 10 bits) | slot within the tile's share of the chunk << 10;
            // every item's chunk is looked up before the first count, so the
            // lookups overlap
            uint32_t cs[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const uint32_t q = j * 256 + threadIdx.x;
                cs[j] = 0xffffffffu;
                if (q < td.len) {
                    if (flat) bk[j] = (uint32_t)(pack8_smem(sb, shift + q) >> 52);
                    cs[j] = cm[bk[j]] & (MAXCH - 1);
                }
            }
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (cs[j] != 0xffffffffu) cs[j] |= atomicAdd(&lcount[cs[j]], 1u) << 10;
            __syncthreads();
            // the global reservation (issued first: its round trip overlaps
            // the scan) and the tile-local exclusive prefix over chunks
            {
                constexpr int PER = MAXCH / 256;
                uint32_t v[PER], g[PER], sum = 0;
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    v[i] = lcount[threadIdx.x * PER + i];
                    g[i] = v[i] ? atomicAdd(&ct.ccur[(size_t)td.blk * MAXCH + threadIdx.x * PER + i], v[i]) : 0u;
                    sum += v[i];
                }
                uint32_t total;
                uint32_t ex = block_exclusive_scan<256>(sum, scan_tmp, &total);
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    const uint32_t c = threadIdx.x * PER + i;
                    pre[c] = ex;
                    if (v[i]) dbase[c] = bi.off + cb[c] + g[i];
                    ex += v[i];
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if (cs[j] != 0xffffffffu) {
                    const uint32_t c = cs[j] & (MAXCH - 1);
                    const uint32_t pos = pre[c] + (cs[j] >> 10);
                    stQC[pos] = (j * 256 + threadIdx.x) | (bk[j] << 16);
                }
            }
            __syncthreads();
            for (uint32_t r = threadIdx.x; r < td.len; r += blockDim.x) {
                const uint32_t qc = stQC[r], q = qc & 0xffffu, b = qc >> 16, e = cm[b], c = e & (MAXCH - 1);
                const uint32_t dst = dbase[c] + (r - pre[c]);
                BWT_DCHECK(dst - bi.off < bi.n, err);  // inside the tile's block
                K[dst] = pack8_smem(sb, shift + q);
                I[dst] = (i0 + q) | ((e & CM_OWN) ? 0u : (b & 0xffu) << TAG_SHIFT);
            }
            __syncthreads();
        }
    }
}

// (ak, ai) < (bk, bi) as an all-ones mask: the borrow out of the 96-bit
// difference ak:ai - bk:bi (the index is the low word), one carry chain
// instead of separate compares of the key halves and the index.
__device__ __forceinline__ uint32_t ki_less_mask(uint64_t ak, uint32_t ai, uint64_t bk, uint32_t bi) {
    uint32_t m;
    asm("{\n\t.reg .u32 t;\n\t"
        "sub.cc.u32 t, %1, %2;\n\t"
        "subc.cc.u32 t, %3, %4;\n\t"
        "subc.cc.u32 t, %5, %6;\n\t"
        "subc.u32 %0, 0, 0;\n\t}"
        : "=r"(m)
        : "r"(ai), "r"(bi), "r"((uint32_t)ak), "r"((uint32_t)bk), "r"((uint32_t)(ak >> 32)),
          "r"((uint32_t)(bk >> 32)));
    return m;
}

// Sorts a thread's MS_IT entries in registers by (K, i): Batcher's odd-even
// merge sorting network for 16 inputs with every comparator that touches
// slots 13..15 dropped (those slots would hold +infinity, which a comparator
// never moves to a lower slot), 48 compare-exchanges instead of the 78 of
// odd-even transposition (checked on every 0/1 input, which suffices for a
// network).
// The rows of a thread that lie in groups of two or more (bit j of mm: its
// row j, at chunk-relative position first + j): each gets its group's start
// as its rank (its rotation read from the compacted SA in sI), and each
// group that ends in these rows goes to the doubling rounds' bins and is
// counted into members[blk]. hm marks the rows that head a group, fm (bit
// j + 1) the rows that do not end one, cur0 is the last head + 1 before the
// thread's first row; the first `nreal` rows are real. All lanes of the warp
// call (the emitter's ballots).
template <int IT>
__device__ __noinline__ void name_chunk_members(WarpEmitter& em, const Bins& bins, uint32_t mm, uint32_t hm,
                                                uint32_t fm, uint32_t cur0, uint32_t first, uint32_t nreal,
                                                const uint32_t* sI, uint32_t* __restrict__ rank, BlockInfo bi,
                                                uint32_t boff, uint32_t gstart, uint32_t blk, uint32_t* members,
                                                uint32_t* err) {
    uint32_t cur = cur0;
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const uint32_t P = first + j;
        if ((uint32_t)j < nreal && ((hm >> j) & 1u)) cur = P + 1;
        const uint32_t gs = cur - 1;
        const bool member = (mm >> j) & 1u;
        if (member) {
            const uint32_t sa = sI[P] & ~SA_FINAL;
            BWT_DCHECK(sa < bi.n && cur > 0u, err);
            if (sa < bi.n) rank[bi.off + sa] = boff + gs;
        }
        const bool want = member && !((fm >> (j + 1)) & 1u);  // the group ends here
        if (want) atomicAdd(&members[blk], P - gs + 1);
        em.emit(bins, want, gstart + gs, P - gs + 1, blk, err);
    }
}

__device__ __forceinline__ void sort13(uint64_t (&k)[MS_IT], uint32_t (&v)[MS_IT]) {
    static_assert(MS_IT == 13, "the network below sorts 13 entries");
    constexpr int NET[48][2] = {
        {0, 1}, {2, 3}, {0, 2}, {1, 3}, {1, 2}, {4, 5}, {6, 7}, {4, 6}, {5, 7}, {5, 6}, {0, 4}, {2, 6}, {2, 4},
        {1, 5}, {3, 7}, {3, 5}, {1, 2}, {3, 4}, {5, 6}, {8, 9}, {10, 11}, {8, 10}, {9, 11}, {9, 10}, {8, 12},
        {10, 12}, {9, 10}, {11, 12}, {0, 8}, {4, 12}, {4, 8}, {2, 10}, {6, 10}, {2, 4}, {6, 8}, {10, 12}, {1, 9},
        {5, 9}, {3, 11}, {7, 11}, {3, 5}, {7, 9}, {1, 2}, {3, 4}, {5, 6}, {7, 8}, {9, 10}, {11, 12}};
#pragma unroll
    for (int c = 0; c < 48; ++c) {
        const int i = NET[c][0], j = NET[c][1];
        const bool sw = ki_less_mask(k[j], v[j], k[i], v[i]) != 0u;
        const uint64_t a = sw ? k[j] : k[i], b = sw ? k[i] : k[j];
        const uint32_t x = sw ? v[j] : v[i], y = sw ? v[i] : v[j];
        k[i] = a;
        k[j] = b;
        v[i] = x;
        v[j] = y;
    }
}

// One CTA per chunk: sort it by (K, i), write its SA, and name it (rank of
// every rotation = block-local start of its group; groups of size > 1 go to
// `bins` for the doubling rounds). NT threads sort chunks of up to
// NT * MS_IT rotations taken from chunks.list[LIST] (256 threads: the packed
// chunks; 1,024 threads: the single over-full buckets up to BIG_CAP).
//
// A chunk is a run of whole fine buckets, and a fine bucket is a key range,
// so the chunk is sorted bucket by bucket: no merge crosses a bucket edge.
//   1. The bucket table: every bucket's chunk-relative start (from the
//      block's scanned counts) and its team of ceil(size / MS_IT) threads
//      (an exclusive scan by one warp), whose run of team * MS_IT slots holds
//      the bucket, padded with entries above every real one.
//   2. Every rotation's bucket in the chunk, read off the tag its value
//      carries from the scatter, and a counting scatter into its bucket's
//      run (a shared-memory atomic a rotation).
//   3. Each thread sorts its MS_IT slots with the network; then merge
//      rounds inside each team (merge path; a team takes part in as many
//      rounds as it needs, ceil(log2(threads)): about 5 for learned buckets
//      of ~220 rotations, against 8 for the whole chunk at once).
//   4. SA is written compacted (the buckets in order, padding dropped),
//      and the chunk is named from the registers the last round left: the
//      ranks of group members are stored and their groups sent to the
//      doubling rounds; groups of one are marked SA_FINAL and their ranks
//      left to the on-demand lookup (LazyRanks), since nearly all rotations
//      of text blocks are told apart by their first 8 bytes. members[block]
//      counts the rotations sent on, which decides whether a block's ranks
//      are filled in full after the chunk sorts (k_fill_ranks).
// Padding entries are (~0, 0xffff0000 + slot): above every real pair (real
// indices are below 2^30) and distinct. A merge step reloads the head it
// consumed without a bounds test, so a head may sit one entry past its run
// (the other run, the next team's slots, or the 16 bytes of slack after the
// arrays); the choice tests the bounds and never takes such a head.
constexpr size_t CHUNK_SORT_SMEM = (size_t)CHUNK_CAP * 12 + 16;
constexpr size_t BIG_SORT_SMEM = (size_t)BIG_CAP * 12 + 16;
constexpr size_t MID_SORT_SMEM = (size_t)MID_CAP * 12 + 16;

template <int NT, int MINB, int LIST>
__global__ void __launch_bounds__(NT, MINB) k_chunk_sort_name(const uint64_t* __restrict__ K,
                                                              uint32_t* __restrict__ SA,
                                                              const BlockInfo* __restrict__ blocks, Bins chunks,
                                                              uint32_t* __restrict__ rank, Bins bins, uint32_t* ctrl,
                                                              uint32_t* __restrict__ chunk_counter,
                                                              const uint32_t* __restrict__ starts,
                                                              uint32_t* __restrict__ members) {
    constexpr uint32_t CAP = NT * MS_IT;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* sK = reinterpret_cast<uint64_t*>(smem);
    uint32_t* sI = reinterpret_cast<uint32_t*>(smem + (size_t)CAP * 8);
    __shared__ uint32_t bstart[MAXB + 1];  // chunk-relative start of every bucket (and the chunk's end)
    __shared__ uint32_t bthr[MAXB + 1];    // first thread of every bucket's team (and the threads used)
    __shared__ uint32_t bcur[MAXB];        // scatter cursors
    __shared__ GroupDesc ebuf[NT / 32][NCLS * EMIT_BUF];
    __shared__ uint64_t s_wlast[NT / 32], s_wfirst[NT / 32];  // each warp's last and first key
    __shared__ uint32_t s_wmax[NT / 32];                      // each warp's last head + 1
    __shared__ uint32_t s_c, s_rounds;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (ld_volatile(&ctrl[CTRL_ERR])) return;  // an earlier stage failed: the chunks are not permutations
    WarpEmitter em;
    em.init(ebuf[warp]);
    const uint32_t count = bin_count(chunks, LIST);
    // chunks in list order from an atomic counter (zeroed before the launch):
    // the chunks in flight stay within a few blocks, whose rank ranges stay
    // in L2 while their scattered rank writes land
    for (;;) {
        if (tid == 0) s_c = atomicAdd(chunk_counter, 1u);
        __syncthreads();
        const uint32_t c = s_c;
        if (c >= count) break;
        const GroupDesc gd = chunks.list[LIST][c];
        const BlockInfo bi = blocks[gd.blk];
        const uint32_t len = min(gd.len, CAP);
        const uint32_t b0 = gd.pad & 0xffffu, nbk = max(1u, min(gd.pad >> 16, MAXB));
        BWT_DCHECK(gd.len <= CAP && (gd.pad >> 16) >= 1u && (gd.pad >> 16) <= MAXB && b0 + nbk <= (uint32_t)NBK &&
                       gd.start - bi.off < bi.n && gd.start - bi.off + gd.len <= bi.n,
                   &ctrl[CTRL_ERR]);
        const uint32_t cstart = gd.start - bi.off;
        const uint32_t* srow = starts + (size_t)gd.blk * NBK;
        // ---- 1. the bucket table
        for (uint32_t j = tid; j <= nbk; j += NT) {
            const uint32_t st = j == nbk ? cstart + len : srow[min(b0 + j, (uint32_t)NBK - 1u)];
            bstart[j] = min(st - cstart, len);
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t run = 0, mx = 0;
            for (uint32_t j0 = 0; j0 < nbk; j0 += 32) {
                const uint32_t j = j0 + lane;
                const uint32_t sz = j < nbk ? bstart[j + 1] - bstart[j] : 0u;
                const uint32_t t = (sz + MS_IT - 1) / MS_IT;
                uint32_t incl = t;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if ((int)lane >= o) incl += y;
                }
                if (j < nbk) {
                    bthr[j] = run + incl - t;
                    bcur[j] = 0u;
                }
                mx = max(mx, t);
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) {
                bthr[nbk] = min(run, (uint32_t)NT);
                s_rounds = mx <= 1u ? 0u : 32u - __clz(mx - 1u);  // ceil(log2(largest team))
                BWT_DCHECK(run <= (uint32_t)NT, &ctrl[CTRL_ERR]);
            }
        }
        __syncthreads();
        const uint32_t T = bthr[nbk];
        // this thread's team: the last bucket whose team starts at or before it
        uint32_t team = 0;
        {
            uint32_t lo = 0, hi = nbk;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (bthr[mid] <= tid) lo = mid; else hi = mid;
            }
            team = lo;
        }
        const uint32_t tfirst = bthr[team], tsize = bstart[team + 1] - bstart[team];
        const uint32_t lt = tid - tfirst;             // index inside the team
        const uint32_t kteam = bthr[team + 1] - tfirst;  // threads of the team
        const bool active = tid < T;
        // ---- 2. loads (all in flight together), buckets, counting scatter
        uint64_t k[MS_IT];
        uint32_t v[MS_IT];
#pragma unroll
        for (int j = 0; j < MS_IT; ++j) {
            const uint32_t i = j * NT + tid;
            k[j] = i < len ? K[gd.start + i] : 0ull;
            v[j] = i < len ? SA[gd.start + i] : 0u;
        }
        if (active && lt + 1 == kteam) {  // the padding: only a team's last thread has any
#pragma unroll
            for (int j = 0; j < MS_IT; ++j) {
                const uint32_t pos = lt * MS_IT + j;  // position inside the team's run
                if (pos >= tsize) {
                    const uint32_t slot = tid * MS_IT + j;
                    sK[slot] = ~0ull;
                    sI[slot] = 0xffff0000u + slot;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < MS_IT; ++j) {
            const uint32_t i = j * NT + tid;
            const bool valid = i < len;
            uint32_t lb = 0xffffffffu;
            if (valid) {
                // packed chunks: the bucket tag; a bucket of its own: untagged
                lb = LIST == 0 ? ((v[j] >> TAG_SHIFT) - b0) & 0xffu : 0u;
                v[j] &= IDX_MASK;
                BWT_DCHECK(lb < nbk && v[j] < bi.n, &ctrl[CTRL_ERR]);
                lb = min(lb, nbk - 1);
            }
            if (valid) {  // any order inside the run: the sort decides it
                const uint32_t slot = min(bthr[lb] * MS_IT + atomicAdd(&bcur[lb], 1u), CAP - 1u);
                sK[slot] = k[j];
                sI[slot] = v[j];
            }
        }
        __syncthreads();
        // ---- 3. sorting network on this thread's slots, then merge rounds inside the team
        const uint32_t R = s_rounds;
        if (active) {
#pragma unroll
            for (int j = 0; j < MS_IT; ++j) {
                k[j] = sK[tid * MS_IT + j];
                v[j] = sI[tid * MS_IT + j];
            }
            sort13(k, v);
        }
        for (uint32_t r = 1; r <= R; ++r) {
            // a team whose runs already form one sorted run sits the round out
            const bool merging = active && (1u << (r - 1)) < kteam;
            if (merging) {  // the sorted runs of the previous step back in place
#pragma unroll
                for (int j = 0; j < MS_IT; ++j) {
                    sK[tid * MS_IT + j] = k[j];
                    sI[tid * MS_IT + j] = v[j];
                }
            }
            __syncthreads();
            if (merging) {
                const uint32_t m = 1u << r;  // threads per merged run
                const uint32_t pf = lt & ~(m - 1u);
                const uint32_t w = (m >> 1) * MS_IT;  // input run length
                const uint32_t L = kteam * MS_IT;
                const uint32_t a0 = pf * MS_IT, a1 = min(a0 + w, L), b1 = min(a0 + 2u * w, L);
                const uint32_t la = a1 - a0, lb = b1 - a1;
                const uint32_t diag = (lt - pf) * MS_IT;
                const uint64_t* AK = sK + tfirst * MS_IT + a0;
                const uint32_t* AI = sI + tfirst * MS_IT + a0;
                const uint64_t* BK = AK + la;
                const uint32_t* BI = AI + la;
                uint32_t lo = diag > lb ? diag - lb : 0u, hi = min(diag, la);
                while (lo < hi) {  // A entries among the first diag outputs (A first on ties)
                    const uint32_t mid = (lo + hi) >> 1;
                    const uint64_t a = AK[mid], b = BK[diag - 1 - mid];
                    const bool a_first = a != b ? a < b : AI[mid] <= BI[diag - 1 - mid];
                    if (a_first) lo = mid + 1; else hi = mid;
                }
                // heads may sit one past their run (valid shared memory: the
                // other run, the next team, or the slack entry after the
                // arrays); the bounds in the choice keep them out
                uint32_t ia = lo, ib = diag - lo;
                uint64_t ka = AK[ia], kb = BK[ib];
                uint32_t va = AI[ia], vb = BI[ib];
#pragma unroll
                for (int j = 0; j < MS_IT; ++j) {
                    const bool take_b = ib < lb && (ia >= la || ki_less_mask(kb, vb, ka, va) != 0u);
                    k[j] = take_b ? kb : ka;
                    v[j] = take_b ? vb : va;
                    if (take_b) {
                        ++ib;
                        kb = BK[ib];
                        vb = BI[ib];
                    } else {
                        ++ia;
                        ka = AK[ia];
                        va = AI[ia];
                    }
                }
            }
            __syncthreads();
        }
        if (R == 0) __syncthreads();  // every thread has read its slots before any compacted write
        // ---- 4. naming, from the registers. A rotation heads a group where
        //      its key differs from the one before it (a bucket's first
        //      rotation always does: a bucket is a key range); it ends one
        //      where the next key differs or its bucket ends. Its group start
        //      is the last head at or before it: inside the thread by a
        //      running value, across threads by a CTA max-scan of every
        //      thread's last head.
        const uint32_t base = bstart[team];  // the team's bucket, chunk-relative
        uint64_t prev_last = __shfl_up_sync(0xffffffffu, k[MS_IT - 1], 1);
        uint64_t next_first = __shfl_down_sync(0xffffffffu, k[0], 1);
        if (lane == 31) s_wlast[warp] = k[MS_IT - 1];
        if (lane == 0) s_wfirst[warp] = k[0];
        __syncthreads();
        if (lane == 0 && warp > 0) prev_last = s_wlast[warp - 1];
        if (lane == 31 && warp + 1 < NT / 32) next_first = s_wfirst[warp + 1];
        const bool emit_ok = bi.n > 8u;   // smaller blocks: every group is final (whole equal rotations)
        uint32_t hm = 0, fm = 0, mm = 0, lh = 0;  // head, not-last and member bits, last head + 1 (0: none)
        if (active) {
#pragma unroll
            for (int j = 0; j < MS_IT; ++j) {
                const uint32_t pos = lt * MS_IT + j;
                if (pos < tsize) {
                    const uint64_t before = j == 0 ? prev_last : k[j > 0 ? j - 1 : 0];
                    const uint64_t after = j == MS_IT - 1 ? next_first : k[j < MS_IT - 1 ? j + 1 : 0];
                    const bool head = pos == 0 || k[j] != before;
                    const bool tail = pos + 1 == tsize || k[j] != after;
                    if (head) {
                        hm |= 1u << j;
                        lh = base + pos + 1;
                    }
                    if (!tail) fm |= 2u << j;  // bit j + 1: not the group's last row
                    const bool final_row = (head && tail) || !emit_ok;
                    if (!final_row) mm |= 1u << j;  // in a group of two or more, sent to the rounds
                    // SA, compacted through shared memory (bucket after bucket,
                    // padding dropped) for a coalesced write
                    sI[base + pos] = v[j] | (final_row ? SA_FINAL : 0u);
                }
            }
        }
        // the barrier also tells whether the chunk holds a group of two or more
        const bool any_member = __syncthreads_or(mm != 0u) != 0;
        for (uint32_t i = tid; i < len; i += NT) SA[gd.start + i] = sI[i];
        if (any_member) {  // CTA-uniform; rare on text
            // group starts: the last head at or before each row, by a CTA
            // max-scan of every thread's last head
            uint32_t incl = lh;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl = max(incl, y);
            }
            if (lane == 31) s_wmax[warp] = incl;
            __syncthreads();
            uint32_t cur = __shfl_up_sync(0xffffffffu, incl, 1);
            if (lane == 0) cur = 0u;
            for (uint32_t w = 0; w < warp; ++w) cur = max(cur, s_wmax[w]);
            // groups of two or more: their ranks stored and the groups sent
            // to the doubling rounds, by a call taken only by warps that
            // hold a member
            if (__any_sync(0xffffffffu, mm != 0u))
                name_chunk_members<MS_IT>(em, bins, mm, hm, fm, cur, base + lt * MS_IT,
                                          active ? tsize - min(tsize, lt * MS_IT) : 0u, sI, rank, bi,
                                          gd.start - bi.off, gd.start, gd.blk, members, &ctrl[CTRL_ERR]);
        }
        __syncthreads();
    }
    em.finish(bins, &ctrl[CTRL_ERR]);
}

// After the chunk sorts: a bucketed block whose chunk sorts sent more than
// 1/32 of its rotations to the doubling rounds has the ranks of its groups
// of one stored here (rank[SA] = row for the rows marked SA_FINAL), since its
// rounds would read many of them; its other ranks are already stored. Such
// blocks and plain-routed ones read ranks directly (lazy = 0); the others
// find them on demand. One CTA per block.
__global__ void __launch_bounds__(256) k_fill_ranks(const BlockInfo* __restrict__ blocks, uint32_t nb,
                                                    const uint32_t* __restrict__ route,
                                                    const uint32_t* __restrict__ members,
                                                    const uint32_t* __restrict__ SA, uint32_t* __restrict__ rank,
                                                    uint32_t* __restrict__ lazy) {
    for (uint32_t blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        const BlockInfo bi = blocks[blk];
        const bool bucketed = route[blk] != 1u;
        const bool fill = bucketed && (uint64_t)members[blk] * 32u > bi.n;
        if (threadIdx.x == 0) lazy[blk] = bucketed && !fill ? 1u : 0u;
        if (!fill) continue;
        for (uint32_t q = threadIdx.x; q < bi.n; q += blockDim.x) {
            const uint32_t x = SA[bi.off + q];
            const uint32_t r = x & ~SA_FINAL;
            if ((x & SA_FINAL) && r < bi.n) rank[bi.off + r] = q;
        }
    }
}

// Blocks routed to equal-width buckets (route 2) take their equal-width row
// as their bucket row.
__global__ void k_select_rows(uint32_t* __restrict__ counts, const uint32_t* __restrict__ route, uint32_t nb) {
    for (uint32_t blk = blockIdx.x; blk < nb; blk += gridDim.x)
        if (route[blk] == 2u)
            for (int i = threadIdx.x; i < NBK; i += blockDim.x)
                counts[(size_t)blk * NBK + i] = counts[((size_t)nb + blk) * NBK + i];
}

// need[b] = 1 for the blocks whose learned over-capacity buckets hold more
// than a quarter of the block (and that are not too large to chunk): the
// ones whose equal-width counts the routing has to see.
__global__ void k_flat_needed(const unsigned long long* __restrict__ bstats, const BlockInfo* __restrict__ blocks,
                              uint32_t nb, uint32_t* __restrict__ need) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        need[b] = bstats[5 * (size_t)b] * 4 > blocks[b].n ? 1u : 0u;
}

// Routes every block and numbers its tiles in its route's tile table, in one
// CTA: route 0 (learned buckets) if the learned over-capacity buckets hold at
// most a quarter of the block, else 2 (equal-width buckets) if those do, else
// 1 (plain radix); blocks too large for the chunk tables go plain. first:
// [2][block] first tile of the block in the plain table and in the bucketed
// table; the two table sizes go to ctrl[CTRL_AUX0] and ctrl[CTRL_AUX1].
__global__ void __launch_bounds__(1024) k_route_scan(const unsigned long long* __restrict__ bstats,
                                                     const BlockInfo* __restrict__ blocks, uint32_t nb, uint32_t tile,
                                                     uint32_t* __restrict__ route, uint32_t* __restrict__ first,
                                                     uint32_t* ctrl) {
    __shared__ uint32_t tmp[32];
    uint32_t run_p = 0, run_b = 0;
    for (uint32_t base = 0; base < nb; base += 1024) {
        const uint32_t b = base + threadIdx.x;
        uint32_t np = 0, nbk = 0;
        if (b < nb) {
            const uint64_t n = blocks[b].n;
            const unsigned long long* bl = bstats + 5 * (size_t)b;
            const unsigned long long* bf = bstats + 5 * ((size_t)nb + b);
            // chunks are packed by padded sizes (at most 12 slots of padding a
            // bucket) and close early at most NBK / MAXB times for the bucket
            // limit, so a block of n rotations needs at most
            // 2 (n + 12 NBK) / CHUNK_CAP + NBK / MAXB + 1 chunks
            const bool too_big = (n + 12ull * NBK) * 2 > (uint64_t)(MAXCH - NBK / MAXB - 2) * CHUNK_CAP;
            const uint32_t r = too_big ? 1u : bl[0] * 4 <= n ? 0u : bf[0] * 4 <= n ? 2u : 1u;
            route[b] = r;
            const uint32_t nt = (uint32_t)((n + tile - 1) / tile);
            if (r == 1u) np = nt; else nbk = nt;
        }
        uint32_t tot_p, tot_b;
        const uint32_t ep = block_exclusive_scan<1024>(np, tmp, &tot_p);
        const uint32_t eb = block_exclusive_scan<1024>(nbk, tmp, &tot_b);
        if (b < nb) {
            first[b] = run_p + ep;
            first[nb + b] = run_b + eb;
        }
        run_p += tot_p;
        run_b += tot_b;
    }
    if (threadIdx.x == 0) {
        ctrl[CTRL_AUX0] = run_p;
        ctrl[CTRL_AUX1] = run_b;
    }
}

// Copies every first-sort tile into its block's route table (plain, or
// bucketed), with its first-tile index relative to that table.
__global__ void k_route_tiles(const TileDesc* __restrict__ tiles0, uint32_t ntiles0, uint32_t nb,
                              const uint32_t* __restrict__ route, const uint32_t* __restrict__ first,
                              TileDesc* __restrict__ tiles_p, TileDesc* __restrict__ tiles_b) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles0; t += gridDim.x * blockDim.x) {
        TileDesc td = tiles0[t];
        const uint32_t b = td.blk;
        const bool plain = route[b] == 1u;
        const uint32_t f = plain ? first[b] : first[nb + b];
        const uint32_t dst = f + (t - td.firstTile);
        td.firstTile = f;
        (plain ? tiles_p : tiles_b)[dst] = td;
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
                const uint32_t peers = match_label<9>(d);
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
    if (!p->splitter_index) CKL(cudaMalloc(&p->splitter_index, sizeof(uint16_t) * IDX_WORDS));
    if (!p->bucket_count) CKL(cudaMalloc(&p->bucket_count, sizeof(uint32_t) * 2 * nbk));
    if (!p->bucket_cursor) CKL(cudaMalloc(&p->bucket_cursor, sizeof(uint32_t) * nbk));
    if (!p->chunk_map) CKL(cudaMalloc(&p->chunk_map, sizeof(uint16_t) * nbk));
    if (!p->chunk_base) CKL(cudaMalloc(&p->chunk_base, sizeof(uint32_t) * nbk));
    if (!p->route) CKL(cudaMalloc(&p->route, sizeof(uint32_t) * p->cap_b));
    if (!p->route_first) CKL(cudaMalloc(&p->route_first, sizeof(uint32_t) * 2 * p->cap_b));
    if (!p->members) CKL(cudaMalloc(&p->members, sizeof(uint32_t) * p->cap_b));
    if (!p->lazy) CKL(cudaMalloc(&p->lazy, sizeof(uint32_t) * p->cap_b));
    if (!p->bstats) CKL(cudaMalloc(&p->bstats, sizeof(unsigned long long) * 10 * p->cap_b));
    if (!p->tiles_aux) CKL(cudaMalloc(&p->tiles_aux, sizeof(TileDesc) * 2 * (size_t)p->cap_tiles0));
    if (!p->splitters_flat) {
        std::vector<uint64_t> flat(NSP);
        for (int j = 0; j < NSP; ++j) flat[j] = (uint64_t)(j + 1) << 52;  // bucket = top 12 key bits
        CKL(cudaMalloc(&p->splitters_flat, sizeof(uint64_t) * NSP));
        CKL(cudaMemcpy(p->splitters_flat, flat.data(), sizeof(uint64_t) * NSP, cudaMemcpyHostToDevice));
    }
    if (!p->h_route) {
        CKL(cudaMallocHost(&p->h_route, sizeof(uint32_t) * p->cap_b));
        CKL(cudaHostGetDevicePointer((void**)&p->hd_route, p->h_route, 0));
    }
    if (!p->h_bstats) {
        CKL(cudaMallocHost(&p->h_bstats, sizeof(unsigned long long) * 10 * p->cap_b));
        CKL(cudaHostGetDevicePointer((void**)&p->hd_bstats, p->h_bstats, 0));
    }
    // kernel attributes and occupancy: set up here, outside any stream capture
    static const int sort_ctas = [] {
        cudaFuncSetAttribute((void*)k_bucket_count<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)COUNT_SMEM);
        cudaFuncSetAttribute((void*)k_bucket_count<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)COUNT_SMEM);
        cudaFuncSetAttribute((void*)k_chunk_sort_name<MS_NT, 4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)CHUNK_SORT_SMEM);
        cudaFuncSetAttribute((void*)k_chunk_sort_name<BIG_NT, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BIG_SORT_SMEM);
        cudaFuncSetAttribute((void*)k_chunk_sort_name<MID_NT, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)MID_SORT_SMEM);
        int per_sm = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chunk_sort_name<MS_NT, 4, 0>, MS_NT,
                                                      CHUNK_SORT_SMEM);
        return std::max(1, per_sm);
    }();
    p->chunk_sort_ctas = sort_ctas;
    return BWT_OK;
}

bwt_status bwt::build_splitter_index(bwt_plan* p) {
    k_build_index<<<(IDX_WORDS + 255) / 256, 256>>>(p->splitters, p->splitter_index);
    CKL(cudaGetLastError());
    CKL(cudaStreamSynchronize(0));
    return BWT_OK;
}

bwt_status bwt::enqueue_learned(bwt_plan* p, const uint8_t* d_in, cudaStream_t st) {
    const uint32_t nb = p->nb, nt = p->ntiles0;
    const int sms = num_sms();
    uint32_t* ctrl = p->ctrl;
    const uint32_t T = (uint32_t)p->tile;
    p->sa = p->vals[0];
    p->key2 = p->vals[1];
    p->kA = reinterpret_cast<uint32_t*>(p->keys[1]);
    p->vA = p->kA + p->cap_n;
    p->kB = reinterpret_cast<uint32_t*>(p->keys[0]);
    p->vB = p->kB + p->cap_n;

    // 1. count the learned bucketing per block and store every rotation's
    //    learned bucket (in the u16 view of keys[1], free until the scatter
    //    has run), then the equal-width bucketing of the blocks the learned
    //    buckets do not fit, 2. per-block statistics of both, 3. route every
    //    block and split the tile table by route -- all on the device
    NvtxStages nv;
    nv.next("bucket_count");
    uint16_t* fb = reinterpret_cast<uint16_t*>(p->keys[1]);
    CKL(cudaMemsetAsync(p->bucket_count, 0, sizeof(uint32_t) * 2 * NBK * nb, st));
    {
        const uint32_t span_max = 65535u / T;  // packed 16-bit counts per span
        const uint32_t span = std::max(1u, std::min(span_max, nt / (uint32_t)(sms * 4)));
        const int grid = std::max(1, std::min<int>((nt + span - 1) / span, sms));
        k_bucket_count<false><<<grid, COUNT_THREADS, COUNT_SMEM, st>>>(
            d_in, p->blocks, p->tiles0, nt, span, p->splitters, p->splitter_index, nb, p->bucket_count, fb, nullptr);
        k_bucket_stats<<<std::min<uint32_t>(nb, 65535), 256, 0, st>>>(p->bucket_count, CHUNK_CAP, nb, p->bstats);
        // the equal-width counts, only where the learned buckets do not fit
        // (route[] holds the flags until the routing overwrites it)
        k_flat_needed<<<(nb + 255) / 256, 256, 0, st>>>(p->bstats, p->blocks, nb, p->route);
        k_bucket_count<true><<<grid, COUNT_THREADS, COUNT_SMEM, st>>>(
            d_in, p->blocks, p->tiles0, nt, span, p->splitters, p->splitter_index, nb, p->bucket_count, fb, p->route);
        k_bucket_stats<<<std::min<uint32_t>(nb, 65535), 256, 0, st>>>(p->bucket_count + (size_t)nb * NBK, CHUNK_CAP,
                                                                      nb, p->bstats + 5 * (size_t)nb);
    }
    nv.next("bucket_route");
    k_route_scan<<<1, 1024, 0, st>>>(p->bstats, p->blocks, nb, T, p->route, p->route_first, ctrl);
    TileDesc* tilesP = p->tiles_aux;
    TileDesc* tilesB = p->tiles_aux + p->cap_tiles0;
    k_route_tiles<<<std::max(1, std::min<int>((nt + 255) / 256, sms * 4)), 256, 0, st>>>(
        p->tiles0, nt, nb, p->route, p->route_first, tilesP, tilesB);
    CKL(cudaGetLastError());
    // for the statistics, read after the call (written by kernels: a memcpy
    // node here would wait behind any large copy queued on the same engine
    // by another stream, and stall the whole call with it)
    CKL(launch_words_to_host(p->hd_bstats, reinterpret_cast<const uint32_t*>(p->bstats), 20 * nb, st));
    CKL(launch_words_to_host(p->hd_route, p->route, nb, st));
    p->stats.kernel_launches += 9;
    const uint32_t* ntp = ctrl + CTRL_AUX0;
    const uint32_t* ntb = ctrl + CTRL_AUX1;

    // 4a. bucketed blocks: bucket starts, chunk plan and scatter (the scatter
    //     consumes fb, so it runs before the plain passes reuse keys[1])
    nv.next("bucket_scatter");
    Bins aux = bins_of(p, 1);
    CKL(cudaMemsetAsync(aux.count, 0, sizeof(uint32_t) * NCLS, st));
    k_select_rows<<<std::min<uint32_t>(nb, 65535), 256, 0, st>>>(p->bucket_count, p->route, nb);
    CKL(launch_scan_rows(p->bucket_count, NBK, nullptr, 0, nb, nb, st));  // counts -> starts in place
    ChunkTables ct{p->chunk_map, p->chunk_base, p->bucket_cursor};
    k_chunk_plan<<<std::min<uint32_t>(nb, 65535), 256, 0, st>>>(p->bucket_count, p->blocks, p->route, nb, ct, aux,
                                                                ctrl);
    {
        const int g = sms * 4;
        if (T <= 1024)
            k_chunk_scatter<4><<<g, 256, CHUNK_SCATTER_SMEM, st>>>(d_in, p->blocks, tilesB, ntb, fb, p->route, ct,
                                                                   p->keys[0], p->vals[0], ctrl + CTRL_ERR);
        else if (T <= 2048)
            k_chunk_scatter<8><<<g, 256, CHUNK_SCATTER_SMEM, st>>>(d_in, p->blocks, tilesB, ntb, fb, p->route, ct,
                                                                   p->keys[0], p->vals[0], ctrl + CTRL_ERR);
        else
            k_chunk_scatter<16><<<g, 256, CHUNK_SCATTER_SMEM, st>>>(d_in, p->blocks, tilesB, ntb, fb, p->route, ct,
                                                                    p->keys[0], p->vals[0], ctrl + CTRL_ERR);
    }
    CKL(cudaGetLastError());
    p->stats.kernel_launches += 4;

    // 4b. plain-routed blocks: the first sort of the plain path, ending in
    //     buffer 0, and its naming (with no plain-routed block every kernel
    //     here finds zero tiles and returns). Their tile table is only known
    //     on the device, so with 16-bit digits (whose part table is built on
    //     the host) they take 8-bit onesweep passes.
    nv.next("bucket_plain");
    const int rb = p->rbits == 16 ? 8 : p->rbits, RADIX = 1 << rb;
    const uint32_t status_cap = (uint32_t)std::min<uint64_t>(p->cap_status, 0xffffffffu);
    {
        const int P = (64 + rb - 1) / rb;
        uint32_t seg_stride;
        if (rb == 8) {
            CKL(cudaMemsetAsync(p->hist, 0, sizeof(uint32_t) * 256 * nb, st));
            CKL(launch_hist_bytes(d_in, p->blocks, tilesP, 0, p->hist, st, ntp));
            CKL(launch_scan_rows(p->hist, 256, nullptr, 0, nb, nb, st));
            seg_stride = 256;
        } else {
            CKL(cudaMemsetAsync(p->hist, 0, sizeof(uint32_t) * 6 * 2048 * nb, st));
            CKL(launch_hist_keys11(d_in, p->blocks, tilesP, 0, p->tile, p->hist, st, ntp));
            CKL(launch_scan_rows(p->hist, 2048, nullptr, 0, nb * 6, nb * 6, st));
            seg_stride = 6 * 2048;
        }
        p->stats.kernel_launches += 2;
        for (int ps = 0; ps < P; ++ps) {
            CKL(launch_zero_by_count(p->status, ntp, (uint32_t)RADIX, status_cap, st));
            OneSweepParams a{};
            const int out = (P - 1 - ps) & 1, in = (P - ps) & 1;
            a.kin = ps == 0 ? nullptr : p->keys[in];
            a.vin = ps == 0 ? nullptr : p->vals[in];
            a.kout = p->keys[out];
            a.vout = p->vals[out];
            a.S = d_in;
            a.blocks = p->blocks;
            a.tiles = tilesP;
            a.num_tiles = ntp;
            a.seg_base = p->hist + (rb == 8 ? 0 : ps * 2048);
            a.seg_base_stride = seg_stride;
            a.status = p->status;
            a.tile_counter = ctrl + CTRL_TILE_CTR + ps;
            a.ctrl = ctrl;
            a.shift = ps * rb;
            CKL(launch_onesweep(8, ps == 0, rb, p->tile, a, 0, st));
            p->stats.kernel_launches += 2;
            p->stats.radix_launches++;
        }
        CKL(launch_name_tiles(p->keys[0], p->vals[0], p->blocks, tilesP, ntp, false, p->rank, bins_of(p, 0), ctrl,
                              st));
        p->stats.kernel_launches++;
    }

    // 4c. bucketed blocks: chunk sorts with naming, then the overflow buckets
    nv.next("bucket_sort");
    uint32_t* chunk_counter = ctrl + CTRL_TILE_CTR + 58;  // control words no radix pass uses
    uint32_t* big_counter = ctrl + CTRL_TILE_CTR + 59;
    uint32_t* mid_counter = ctrl + CTRL_TILE_CTR + 50;  // no radix pass of a learned call uses it either
    CKL(cudaMemsetAsync(chunk_counter, 0, 8, st));
    CKL(cudaMemsetAsync(mid_counter, 0, 4, st));
    CKL(cudaMemsetAsync(p->members, 0, sizeof(uint32_t) * nb, st));
    const bool timing = !p->events.empty() && !p->capturing && p->ev_used + 2 <= p->events.size();
    if (timing) CKL(cudaEventRecord(p->events[p->ev_used], st));
    k_chunk_sort_name<MS_NT, 4, 0><<<sms * p->chunk_sort_ctas, MS_NT, CHUNK_SORT_SMEM, st>>>(
        p->keys[0], p->vals[0], p->blocks, aux, p->rank, bins_of(p, 0), ctrl, chunk_counter, p->bucket_count,
        p->members);
    CKL(cudaGetLastError());
    if (timing) {
        CKL(cudaEventRecord(p->events[p->ev_used + 1], st));
        EvMeta m{};
        m.ctrl_word = -1;
        m.chunk_sort = true;
        p->ev_meta.push_back(m);
        p->ev_used += 2;
    }
    // over-full buckets: one CTA each, 512 threads up to MID_CAP (two an SM)
    // and 1,024 up to BIG_CAP
    k_chunk_sort_name<MID_NT, 2, 2><<<2 * sms, MID_NT, MID_SORT_SMEM, st>>>(p->keys[0], p->vals[0], p->blocks, aux,
                                                                            p->rank, bins_of(p, 0), ctrl, mid_counter,
                                                                            p->bucket_count, p->members);
    k_chunk_sort_name<BIG_NT, 1, 1><<<sms, BIG_NT, BIG_SORT_SMEM, st>>>(p->keys[0], p->vals[0], p->blocks, aux,
                                                                        p->rank, bins_of(p, 0), ctrl, big_counter,
                                                                        p->bucket_count, p->members);
    CKL(cudaGetLastError());
    p->stats.kernel_launches += 4;

    // overflow buckets: radix on the index, then on the key
    nv.next("bucket_overflow");
    const int PI = std::max(1, (bits_needed(p->max_n - 1) + 7) / 8), PK = 8, PT = PI + PK;
    CKL(launch_build_large_tiles(aux, p->tile, p->ltiles, p->cap_ltiles, ctrl, st));
    CKL(launch_zero_by_count(p->hist, aux.count + CLS_LARGE, (uint32_t)(PT * 256),
                             (uint32_t)std::min<uint64_t>(p->cap_hist, 0xffffffffu), st));
    k_seg_hist_u64<<<sms * 4, 256, PT * 256 * 4, st>>>(p->keys[0], p->vals[0], p->ltiles, ctrl + CTRL_NUM_LTILES,
                                                       p->hist, PI, PK);
    CKL(cudaGetLastError());
    CKL(launch_scan_rows(p->hist, 256, aux.count + CLS_LARGE, (uint32_t)PT, 0, (uint32_t)(p->cap_hist / 256), st));
    p->stats.kernel_launches += 4;
    for (int ps = 0; ps < PT; ++ps) {
        CKL(launch_zero_by_count(p->status, ctrl + CTRL_NUM_LTILES, 256u, status_cap, st));
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
    }
    if (PT & 1) {
        k_copy_tiles<<<sms * 4, 256, 0, st>>>(p->keys[1], p->vals[1], p->keys[0], p->vals[0], p->ltiles,
                                              ctrl + CTRL_NUM_LTILES);
        CKL(cudaGetLastError());
        p->stats.kernel_launches++;
    }
    // overflow buckets are whole key ranges too: name them inside their own bounds
    CKL(launch_name_tiles(p->keys[0], p->vals[0], p->blocks, p->ltiles, ctrl + CTRL_NUM_LTILES, true, p->rank,
                          bins_of(p, 0), ctrl, st));
    p->stats.kernel_launches++;
    p->learned_overflow_passes = (uint32_t)PT;

    // 4d. ranks: blocks with many group members get every rank stored; the
    //     rest find the ranks of their groups of one on demand
    nv.next("bucket_ranks");
    k_fill_ranks<<<std::min<uint32_t>(nb, 65535), 256, 0, st>>>(p->blocks, nb, p->route, p->members, p->vals[0],
                                                                p->rank, p->lazy);
    CKL(cudaGetLastError());
    p->stats.kernel_launches++;
    LazyRanks lz;
    lz.lazy = p->lazy;
    lz.S = d_in;
    lz.SA = p->vals[0];
    lz.route = p->route;
    lz.starts = p->bucket_count;
    lz.splitters = p->splitters;
    lz.index = p->splitter_index;
    lz.own_cap = BIG_CAP;
    p->lazy_ranks = lz;
    return BWT_OK;
}

void bwt::learned_stats(bwt_plan* p) {
    const uint32_t nb = p->nb;
    const int rb = p->rbits == 16 ? 8 : p->rbits;  // the plain-routed blocks' digit width
    const int P = (64 + rb - 1) / rb;
    for (uint32_t b = 0; b < nb; ++b) {
        const unsigned long long* bl = p->h_bstats + 5 * (size_t)b;
        const unsigned long long* bf = p->h_bstats + 5 * ((size_t)nb + b);
        const uint32_t r = p->h_route[b];
        p->stats.max_bucket = std::max<uint32_t>(p->stats.max_bucket, (uint32_t)bl[2]);
        p->stats.bucket_sq_sum += bl[3];
        p->stats.buckets_nonempty += bl[4];
        if (r == 1u) {
            p->stats.blocks_routed_plain++;
            p->stats.radix_keys += (uint64_t)P * p->h_blocks[b].n;
        } else {
            const unsigned long long* bs = r == 2u ? bf : bl;
            if (r == 2u) p->stats.blocks_routed_flat++;
            p->stats.buckets_overflowed += bs[1];
            p->stats.keys_overflowed += bs[0];
            p->stats.chunk_keys += p->h_blocks[b].n - bs[0];
        }
    }
    p->stats.chunk_bytes = 16.0 * (double)p->stats.chunk_keys;
    p->stats.radix_keys += (uint64_t)p->learned_overflow_passes * p->stats.keys_overflowed;
}

// Host-driven learned mode: the learned first stage, then doubling rounds
// driven from the host, then the L gather.
bwt_status bwt::run_learned(bwt_plan* p, const uint8_t* d_in, uint8_t* d_L, int32_t* d_primary, cudaStream_t st) {
    if (!p->have_model) return BWT_ENOMODEL;
    bwt_status s;
    if ((s = ensure_learned_buffers(p)) != BWT_OK) return s;
    if ((s = reset_ctrl(p, st)) != BWT_OK) return s;
    if ((s = enqueue_learned(p, d_in, st)) != BWT_OK) return s;
    if ((s = run_doubling_host_loop(p, st)) != BWT_OK) return s;
    CKL(launch_gather_L(d_in, p->sa, p->blocks, p->tiles0, p->ntiles0, d_L, d_primary, p->ctrl, st));
    p->stats.kernel_launches++;
    return BWT_OK;
}
