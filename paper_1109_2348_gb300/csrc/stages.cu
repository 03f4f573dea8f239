// Run-length encoding and decoding of a batch (Section 3.2, Fig. 1 and
// Fig. 2 of the paper; the method of Fang et al. it describes).
//
// Encode: a byte ends a run if the next byte differs or starts another block
// (runs never cross blocks); an exclusive prefix sum of these flags gives
// every run its output slot; the run's byte and its end index (global, one
// past the last byte) go to that slot; a run's length is the difference of
// consecutive end indices. Decode: the inclusive prefix sum of the lengths
// gives every run's end; flags at the last byte of every run, prefix-summed
// over the output, give every output byte its run; the byte is copied.
//
// Variable-length encoding (Section 3.4, Fig. 3; the substitution method of
// Balevic it describes): every byte is looked up in a codeword table, the
// exclusive prefix sum of the codeword lengths gives every codeword's first
// bit, and the codewords are written there (most significant bit first;
// each block's stream starts at a byte boundary).
//
// Move-to-front encoding (Section 3.3): the paper's parallelism is over
// the list -- its 256 entries are spread over a warp's lanes, 8 a lane (kept
// as every value's position, so a byte's position is one shuffle away and
// the move is one byte-wise compare-and-add per lane). A block's bytes form one chain of list states, so blocks are cut
// into chunks: a chunk's effect on the list is the chunk's distinct bytes
// in order of last occurrence, followed by the old list without them. Pass
// 1 finds that list for every chunk, pass 2 chains the chunks of every
// block to get each chunk's starting list, pass 3 encodes all chunks at
// once.
//
// GB300 layout: the prefix sums are single passes over 4,096-element tiles
// (256 threads x 16) with decoupled look-back between tiles, so each of the
// steps reads and writes every element once; tiles start in order from a
// tile counter. A tile's codewords are packed into 32-bit words in shared
// memory and stored whole; only the two words a tile shares with its
// neighbours are merged with atomic ORs.
#include <algorithm>
#include <cstring>

#include "bwt.h"
#include "kernels.h"
#include "plan_internal.h"

using namespace bwt;

#define CKS(call)                                              \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return record_cuda(_e, #call);  \
    } while (0)

namespace {

constexpr int RT = 256;                 // threads per tile
constexpr int RI = 16;                  // elements per thread
constexpr uint32_t RTILE = RT * RI;     // 4096

// Block holding global position i (blocks are contiguous and cover the batch).
__device__ __forceinline__ uint32_t block_at(const BlockInfo* blocks, uint32_t nb, uint32_t i) {
    uint32_t lo = 0, hi = nb;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (blocks[mid].off <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t next_tile(uint32_t* s_tile, uint32_t* counter) {
    if (threadIdx.x == 0) *s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t t = *s_tile;
    __syncthreads();
    return t;
}

// Encode steps 1-3: run-end flags, their prefix sum, and the scatter of
// (byte, end index) to the run's slot. run_off[b] = the first run of block b
// (run_off[nb] = the number of runs).
__global__ void __launch_bounds__(RT) k_rle_encode(const uint8_t* __restrict__ S, uint32_t N,
                                                   const BlockInfo* __restrict__ blocks, uint32_t nb,
                                                   uint8_t* __restrict__ chars, uint32_t* __restrict__ ends,
                                                   uint64_t* __restrict__ run_off, uint64_t* __restrict__ status,
                                                   uint32_t* __restrict__ counter, uint32_t* ctrl) {
    __shared__ __align__(16) uint8_t sb[RTILE + 16];
    __shared__ uint32_t s_tile, scan_tmp[32];
    __shared__ uint64_t s_excl;
    const uint32_t ntiles = (N + RTILE - 1) / RTILE;
    const uint32_t spin = ctrl[CTRL_SPIN], withhold = ctrl[CTRL_WITHHOLD];
    for (;;) {
        const uint32_t t = next_tile(&s_tile, counter);
        if (t >= ntiles) break;
        const uint32_t t0 = t * RTILE, len = min(RTILE, N - t0);
        for (uint32_t q = threadIdx.x; q < len + 1 && t0 + q < N; q += RT) sb[q] = S[t0 + q];
        __syncthreads();
        const uint32_t q0 = threadIdx.x * RI, i0 = t0 + q0;
        uint32_t flags = 0;  // bit j: element q0 + j ends a run
        uint32_t b = i0 < N ? block_at(blocks, nb, i0) : 0u;
        {
            uint32_t bend = i0 < N ? blocks[b].off + blocks[b].n : 0u, bb = b;
#pragma unroll
            for (int j = 0; j < RI; ++j) {
                const uint32_t i = i0 + j;
                if (i >= N) break;
                while (i >= bend) {
                    ++bb;
                    bend = blocks[bb].off + blocks[bb].n;
                }
                const bool end = i + 1 == N || i + 1 == bend || sb[q0 + j + 1] != sb[q0 + j];
                flags |= (uint32_t)end << j;
            }
        }
        uint32_t total;
        const uint32_t pre = block_exclusive_scan<RT>(__popc(flags), scan_tmp, &total);
        if (threadIdx.x < 32) {
            const uint64_t e = lookback_u64(status, t, 0, total, spin, &ctrl[CTRL_ERR], withhold);
            if (threadIdx.x == 0) s_excl = e;
        }
        __syncthreads();
        uint64_t k = s_excl + pre;
#pragma unroll
        for (int j = 0; j < RI; ++j) {
            const uint32_t i = i0 + j;
            if (i >= N) break;
            while (b + 1 < nb && blocks[b + 1].off <= i) ++b;
            if (blocks[b].off == i) run_off[b] = k;  // runs before the block's first byte
            if ((flags >> j) & 1u) {
                if (k < N) {
                    chars[k] = sb[q0 + j];
                    ends[k] = i + 1;
                }
                ++k;
            }
            if (i + 1 == N) run_off[nb] = k;
        }
        __syncthreads();
    }
}

// Encode step 4: run lengths from consecutive end indices.
__global__ void k_rle_lengths(const uint32_t* __restrict__ ends, const uint64_t* __restrict__ run_off, uint32_t nb,
                              uint32_t* __restrict__ lens) {
    const uint64_t R = run_off[nb];
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < R; k += (uint64_t)gridDim.x * blockDim.x)
        lens[k] = ends[k] - (k ? ends[k - 1] : 0u);
}

// Decode step 1: B[k] = end of run k (inclusive prefix sum of the lengths,
// global). A zero length is an input error.
__global__ void __launch_bounds__(RT) k_rle_scan(const uint32_t* __restrict__ lens, const uint64_t* __restrict__ run_off,
                                                 uint32_t nb, uint32_t N, uint32_t* __restrict__ B,
                                                 uint64_t* __restrict__ status,
                                                 uint32_t* __restrict__ counter, uint32_t* ctrl) {
    __shared__ uint32_t s_tile, scan_tmp[32];
    __shared__ uint64_t s_excl;
    const uint64_t R = min(run_off[nb], (uint64_t)N);  // a run holds at least one byte
    const uint32_t ntiles = (uint32_t)((R + RTILE - 1) / RTILE);
    const uint32_t spin = ctrl[CTRL_SPIN], withhold = ctrl[CTRL_WITHHOLD];
    for (;;) {
        const uint32_t t = next_tile(&s_tile, counter);
        if (t >= ntiles) break;
        const uint64_t k0 = (uint64_t)t * RTILE + threadIdx.x * RI;
        uint32_t v[RI], sum = 0;
#pragma unroll
        for (int j = 0; j < RI; ++j) {
            v[j] = k0 + j < R ? lens[k0 + j] : 0u;
            if (k0 + j < R && v[j] == 0u) atomicOr(&ctrl[CTRL_ERR], ERR_INPUT);
            sum += v[j];
        }
        uint32_t total;
        const uint32_t pre = block_exclusive_scan<RT>(sum, scan_tmp, &total);
        if (threadIdx.x < 32) {
            const uint64_t e = lookback_u64(status, t, 0, total, spin, &ctrl[CTRL_ERR], withhold);
            if (threadIdx.x == 0) s_excl = e;
        }
        __syncthreads();
        uint64_t acc = s_excl + pre;
#pragma unroll
        for (int j = 0; j < RI; ++j) {
            acc += v[j];
            if (k0 + j < R) B[k0 + j] = (uint32_t)acc;
        }
        __syncthreads();
    }
}

// Decode check: every block's runs end exactly at the block's end.
__global__ void k_rle_check(const uint32_t* __restrict__ B, const uint64_t* __restrict__ run_off,
                            const BlockInfo* __restrict__ blocks, uint32_t nb, uint32_t cap, uint32_t* ctrl) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const uint64_t r0 = run_off[b], r1 = run_off[b + 1];
        const bool ok = (b > 0 || r0 == 0) && r1 > r0 && r1 <= cap && B[r1 - 1] == blocks[b].off + blocks[b].n;
        if (!ok) atomicOr(&ctrl[CTRL_ERR], ERR_INPUT);
    }
}

// Decode steps 2-4 for one output tile: flags at the last byte of every run
// that ends in the tile, their exclusive prefix sum = the run of every byte
// (after the runs that end before the tile), and the copy of the run's byte.
__global__ void __launch_bounds__(RT) k_rle_expand(const uint8_t* __restrict__ chars, const uint32_t* __restrict__ B,
                                                   const uint64_t* __restrict__ run_off, uint32_t nb, uint32_t N,
                                                   uint8_t* __restrict__ out) {
    __shared__ uint8_t sflag[RTILE];
    __shared__ uint32_t s_k0, scan_tmp[32];
    const uint64_t R = min(run_off[nb], (uint64_t)N);
    if (R == 0) return;  // no runs: the check has flagged the input
    const uint32_t ntiles = (N + RTILE - 1) / RTILE;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t t0 = t * RTILE, len = min(RTILE, N - t0);
        for (uint32_t q = threadIdx.x; q < RTILE; q += RT) sflag[q] = 0;
        if (threadIdx.x == 0) {  // first run ending after t0: runs before it end at or before t0
            uint64_t lo = 0, hi = R;
            while (lo < hi) {
                const uint64_t mid = (lo + hi) >> 1;
                if (B[mid] <= t0) lo = mid + 1; else hi = mid;
            }
            s_k0 = (uint32_t)lo;
        }
        __syncthreads();
        const uint32_t k0 = s_k0;
        for (uint32_t x = threadIdx.x; x < len; x += RT) {  // at most len runs end inside the tile
            const uint64_t k = (uint64_t)k0 + x;
            if (k >= R) break;
            const uint32_t e = B[k];
            if (e - 1 - t0 >= len) break;  // ends after the tile (B increases)
            sflag[e - 1 - t0] = 1;
        }
        __syncthreads();
        const uint32_t q0 = threadIdx.x * RI;
        uint32_t f[RI], cnt = 0;
#pragma unroll
        for (int j = 0; j < RI; ++j) {
            f[j] = q0 + j < len ? sflag[q0 + j] : 0u;
            cnt += f[j];
        }
        uint32_t total;
        uint32_t r = block_exclusive_scan<RT>(cnt, scan_tmp, &total);
#pragma unroll
        for (int j = 0; j < RI; ++j) {
            if (q0 + j >= len) break;
            const uint64_t k = min((uint64_t)k0 + r, R - 1);
            out[t0 + q0 + j] = chars[k];
            r += f[j];
        }
        __syncthreads();
    }
}

// ---- variable-length encoding ------------------------------------------------

// Bits of every block's stream (sum of its bytes' codeword lengths). A byte
// whose codeword length is outside 1..32 is an input error.
__global__ void __launch_bounds__(RT) k_vle_bits(const uint8_t* __restrict__ S, const TileDesc* __restrict__ tiles,
                                                 uint32_t ntiles, const uint8_t* __restrict__ len,
                                                 unsigned long long* __restrict__ block_bits, uint32_t* ctrl) {
    __shared__ uint8_t slen[256];
    __shared__ uint32_t red[RT / 32];
    slen[threadIdx.x] = len[threadIdx.x];
    __syncthreads();
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileDesc td = tiles[t];
        uint32_t sum = 0;
        for (uint32_t q = threadIdx.x; q < td.len; q += RT) {
            const uint32_t l = slen[S[td.start + q]];
            if (l == 0u || l > 32u) atomicOr(&ctrl[CTRL_ERR], ERR_INPUT);
            sum += l;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < RT / 32; ++w) tot += red[w];
            atomicAdd(&block_bits[td.blk], (unsigned long long)tot);
        }
        __syncthreads();
    }
}

// 64-bit block-wide exclusive scan (1024 threads).
__device__ __forceinline__ unsigned long long scan64_1024(unsigned long long v, unsigned long long* tmp,
                                                          unsigned long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = tmp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        tmp[lane] = w;
    }
    __syncthreads();
    const unsigned long long r = (warp ? tmp[warp - 1] : 0ull) + x - v;
    *total = tmp[31];
    __syncthreads();
    return r;
}

// Byte offsets of the block streams (exclusive scan of ceil(bits / 8)); the
// total goes to byte_off[nb]. The buffer must hold the total rounded up to
// whole 32-bit words. One CTA.
__global__ void __launch_bounds__(1024) k_vle_offsets(const unsigned long long* __restrict__ block_bits, uint32_t nb,
                                                      uint64_t cap, uint64_t* __restrict__ byte_off, uint32_t* ctrl) {
    __shared__ unsigned long long tmp[32];
    unsigned long long run = 0;  // the same in every thread
    for (uint32_t base = 0; base < nb; base += 1024) {
        const uint32_t b = base + threadIdx.x;
        const unsigned long long bytes = b < nb ? (block_bits[b] + 7) / 8 : 0ull;
        unsigned long long tot;
        const unsigned long long ex = scan64_1024(bytes, tmp, &tot);
        if (b < nb) byte_off[b] = run + ex;
        run += tot;
    }
    if (threadIdx.x == 0) {
        byte_off[nb] = run;
        if ((run + 3) / 4 * 4 > cap) atomicOr(&ctrl[CTRL_ERR], ERR_CAPACITY);
    }
}

// Zeroes the output words [0, ceil(byte_off[nb] / 4)) that lie inside the
// buffer (partial words at the end are merged by atomic OR, so they need it).
__global__ void k_vle_zero(uint32_t* __restrict__ out32, const uint64_t* __restrict__ byte_off, uint32_t nb,
                           uint64_t cap_words) {
    const uint64_t words = min((byte_off[nb] + 3) / 4, cap_words);
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x)
        out32[w] = 0u;
}

// Packs every tile's codewords: bit offsets inside the block by a block
// scan plus look-back over the block's earlier tiles, words assembled in
// shared memory (stream bit j of a word is bit 31 - j, stored byte-swapped so
// that memory order is stream order), interior words stored, edge words
// OR-ed. out32 is the output viewed as 32-bit words (4-byte aligned).
constexpr uint32_t VLE_WORDS = RTILE + 2;  // a tile spans at most 4096 * 32 bits + alignment

__global__ void __launch_bounds__(RT) k_vle_pack(const uint8_t* __restrict__ S, const TileDesc* __restrict__ tiles,
                                                 uint32_t ntiles, const uint32_t* __restrict__ code,
                                                 const uint8_t* __restrict__ len, const uint64_t* __restrict__ byte_off,
                                                 uint64_t cap_words, uint32_t* __restrict__ out32,
                                                 uint64_t* __restrict__ status, uint32_t* __restrict__ counter,
                                                 uint32_t* ctrl) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* words = reinterpret_cast<uint32_t*>(smem);           // [VLE_WORDS]
    uint32_t* scode = words + VLE_WORDS;                           // [256]
    uint8_t* slen = reinterpret_cast<uint8_t*>(scode + 256);       // [256]
    __shared__ uint32_t s_tile, scan_tmp[32];
    __shared__ uint64_t s_excl;
    scode[threadIdx.x] = code[threadIdx.x];
    slen[threadIdx.x] = len[threadIdx.x];
    const uint32_t spin = ctrl[CTRL_SPIN], withhold = ctrl[CTRL_WITHHOLD];
    if (ld_volatile(&ctrl[CTRL_ERR]) & (ERR_INPUT | ERR_CAPACITY)) return;  // bad table or too small a buffer
    for (;;) {
        const uint32_t t = next_tile(&s_tile, counter);
        if (t >= ntiles) break;
        const TileDesc td = tiles[t];
        const uint32_t q0 = threadIdx.x * RI;
        uint32_t lsum = 0;
        uint32_t c[RI];
        uint8_t l[RI];
#pragma unroll
        for (int j = 0; j < RI; ++j) {
            const uint32_t q = q0 + j;
            l[j] = 0;
            c[j] = 0;
            if (q < td.len) {
                const uint8_t x = S[td.start + q];
                l[j] = slen[x];
                c[j] = scode[x];
                lsum += l[j];
            }
        }
        uint32_t total;
        const uint32_t pre = block_exclusive_scan<RT>(lsum, scan_tmp, &total);
        if (threadIdx.x < 32) {
            const uint64_t e = lookback_u64(status, t, td.firstTile, total, spin, &ctrl[CTRL_ERR], withhold);
            if (threadIdx.x == 0) s_excl = e;
        }
        for (uint32_t w = threadIdx.x; w < VLE_WORDS; w += RT) words[w] = 0u;
        __syncthreads();
        const uint64_t g0 = byte_off[td.blk] * 8 + s_excl;  // first bit of the tile
        const uint64_t w0 = g0 >> 5;
        uint64_t g = g0 + pre;
#pragma unroll
        for (int j = 0; j < RI; ++j) {
            const uint32_t L = l[j];
            if (L) {
                const uint32_t cw = L == 32u ? c[j] : (c[j] & ((1u << L) - 1u));
                const uint32_t x = (uint32_t)(g - (w0 << 5));  // bit offset inside the tile's words
                const uint32_t wi = x >> 5, sh = x & 31u;       // codeword bits [sh, sh + L) of word wi
                if (sh + L <= 32u) {
                    atomicOr(&words[wi], cw << (32u - sh - L));
                } else {
                    const uint32_t rest = sh + L - 32u;          // bits spilling into word wi + 1
                    atomicOr(&words[wi], cw >> rest);
                    atomicOr(&words[wi + 1], cw << (32u - rest));
                }
                g += L;
            }
        }
        __syncthreads();
        const uint32_t nwords = (uint32_t)(((g0 + total + 31) >> 5) - w0);
        for (uint32_t x = threadIdx.x; x < nwords; x += RT) {
            const uint64_t w = w0 + x;
            if (w >= cap_words) break;
            const uint32_t v = __byte_perm(words[x], 0, 0x0123);
            if (x == 0 || x + 1 == nwords) atomicOr(&out32[w], v);
            else out32[w] = v;
        }
        __syncthreads();
    }
}

// ---- move-to-front encoding ---------------------------------------------------

// Pass 1: per chunk (a first-sort tile), its distinct bytes ordered by last
// occurrence, most recent first: mru[chunk][0 .. mcnt[chunk]).
__global__ void __launch_bounds__(RT) k_mtf_mru(const uint8_t* __restrict__ S, const TileDesc* __restrict__ tiles,
                                                uint32_t ntiles, uint8_t* __restrict__ mru,
                                                uint32_t* __restrict__ mcnt) {
    __shared__ int32_t last[256];
    __shared__ uint8_t sb[RTILE];
    __shared__ uint32_t s_cnt;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileDesc td = tiles[t];
        last[threadIdx.x] = -1;
        if (threadIdx.x == 0) s_cnt = 0;
        for (uint32_t q = threadIdx.x; q < td.len; q += RT) sb[q] = S[td.start + q];
        __syncthreads();
        const uint32_t q0 = threadIdx.x * RI;
        for (int j = RI - 1; j >= 0; --j) {  // the last occurrence inside this thread's range only
            const uint32_t q = q0 + j;
            if (q >= td.len) continue;
            const uint8_t x = sb[q];
            bool later = false;
            for (int k = j + 1; k < RI && q0 + k < td.len; ++k) later |= sb[q0 + k] == x;
            if (!later) atomicMax(&last[x], (int32_t)q);
        }
        __syncthreads();
        const int32_t mine = last[threadIdx.x];
        if (mine >= 0) {
            uint32_t rank = 0;
            for (int u = 0; u < 256; ++u) rank += last[u] > mine;
            mru[(size_t)t * 256 + rank] = (uint8_t)threadIdx.x;
            atomicAdd(&s_cnt, 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) mcnt[t] = s_cnt;
        __syncthreads();
    }
}

// Pass 2: one warp per block chains its chunks: the list before chunk c
// goes to tlist[c]; the next list is mru[c] followed by the list without
// mru[c]'s bytes. A lane holds list entries 8 lane .. 8 lane + 7 (byte k of
// its 64-bit word is entry 8 lane + k).
__global__ void __launch_bounds__(256) k_mtf_chain(const uint32_t* __restrict__ tfirst, uint32_t nb,
                                                   const uint8_t* __restrict__ mru, const uint32_t* __restrict__ mcnt,
                                                   uint8_t* __restrict__ tlist) {
    __shared__ uint32_t member[8][8];
    __shared__ __align__(8) uint8_t nlist[8][256];
    const uint32_t lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    for (uint32_t b = blockIdx.x * 8 + wl; b < nb; b += gridDim.x * 8) {
        uint64_t L = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) L |= (uint64_t)(lane * 8 + k) << (8 * k);
        for (uint32_t c = tfirst[b]; c < tfirst[b + 1]; ++c) {
            reinterpret_cast<uint64_t*>(tlist + (size_t)c * 256)[lane] = L;
            if (lane < 8) member[wl][lane] = 0u;
            __syncwarp();
            const uint32_t cnt = mcnt[c];
            const uint8_t* m = mru + (size_t)c * 256;
            for (uint32_t i = lane; i < cnt; i += 32) {
                const uint32_t v = m[i];
                atomicOr(&member[wl][v >> 5], 1u << (v & 31));
                nlist[wl][i] = (uint8_t)v;
            }
            __syncwarp();
            uint32_t keep = 0;  // bit k: entry 8 lane + k stays (not among the chunk's bytes)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t v = (uint32_t)(L >> (8 * k)) & 0xffu;
                keep |= (uint32_t)(((member[wl][v >> 5] >> (v & 31)) & 1u) == 0u) << k;
            }
            uint32_t n = __popc(keep), x = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            uint32_t pos = cnt + x - n;
            (void)lt;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if ((keep >> k) & 1u) nlist[wl][pos++] = (uint8_t)(L >> (8 * k));
            __syncwarp();
            L = reinterpret_cast<const uint64_t*>(nlist[wl])[lane];
            __syncwarp();
        }
    }
}

// Pass 3: one warp per chunk encodes it from its starting list. The warp
// keeps every byte value's position in the list instead of the list itself:
// lane l holds the positions of values 8 l .. 8 l + 7, one byte each. Byte x
// at position p: output p; every position below p moves up by one (a byte-
// wise compare and add on the lane's two words) and x's becomes 0. A byte
// already at the front costs one compare. The chunk sits in the warp's
// shared buffer and every byte is replaced there by its position.
constexpr int MTF_WARPS = 8;

__global__ void __launch_bounds__(MTF_WARPS * 32) k_mtf_encode(const uint8_t* __restrict__ S,
                                                               const TileDesc* __restrict__ tiles, uint32_t ntiles,
                                                               const uint8_t* __restrict__ tlist,
                                                               uint8_t* __restrict__ out) {
    __shared__ __align__(16) uint8_t buf[MTF_WARPS][RTILE];
    __shared__ __align__(16) uint8_t posb[MTF_WARPS][256];
    const uint32_t lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    uint8_t* bw = buf[wl];
    for (uint32_t t = blockIdx.x * MTF_WARPS + wl; t < ntiles; t += gridDim.x * MTF_WARPS) {
        const TileDesc td = tiles[t];
        for (uint32_t q = lane; q < td.len; q += 32) bw[q] = S[td.start + q];
        const uint8_t* T = tlist + (size_t)t * 256;  // starting list: T[j] = value at position j
        for (uint32_t j = lane; j < 256; j += 32) posb[wl][T[j]] = (uint8_t)j;
        __syncwarp();
        uint32_t lo = reinterpret_cast<const uint32_t*>(posb[wl])[2 * lane];      // positions of 8 l .. 8 l + 3
        uint32_t hi = reinterpret_cast<const uint32_t*>(posb[wl])[2 * lane + 1];  // positions of 8 l + 4 .. 8 l + 7
        uint32_t front = T[0];
        __syncwarp();
        for (uint32_t i = 0; i < td.len; ++i) {
            const uint32_t x = bw[i];
            if (x == front) {  // warp-uniform: x and front are the same in every lane
                if (lane == 0) bw[i] = 0;
                continue;
            }
            const uint32_t owner = x >> 3, k = x & 7u;
            const uint32_t word = __shfl_sync(0xffffffffu, k < 4 ? lo : hi, owner);
            const uint32_t p = (word >> (8 * (k & 3))) & 0xffu;
            const uint32_t p4 = p * 0x01010101u;
            lo += __vcmpltu4(lo, p4) & 0x01010101u;  // positions below p move up (they stay <= 255)
            hi += __vcmpltu4(hi, p4) & 0x01010101u;
            if (lane == owner) {
                const uint32_t clear = ~(0xffu << (8 * (k & 3)));
                if (k < 4) lo &= clear; else hi &= clear;
            }
            if (lane == 0) bw[i] = (uint8_t)p;
            front = x;
        }
        __syncwarp();
        for (uint32_t q = lane; q < td.len; q += 32) out[td.start + q] = bw[q];
        __syncwarp();
    }
}

}  // namespace

extern "C" bwt_status bwt_rle_encode(bwt_plan* p, const uint8_t* d_in, const uint64_t* offsets, uint32_t num_blocks,
                                     uint8_t* d_chars, uint32_t* d_lens, uint64_t* d_run_off, void* stream) {
    if (!p || !d_in || !offsets || !d_chars || !d_lens || !d_run_off) return BWT_EINVAL;
    bwt::NvtxRange nvtx_range("rle_encode");
    if (cudaSetDevice(p->device) != cudaSuccess) return BWT_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::memset(&p->stats, 0, sizeof(p->stats));
    bwt_status s = prepare_batch(p, offsets, num_blocks, st);
    if (s != BWT_OK) return p->last = s;
    if ((s = reset_ctrl(p, st)) != BWT_OK) return p->last = s;
    const uint32_t N = p->total, nt = (N + RTILE - 1) / RTILE;
    uint64_t* status = reinterpret_cast<uint64_t*>(p->status);
    CKS(cudaMemsetAsync(status, 0, sizeof(uint64_t) * nt, st));
    uint32_t* ends = p->vals[0];
    const int sms = num_sms();
    k_rle_encode<<<std::max(1, std::min<int>(nt, sms * 8)), RT, 0, st>>>(
        d_in, N, p->blocks, p->nb, d_chars, ends, d_run_off, status, p->ctrl + CTRL_TILE_CTR, p->ctrl);
    k_rle_lengths<<<sms * 8, 256, 0, st>>>(ends, d_run_off, p->nb, d_lens);
    CKS(cudaGetLastError());
    p->stats.kernel_launches = 3;
    return p->last = finish_status(p, st);
}

extern "C" bwt_status bwt_rle_decode(bwt_plan* p, const uint8_t* d_chars, const uint32_t* d_lens,
                                     const uint64_t* d_run_off, const uint64_t* offsets, uint32_t num_blocks,
                                     uint8_t* d_out, void* stream) {
    if (!p || !d_chars || !d_lens || !d_run_off || !offsets || !d_out) return BWT_EINVAL;
    bwt::NvtxRange nvtx_range("rle_decode");
    if (cudaSetDevice(p->device) != cudaSuccess) return BWT_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::memset(&p->stats, 0, sizeof(p->stats));
    bwt_status s = prepare_batch(p, offsets, num_blocks, st);
    if (s != BWT_OK) return p->last = s;
    if ((s = reset_ctrl(p, st)) != BWT_OK) return p->last = s;
    const uint32_t N = p->total, nt = (N + RTILE - 1) / RTILE;  // runs <= N, so <= nt tiles of runs
    uint64_t* status = reinterpret_cast<uint64_t*>(p->status);
    CKS(cudaMemsetAsync(status, 0, sizeof(uint64_t) * nt, st));
    uint32_t* B = p->vals[0];
    const int sms = num_sms();
    k_rle_scan<<<std::max(1, std::min<int>(nt, sms * 8)), RT, 0, st>>>(d_lens, d_run_off, p->nb, N, B, status,
                                                                     p->ctrl + CTRL_TILE_CTR, p->ctrl);
    k_rle_check<<<std::max(1u, std::min<uint32_t>((p->nb + 255) / 256, 1024)), 256, 0, st>>>(B, d_run_off, p->blocks,
                                                                                          p->nb, N, p->ctrl);
    k_rle_expand<<<std::max(1, std::min<int>(nt, sms * 8)), RT, 0, st>>>(d_chars, B, d_run_off, p->nb, N, d_out);
    CKS(cudaGetLastError());
    p->stats.kernel_launches = 4;
    return p->last = finish_status(p, st);
}

extern "C" bwt_status bwt_vle_encode(bwt_plan* p, const uint8_t* d_in, const uint64_t* offsets, uint32_t num_blocks,
                                     const uint32_t* d_code, const uint8_t* d_len, uint8_t* d_out, uint64_t out_cap,
                                     uint64_t* d_byte_off, uint64_t* d_block_bits, void* stream) {
    if (!p || !d_in || !offsets || !d_code || !d_len || !d_out || !d_byte_off || !d_block_bits) return BWT_EINVAL;
    bwt::NvtxRange nvtx_range("vle_encode");
    if ((reinterpret_cast<uintptr_t>(d_out) & 3u) != 0) return BWT_EINVAL;  // written as 32-bit words
    if (cudaSetDevice(p->device) != cudaSuccess) return BWT_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::memset(&p->stats, 0, sizeof(p->stats));
    bwt_status s = prepare_batch(p, offsets, num_blocks, st);
    if (s != BWT_OK) return p->last = s;
    if ((s = reset_ctrl(p, st)) != BWT_OK) return p->last = s;
    const uint32_t nb = p->nb, nt = p->ntiles0;
    if (p->tile > (int)RTILE) return p->last = BWT_EINVAL;
    static bool attr = [] {
        cudaFuncSetAttribute((void*)k_vle_pack, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(VLE_WORDS * 4 + 256 * 5));
        return true;
    }();
    (void)attr;
    const int sms = num_sms();
    unsigned long long* bits = reinterpret_cast<unsigned long long*>(d_block_bits);
    CKS(cudaMemsetAsync(bits, 0, sizeof(uint64_t) * nb, st));
    k_vle_bits<<<std::max(1, std::min<int>(nt, sms * 8)), RT, 0, st>>>(d_in, p->tiles0, nt, d_len, bits, p->ctrl);
    k_vle_offsets<<<1, 1024, 0, st>>>(bits, nb, out_cap, d_byte_off, p->ctrl);
    const uint64_t cap_words = out_cap / 4;  // whole words inside the buffer
    k_vle_zero<<<sms * 8, 256, 0, st>>>(reinterpret_cast<uint32_t*>(d_out), d_byte_off, nb, cap_words);
    uint64_t* status = reinterpret_cast<uint64_t*>(p->status);
    CKS(cudaMemsetAsync(status, 0, sizeof(uint64_t) * nt, st));
    k_vle_pack<<<std::max(1, std::min<int>(nt, sms * 6)), RT, VLE_WORDS * 4 + 256 * 5, st>>>(
        d_in, p->tiles0, nt, d_code, d_len, d_byte_off, cap_words, reinterpret_cast<uint32_t*>(d_out), status,
        p->ctrl + CTRL_TILE_CTR, p->ctrl);
    CKS(cudaGetLastError());
    p->stats.kernel_launches = 5;
    return p->last = finish_status(p, st);
}

extern "C" bwt_status bwt_mtf_encode(bwt_plan* p, const uint8_t* d_in, const uint64_t* offsets, uint32_t num_blocks,
                                     uint8_t* d_out, void* stream) {
    if (!p || !d_in || !offsets || !d_out) return BWT_EINVAL;
    bwt::NvtxRange nvtx_range("mtf_encode");
    if (cudaSetDevice(p->device) != cudaSuccess) return BWT_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::memset(&p->stats, 0, sizeof(p->stats));
    bwt_status s = prepare_batch(p, offsets, num_blocks, st);
    if (s != BWT_OK) return p->last = s;
    if (p->tile > (int)RTILE) return p->last = BWT_EINVAL;
    const uint32_t nb = p->nb, nt = p->ntiles0;
    // scratch (first use): per chunk its list of last occurrences, its count and its starting list;
    // per block its first chunk
    if (!p->mtf_lists) CKS(cudaMalloc(&p->mtf_lists, (size_t)p->cap_tiles0 * (512 + 4) + 4 * ((size_t)p->cap_b + 1)));
    uint8_t* mru = p->mtf_lists;
    uint8_t* tlist = mru + (size_t)p->cap_tiles0 * 256;
    uint32_t* mcnt = reinterpret_cast<uint32_t*>(tlist + (size_t)p->cap_tiles0 * 256);
    uint32_t* tfirst = mcnt + p->cap_tiles0;
    uint32_t* h_first = p->h_inv_items;  // pinned staging, free outside the inverse
    for (uint32_t t = 0, b = 0; t < nt; ++t)
        if (t == 0 || p->h_tiles[t].blk != p->h_tiles[t - 1].blk) h_first[b++] = t;
    h_first[nb] = nt;
    CKS(cudaMemcpyAsync(tfirst, h_first, sizeof(uint32_t) * (nb + 1), cudaMemcpyHostToDevice, st));
    const int sms = num_sms();
    k_mtf_mru<<<std::max(1, std::min<int>(nt, sms * 8)), RT, 0, st>>>(d_in, p->tiles0, nt, mru, mcnt);
    k_mtf_chain<<<std::max(1u, std::min<uint32_t>((nb + 7) / 8, (uint32_t)sms * 8)), 256, 0, st>>>(tfirst, nb, mru,
                                                                                                 mcnt, tlist);
    k_mtf_encode<<<std::max(1, std::min<int>((nt + MTF_WARPS - 1) / MTF_WARPS, sms * 6)), MTF_WARPS * 32, 0, st>>>(
        d_in, p->tiles0, nt, tlist, d_out);
    CKS(cudaGetLastError());
    p->stats.kernel_launches = 3;
    CKS(cudaStreamSynchronize(st));
    return p->last = BWT_OK;
}
