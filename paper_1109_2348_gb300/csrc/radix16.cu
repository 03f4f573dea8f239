// 16-bit digit LSD passes of the first sort (radix_bits = 16): four passes
// over the u64 rotation prefixes instead of eight 8-bit ones.
//
// A 16-bit digit has 65,536 values, too many for the onesweep pass's
// per-warp counters and per-tile look-back words (65,536 status words a
// 4,096-key tile). So a pass is a reduce-then-scan over *parts* of up to
// PART16_KEYS keys (parts never straddle blocks):
//   1. k_hist16:        per part, the count of every digit (shared-memory
//                       counters, 16 bits each: a part's counts fit);
//   2. k_scan16_cols:   per block and digit, the exclusive prefix of the
//                       counts over the block's parts (in place) and the
//                       block's total;
//   3. k_scan16_digits: per block, the exclusive prefix of the totals over
//                       the digits: where each digit's keys start;
//   4. k_scatter16:     one CTA per part walks it in 4,096-key sub-tiles, in
//                       order. A sub-tile is sorted stably by digit in
//                       shared memory -- (digit, position) pairs ranked by
//                       the low digit byte, then by the high one, each rank
//                       from warp peer masks and per-warp counters as in the
//                       onesweep pass -- so equal digits form runs in
//                       position order. A run of digit D goes to block start
//                       + start of D + keys of D in earlier parts and
//                       sub-tiles, consecutively; the part's prefix row then
//                       advances by the run's length.
// There are no inter-CTA waits. Stability: sub-tiles are visited in order,
// and inside one the ranking keeps position order among equal digits.
// Algorithmic bytes per key and pass: 8 read (histogram) + 12 read + 12
// written (scatter), plus the count rows (about 4 bytes per key written and
// read twice).
#include <algorithm>

#include "kernels.h"

namespace bwt {

namespace {

constexpr int R16 = 65536;
constexpr int H16_THREADS = 1024;
constexpr size_t H16_SMEM = (size_t)R16 / 2 * 4;  // 32,768 words: two 16-bit counters each
constexpr int S16_THREADS = 512;
constexpr int S16_WARPS = S16_THREADS / 32;
constexpr int S16_ITEMS = 8;
constexpr int S16_TILE = S16_THREADS * S16_ITEMS;  // 4,096 keys per sub-tile
constexpr int S16_WKEYS = 32 * S16_ITEMS;          // keys per warp (warp-striped)
static_assert(S16_TILE == 4096, "positions inside a sub-tile take 12 bits");
static_assert(PART16_KEYS < 65536 && PART16_KEYS % S16_TILE == 0, "16-bit part counters");

// Scatter kernel's shared memory.
struct S16Layout {
    static constexpr size_t KEYS = 0;                                  // u64[4096]
    static constexpr size_t VALS = KEYS + (size_t)S16_TILE * 8;        // u32[4096]
    static constexpr size_t TA = VALS + (size_t)S16_TILE * 4;          // u32[4096]: after pass A; then run bases
    static constexpr size_t TB = TA + (size_t)S16_TILE * 4;            // u32[4096]: sorted (digit << 12 | position)
    static constexpr size_t WHIST = TB + (size_t)S16_TILE * 4;         // u16[warps][256]
    static constexpr size_t DSTART = WHIST + (size_t)S16_WARPS * 256 * 2;  // u32[256]
    static constexpr size_t RS = DSTART + 256 * 4;                     // u16[4096]: run start of every sorted row
    static constexpr size_t BYTES = RS + (size_t)S16_TILE * 2;         // staged block bytes (first pass)
    static constexpr size_t TOTAL = BYTES + S16_TILE + 48;
};

// Digit of rotation i of a block of n bytes for the first pass (shift 0): the
// key's last two bytes, S[(i + 6) mod n] and S[(i + 7) mod n].
__device__ __forceinline__ uint32_t digit_from_s(const uint8_t* __restrict__ S, BlockInfo bi, uint32_t i) {
    uint32_t a = i + 6, b = i + 7;
    if (b >= bi.n) {
        a %= bi.n;
        b %= bi.n;
    }
    return ((uint32_t)S[bi.off + a] << 8) | S[bi.off + b];
}

template <bool FROM_S>
__global__ void __launch_bounds__(H16_THREADS) k_hist16(const uint64_t* __restrict__ kin, const uint8_t* __restrict__ S,
                                                      const BlockInfo* __restrict__ blocks,
                                                      const TileDesc* __restrict__ parts, uint32_t nparts, int shift,
                                                      uint32_t* __restrict__ partcnt) {
    extern __shared__ __align__(16) uint32_t h16[];  // [R16 / 2]: digit d in half d & 1 of word d >> 1
    for (uint32_t part = blockIdx.x; part < nparts; part += gridDim.x) {
        for (int w = threadIdx.x; w < R16 / 2; w += H16_THREADS) h16[w] = 0u;
        __syncthreads();
        const TileDesc td = parts[part];
        const BlockInfo bi = blocks[td.blk];
        const uint32_t i0 = td.start - bi.off;
        const uint32_t rounds = (td.len + H16_THREADS - 1) / H16_THREADS;
        for (uint32_t r = 0; r < rounds; ++r) {
            const uint32_t q = r * H16_THREADS + threadIdx.x;
            const bool valid = q < td.len;
            uint32_t d = 0;
            if (valid) {
                if constexpr (FROM_S) d = digit_from_s(S, bi, i0 + q);
                else d = (uint32_t)(kin[td.start + q] >> shift) & 0xffffu;
            }
            // one shared-memory atomic per distinct digit of the warp (runs of
            // equal digits, e.g. constant blocks, do not serialise on one word)
            const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 0x10000u);
            if (valid && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
                atomicAdd(&h16[d >> 1], (uint32_t)__popc(peers) << ((d & 1u) * 16u));
        }
        __syncthreads();
        uint2* row = reinterpret_cast<uint2*>(partcnt + (size_t)part * R16);
        for (int w = threadIdx.x; w < R16 / 2; w += H16_THREADS) {
            const uint32_t v = h16[w];
            row[w] = make_uint2(v & 0xffffu, v >> 16);
        }
        __syncthreads();
    }
}

// One thread per (block, digit): exclusive prefix over the block's parts, in
// place, and the block's total of the digit.
__global__ void __launch_bounds__(256) k_scan16_cols(uint32_t* __restrict__ partcnt,
                                                     const uint32_t* __restrict__ part_first, uint32_t nseg,
                                                     uint32_t* __restrict__ segtot) {
    const uint64_t total = (uint64_t)nseg * R16;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t seg = (uint32_t)(x >> 16), d = (uint32_t)(x & 0xffffu);
        const uint32_t p0 = part_first[seg], p1 = part_first[seg + 1];
        uint32_t s = 0;
        for (uint32_t p = p0; p < p1; ++p) {
            uint32_t* c = partcnt + (size_t)p * R16 + d;
            const uint32_t v = *c;
            *c = s;
            s += v;
        }
        segtot[(size_t)seg * R16 + d] = s;
    }
}

// One CTA per block: exclusive prefix of its 65,536 digit totals, in place.
__global__ void __launch_bounds__(1024) k_scan16_digits(uint32_t* __restrict__ segtot, uint32_t nseg) {
    __shared__ uint32_t tmp[32];
    constexpr int PER = R16 / 1024;
    for (uint32_t seg = blockIdx.x; seg < nseg; seg += gridDim.x) {
        uint4* row = reinterpret_cast<uint4*>(segtot + (size_t)seg * R16 + threadIdx.x * PER);
        uint32_t s = 0;
#pragma unroll 1
        for (int i = 0; i < PER / 4; ++i) {  // a thread's 64 consecutive totals, read twice (L2)
            const uint4 v = row[i];
            s += v.x + v.y + v.z + v.w;
        }
        uint32_t total;
        uint32_t ex = block_exclusive_scan<1024>(s, tmp, &total);
#pragma unroll 1
        for (int i = 0; i < PER / 4; ++i) {
            const uint4 v = row[i];
            uint4 o;
            o.x = ex;
            o.y = o.x + v.x;
            o.z = o.y + v.y;
            o.w = o.z + v.z;
            ex = o.w + v.w;
            row[i] = o;
        }
        __syncthreads();
    }
}

// Stable rank of this warp-striped slice of the sub-tile by an 8-bit digit
// (256 = invalid): per-warp counters (the onesweep pass's ranking), an
// exclusive prefix over warps per digit, then over digits. Returns in every
// item its position in the stable order (0xffffffff for invalid items).
__device__ __forceinline__ void rank8_striped(const uint32_t (&dig)[S16_ITEMS], uint32_t (&pos)[S16_ITEMS],
                                              uint16_t* whist, uint32_t* dstart, uint32_t* scan_tmp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    {
        uint32_t* w32 = reinterpret_cast<uint32_t*>(whist);
        for (int i = tid; i < S16_WARPS * 256 / 2; i += S16_THREADS) w32[i] = 0u;
    }
    __syncthreads();
    uint16_t* mine = whist + warp * 256;
#pragma unroll
    for (int j = 0; j < S16_ITEMS; ++j) {
        const uint32_t d = dig[j];
        const uint32_t peers = match_label<9>(d);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (d < 256u && lane == leader) {
            base = mine[d];
            mine[d] = (uint16_t)(base + __popc(peers));
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        __syncwarp();
        pos[j] = base + __popc(peers & lt);
    }
    __syncthreads();
    uint32_t cnt = 0;
    if (tid < 256) {
        for (int w = 0; w < S16_WARPS; ++w) {
            const uint32_t c = whist[w * 256 + tid];
            whist[w * 256 + tid] = (uint16_t)cnt;
            cnt += c;
        }
    }
    uint32_t total;
    const uint32_t ex = block_exclusive_scan<S16_THREADS>(cnt, scan_tmp, &total);
    if (tid < 256) dstart[tid] = ex;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < S16_ITEMS; ++j) {
        const uint32_t d = dig[j];
        pos[j] = d < 256u ? dstart[d] + whist[warp * 256 + d] + pos[j] : 0xffffffffu;
    }
    __syncthreads();  // whist and dstart are reused by the next call
}

template <bool FROM_S>
__global__ void __launch_bounds__(S16_THREADS, 2) k_scatter16(const uint64_t* __restrict__ kin,
                                                            const uint32_t* __restrict__ vin,
                                                            uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                            const uint8_t* __restrict__ S,
                                                            const BlockInfo* __restrict__ blocks,
                                                            const TileDesc* __restrict__ parts, uint32_t nparts,
                                                            int shift, uint32_t* __restrict__ partoff,
                                                            const uint32_t* __restrict__ segbase, uint32_t* ctrl) {
    using Lay = S16Layout;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* skeys = reinterpret_cast<uint64_t*>(smem + Lay::KEYS);
    uint32_t* svals = reinterpret_cast<uint32_t*>(smem + Lay::VALS);
    uint32_t* tA = reinterpret_cast<uint32_t*>(smem + Lay::TA);
    uint32_t* tB = reinterpret_cast<uint32_t*>(smem + Lay::TB);
    uint16_t* whist = reinterpret_cast<uint16_t*>(smem + Lay::WHIST);
    uint32_t* dstart = reinterpret_cast<uint32_t*>(smem + Lay::DSTART);
    uint16_t* rs = reinterpret_cast<uint16_t*>(smem + Lay::RS);
    uint8_t* sbytes = smem + Lay::BYTES;
    __shared__ uint32_t scan_tmp[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (uint32_t part = blockIdx.x; part < nparts; part += gridDim.x) {
        const TileDesc td = parts[part];
        const BlockInfo bi = blocks[td.blk];
        const uint32_t i0 = td.start - bi.off;
        uint32_t* prow = partoff + (size_t)part * R16;
        const uint32_t* srow = segbase + (size_t)td.seg * R16;
        for (uint32_t s0 = 0; s0 < td.len; s0 += S16_TILE) {
            const uint32_t len = min((uint32_t)S16_TILE, td.len - s0);
            // ---- stage the sub-tile's keys and values by position
            if constexpr (FROM_S) {
                const uint32_t sh = stage_tile_bytes(S, bi, i0 + s0, len, sbytes, tid, S16_THREADS);
                __syncthreads();
                for (uint32_t q = tid; q < len; q += S16_THREADS) {
                    skeys[q] = pack8_smem(sbytes, sh + q);
                    svals[q] = i0 + s0 + q;
                }
            } else {
                for (uint32_t q = tid; q < len; q += S16_THREADS) {
                    skeys[q] = kin[td.start + s0 + q];
                    svals[q] = vin[td.start + s0 + q];
                }
            }
            __syncthreads();
            // ---- pass A: by the digit's low byte; tA holds (digit << 12 | position)
            uint32_t dig[S16_ITEMS], pos[S16_ITEMS], ent[S16_ITEMS];
#pragma unroll
            for (int j = 0; j < S16_ITEMS; ++j) {
                const uint32_t idx = warp * S16_WKEYS + j * 32 + lane;
                const uint32_t D = idx < len ? (uint32_t)(skeys[idx] >> shift) & 0xffffu : 0u;
                ent[j] = (D << 12) | idx;
                dig[j] = idx < len ? (D & 0xffu) : 256u;
            }
            rank8_striped(dig, pos, whist, dstart, scan_tmp);
#pragma unroll
            for (int j = 0; j < S16_ITEMS; ++j)
                if (pos[j] != 0xffffffffu) tA[pos[j]] = ent[j];
            __syncthreads();
            // ---- pass B: by the high byte; tB is sorted by digit, positions ascending
#pragma unroll
            for (int j = 0; j < S16_ITEMS; ++j) {
                const uint32_t idx = warp * S16_WKEYS + j * 32 + lane;
                ent[j] = idx < len ? tA[idx] : 0u;
                dig[j] = idx < len ? (ent[j] >> 20) & 0xffu : 256u;
            }
            rank8_striped(dig, pos, whist, dstart, scan_tmp);
#pragma unroll
            for (int j = 0; j < S16_ITEMS; ++j)
                if (pos[j] != 0xffffffffu) tB[pos[j]] = ent[j];
            __syncthreads();
            // ---- runs of equal digits: thread t owns sorted rows 8t .. 8t + 7;
            //      a run's start is the last head at or before a row
            const uint32_t r0 = (uint32_t)tid * S16_ITEMS;
            uint32_t last = 0;  // last head among this thread's rows (row 0 is always a head)
            uint32_t e[S16_ITEMS];
#pragma unroll
            for (int j = 0; j < S16_ITEMS; ++j) {
                const uint32_t r = r0 + j;
                e[j] = r < len ? tB[r] : 0u;
                const bool head = r < len && (r == 0 || (tB[r - 1] >> 12) != (e[j] >> 12));
                if (head) {
                    last = r;
                    // block start + digit start + keys of the digit before this
                    // sub-tile; row x of the run goes to tA[start] + x
                    const uint32_t D = e[j] >> 12;
                    tA[r] = bi.off + srow[D] + prow[D] - r;
                }
            }
            // exclusive max-scan of the threads' last heads: the run that a
            // thread's first rows continue
            uint32_t incl = last;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl = max(incl, y);
            }
            if (lane == 31) scan_tmp[warp] = incl;
            __syncthreads();  // also: every head has read its digit's count
            uint32_t start = 0;
            for (int w = 0; w < warp; ++w) start = max(start, scan_tmp[w]);
            {
                const uint32_t prev = __shfl_up_sync(0xffffffffu, incl, 1);
                if (lane > 0) start = max(start, prev);
            }
#pragma unroll
            for (int j = 0; j < S16_ITEMS; ++j) {
                const uint32_t r = r0 + j;
                if (r >= len) break;
                const uint32_t D = e[j] >> 12;
                if (r == 0 || (tB[r - 1] >> 12) != D) start = r;
                rs[r] = (uint16_t)start;
                if (r + 1 == len || (tB[r + 1] >> 12) != D) prow[D] += r - start + 1;  // the run's last row
            }
            __syncthreads();
            // ---- scatter in row order: consecutive lanes write consecutive
            //      destinations inside a run
            for (uint32_t r = tid; r < len; r += S16_THREADS) {
                const uint32_t q = tB[r] & 0xfffu;
                const uint32_t dst = tA[rs[r]] + r;
                if (dst - bi.off < bi.n) {
                    kout[dst] = skeys[q];
                    vout[dst] = svals[q];
                } else {
                    atomicOr(&ctrl[CTRL_ERR], ERR_CAPACITY);  // counts and keys disagree: never write outside the block
                }
            }
            __syncthreads();  // the next sub-tile reuses every array and reads the advanced counts
        }
    }
}

}  // namespace

size_t scatter16_smem() { return S16Layout::TOTAL; }

cudaError_t launch_first16_pass(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                                const uint8_t* S, const BlockInfo* blocks, const TileDesc* parts, uint32_t nparts,
                                const uint32_t* part_first, uint32_t nseg, int shift, uint32_t* partcnt,
                                uint32_t* segtot, uint32_t* ctrl, cudaStream_t st) {
    if (nparts == 0) return cudaSuccess;
    static const bool attr = [] {
        cudaFuncSetAttribute((void*)k_hist16<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)H16_SMEM);
        cudaFuncSetAttribute((void*)k_hist16<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)H16_SMEM);
        cudaFuncSetAttribute((void*)k_scatter16<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)S16Layout::TOTAL);
        cudaFuncSetAttribute((void*)k_scatter16<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)S16Layout::TOTAL);
        return true;
    }();
    (void)attr;
    const int sms = num_sms();
    const bool from_s = kin == nullptr;
    const int hgrid = (int)std::min<uint32_t>(nparts, (uint32_t)sms);
    if (from_s) k_hist16<true><<<hgrid, H16_THREADS, H16_SMEM, st>>>(kin, S, blocks, parts, nparts, shift, partcnt);
    else k_hist16<false><<<hgrid, H16_THREADS, H16_SMEM, st>>>(kin, S, blocks, parts, nparts, shift, partcnt);
    const uint64_t cols = (uint64_t)nseg * R16;
    k_scan16_cols<<<(unsigned)std::min<uint64_t>((cols + 255) / 256, (uint64_t)sms * 64), 256, 0, st>>>(
        partcnt, part_first, nseg, segtot);
    k_scan16_digits<<<(unsigned)std::min<uint32_t>(nseg, (uint32_t)sms * 2), 1024, 0, st>>>(segtot, nseg);
    const int sgrid = (int)std::min<uint32_t>(nparts, (uint32_t)sms * 2);
    if (from_s)
        k_scatter16<true><<<sgrid, S16_THREADS, S16Layout::TOTAL, st>>>(kin, vin, kout, vout, S, blocks, parts, nparts,
                                                                         shift, partcnt, segtot, ctrl);
    else
        k_scatter16<false><<<sgrid, S16_THREADS, S16Layout::TOTAL, st>>>(kin, vin, kout, vout, S, blocks, parts,
                                                                          nparts, shift, partcnt, segtot, ctrl);
    return cudaGetLastError();
}

}  // namespace bwt
