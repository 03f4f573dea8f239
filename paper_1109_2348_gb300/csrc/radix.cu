// Segmented, stable onesweep LSD radix pass and the histograms it needs.
//
// The first sort of the BWT (the rotation sort of Section 3.1) orders every
// rotation by its 8-byte prefix, packed big-endian into a u64,
// and carries the rotation index as the value. A segment is a block (first
// sort) or a group of still-equal rotations (prefix-doubling rounds); tiles
// never straddle segments, so one launch sorts every segment of a batch.
//
// One pass = one launch. A CTA takes the next tile index from an atomic
// counter, ranks its keys by digit with warp-level peer masks (stable:
// warp-striped order, warps in order), publishes its per-digit counts,
// stages the tile in shared memory in digit order, then looks back over the
// preceding tiles of its segment for the exclusive prefix (decoupled
// look-back; each wait is bounded and sets ERR_TIMEOUT when it runs out) and
// scatters the tile with runs of consecutive destinations. Staging before
// the look-back overlaps the value loads with the wait for earlier tiles
// (measured: 5% faster per u64 pass than looking back first). Keys are
// read once and written once per pass: 2 x (8 + 4) bytes per u64 key.
#include <algorithm>
#include <cstdio>

#include "kernels.h"

namespace bwt {

namespace {

// Threads per radix CTA: 256 for every tile size (measured: a 4096-key tile
// with 512 threads at <= 64 registers ran slower than 256 threads at 128).
template <int TILE>
struct OsThreads {
    static constexpr int value = 256;
};

// Resident CTAs per SM the register budget is sized for: a pass is bound by
// the latency of each tile's chain of phases, so more CTAs in flight beat
// more registers (measured on 64 x 900,000 keys: 3 CTAs of <= 80 registers
// ran a u64 pass 16% faster than 2 of 128).
template <int TILE>
struct OsMinBlocks {
    static constexpr int value = TILE >= 4096 ? 3 : TILE >= 2048 ? 5 : 6;
};

template <typename KeyT, int RBITS, int TILE, bool FROM_S>
struct OneSweepLayout {
    static constexpr int RADIX = 1 << RBITS;
    static constexpr int WARPS = OsThreads<TILE>::value / 32;
    static constexpr size_t WHIST = (size_t)WARPS * RADIX * 2;
    static constexpr size_t STAGE = (size_t)TILE * (sizeof(KeyT) + 4);
    static constexpr size_t BYTES = FROM_S ? (size_t)TILE + 48 : 0;  // tile + 7 halo bytes + alignment slack
    static constexpr size_t U0 = WHIST > STAGE ? WHIST : STAGE;
    static constexpr size_t U = ((U0 > BYTES ? U0 : BYTES) + 15) & ~(size_t)15;
    static constexpr size_t TOTAL = U + 2 * RADIX * 4 + 32 * 4 + 16;
};

// VDIG: the digit comes from the value (the rotation index) instead of the
// key; used to put overflow buckets of the learned bucketing in index order
// before their key passes.
template <typename KeyT, int RBITS, int TILE, bool FROM_S, bool VDIG = false>
__global__ void __launch_bounds__(OsThreads<TILE>::value, OsMinBlocks<TILE>::value) k_onesweep(OneSweepParams p) {
    using Lay = OneSweepLayout<KeyT, RBITS, TILE, FROM_S>;
    constexpr int OS_THREADS = OsThreads<TILE>::value;
    constexpr int OS_WARPS = OS_THREADS / 32;
    constexpr int RADIX = 1 << RBITS;
    constexpr int ITEMS = TILE / OS_THREADS;
    constexpr int WKEYS = 32 * ITEMS;
    // digits owned per thread; with fewer digits than threads, threads
    // tid < RADIX own one digit each and the others own none
    constexpr int DPT = RADIX >= OS_THREADS ? RADIX / OS_THREADS : 1;
    constexpr int OWNERS = RADIX / DPT;

    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t* whist = reinterpret_cast<uint16_t*>(smem);
    KeyT* skeys = reinterpret_cast<KeyT*>(smem);
    uint32_t* svals = reinterpret_cast<uint32_t*>(smem + (size_t)TILE * sizeof(KeyT));
    uint8_t* sbytes = smem;
    uint32_t* digit_start = reinterpret_cast<uint32_t*>(smem + Lay::U);
    uint32_t* gbase = digit_start + RADIX;
    uint32_t* scan_tmp = gbase + RADIX;
    uint32_t* s_tile = scan_tmp + 32;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t num_tiles = *p.num_tiles;
    const uint32_t spin_limit = p.ctrl[CTRL_SPIN];
    const uint32_t withhold = p.ctrl[CTRL_WITHHOLD];
    const KeyT* kin = static_cast<const KeyT*>(p.kin);
    KeyT* kout = static_cast<KeyT*>(p.kout);
    const uint32_t lt = lanemask_lt();

    for (;;) {
        if (tid == 0) *s_tile = atomicAdd(p.tile_counter, 1u);
        __syncthreads();
        const uint32_t t = *s_tile;
        if (t >= num_tiles) break;
        const TileDesc td = p.tiles[t];
        if constexpr (sizeof(KeyT) == 4) {
            // a doubling round's group whose keys are all equal does not move:
            // its tiles are skipped whole (no tile of another group looks
            // back at them)
            if (p.seg_varied && p.seg_varied[td.seg] == 0u) {
                __syncthreads();  // every thread has read s_tile
                continue;
            }
        }

        // ---- load the tile (warp-striped: item j of lane l of warp w is
        //      tile index w*WKEYS + j*32 + l)
        //      With u64 keys the values are read only when the tile is staged
        //      (fewer live registers through ranking and look-back), unless
        //      they carry the digit (VDIG); u32-key tiles load them up front.
        constexpr bool EARLY_VALS = VDIG || sizeof(KeyT) == 4;
        KeyT key[ITEMS];
        uint32_t val[EARLY_VALS ? ITEMS : 1];
        uint32_t i0 = 0;  // FROM_S: block-relative index of the tile's first rotation (its value)
        if constexpr (FROM_S) {
            const BlockInfo bi = p.blocks[td.blk];
            i0 = td.start - bi.off;
            const uint32_t shift = stage_tile_bytes(p.S, bi, i0, td.len, sbytes, tid, OS_THREADS);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const uint32_t idx = warp * WKEYS + j * 32 + lane;
                key[j] = idx < td.len ? (KeyT)pack8_smem(sbytes, shift + idx) : (KeyT)0;
            }
            __syncthreads();
        } else {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const uint32_t idx = warp * WKEYS + j * 32 + lane;
                key[j] = idx < td.len ? kin[td.start + idx] : (KeyT)0;
                if constexpr (EARLY_VALS) val[j] = idx < td.len ? p.vin[td.start + idx] : 0u;
            }
        }

        // ---- per-warp digit counts and stable ranks
        {
            uint32_t* w32 = reinterpret_cast<uint32_t*>(whist);
            for (int i = tid; i < OS_WARPS * RADIX / 2; i += OS_THREADS) w32[i] = 0u;
        }
        __syncthreads();
        uint32_t rkdg[ITEMS];  // rank within warp (low 16) | digit (high 16)
        uint16_t* my_hist = whist + warp * RADIX;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t idx = warp * WKEYS + j * 32 + lane;
            const bool valid = idx < td.len;
            uint32_t d = (uint32_t)RADIX;
            if (valid) {
                if constexpr (VDIG) d = (val[j] >> p.shift) & (uint32_t)(RADIX - 1);
                else d = (uint32_t)((key[j] >> p.shift) & (KeyT)(RADIX - 1));
            }
            // peer masks: one ballot per digit bit for u64 passes (the first
            // sort: many distinct digits per warp), match.any for u32 passes
            // (doubling rounds: repetitive rank digits, where it measured faster)
            uint32_t peers;
            if constexpr (sizeof(KeyT) == 8) peers = match_label<RBITS + 1>(d);
            else peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (valid && lane == leader) {
                base = my_hist[d];
                my_hist[d] = (uint16_t)(base + __popc(peers));
            }
            base = __shfl_sync(0xffffffffu, base, leader);
            __syncwarp();
            rkdg[j] = (base + __popc(peers & lt)) | (d << 16);
        }
        __syncthreads();

        // ---- tile counts per digit, exclusive prefix over warps (in place)
        const bool owner = tid < OWNERS;
        uint32_t cnt[DPT];
        uint32_t tsum = 0;
#pragma unroll
        for (int i = 0; i < DPT; ++i) {
            cnt[i] = 0;
            if (owner) {
                const int d = tid * DPT + i;
                uint32_t s = 0;
#pragma unroll
                for (int w = 0; w < OS_WARPS; ++w) {
                    const uint32_t c = whist[w * RADIX + d];
                    whist[w * RADIX + d] = (uint16_t)s;
                    s += c;
                }
                cnt[i] = s;
                tsum += s;
            }
        }
        uint32_t total;
        uint32_t ex = block_exclusive_scan<OS_THREADS>(tsum, scan_tmp, &total);
        if (owner) {
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                digit_start[tid * DPT + i] = ex;
                ex += cnt[i];
            }
        }

        // ---- publish this tile's counts (inclusive when it opens its segment)
        const bool first = (t == td.firstTile);
        if (owner) {
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                uint32_t* mine = p.status + (size_t)t * RADIX + tid * DPT + i;
                if (first) {
                    if (!(withhold && t == 0)) st_volatile(mine, ST_INC | cnt[i]);
                } else {
                    st_volatile(mine, ST_AGG | cnt[i]);
                }
            }
        }
        __syncthreads();

        // ---- stage in digit order (needs no global prefix)
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t d = rkdg[j] >> 16;
            if (d < (uint32_t)RADIX) rkdg[j] = digit_start[d] + whist[warp * RADIX + d] + (rkdg[j] & 0xffffu);
            else rkdg[j] = 0xffffffffu;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (rkdg[j] != 0xffffffffu) {
                const uint32_t idx = warp * WKEYS + j * 32 + lane;
                uint32_t v;
                if constexpr (FROM_S) v = i0 + idx;
                else if constexpr (EARLY_VALS) v = val[j];
                else v = p.vin[td.start + idx];
                skeys[rkdg[j]] = key[j];
                svals[rkdg[j]] = v;
            }
        }

        // ---- decoupled look-back over this segment's earlier tiles
        if constexpr (DPT == 1) {
            if (owner) {
                const int d = tid;
                uint32_t excl = 0;
                if (!first) {
                    // Walk back LB predecessors a step: their words are loaded
                    // together, then added in order until an inclusive one. When
                    // the tiles of a segment run at once (a small batch), their
                    // words are mostly aggregates, and the walk is a chain of
                    // L2 round trips that this shortens LB-fold.
                    constexpr uint32_t LB = 4;
                    uint32_t q = t - 1;  // the next predecessor to add (>= firstTile)
                    for (;;) {
                        const uint32_t m = min(LB, q - td.firstTile + 1);
                        uint32_t v[LB];
#pragma unroll
                        for (uint32_t k = 0; k < LB; ++k)
                            v[k] = k < m ? ld_volatile(p.status + (size_t)(q - k) * RADIX + d) : 0u;
                        bool done = false;
#pragma unroll
                        for (uint32_t k = 0; k < LB; ++k) {
                            if (k >= m || done) break;
                            uint32_t it = 0;
                            while ((v[k] & (ST_AGG | ST_INC)) == 0u) {
                                if (++it > spin_limit) {
                                    atomicOr(&p.ctrl[CTRL_ERR], ERR_TIMEOUT);
                                    v[k] = ST_INC;  // give up: proceed with a short prefix (stays in bounds)
                                    break;
                                }
                                if (it > 32) __nanosleep(64);
                                v[k] = ld_volatile(p.status + (size_t)(q - k) * RADIX + d);
                            }
                            excl += v[k] & ST_VALUE;
                            if (v[k] & ST_INC) done = true;
                        }
                        // the segment's first tile is always inclusive: reaching it ends the walk
                        if (done || q + 1 - m == td.firstTile) break;
                        q -= m;
                    }
                    st_volatile(p.status + (size_t)t * RADIX + d, ST_INC | ((excl + cnt[0]) & ST_VALUE));
                }
                gbase[d] = td.segStart + p.seg_base[(size_t)td.seg * p.seg_base_stride + d] + excl - digit_start[d];
            }
        } else {
            // several digits a thread: walk back for all of them at once, one
            // round of independent loads per step, so a thread waits for one
            // chain of L2 round trips rather than DPT chains in a row. The
            // rounds without progress are bounded by spin_limit in total.
            static_assert(DPT <= 32, "pending mask");
            uint32_t excl[DPT], q[DPT];
            uint32_t pending = (owner && !first) ? (uint32_t)((1ull << DPT) - 1) : 0u;
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                excl[i] = 0;
                q[i] = t - 1;
            }
            uint32_t it = 0;
            while (pending) {
                uint32_t v[DPT];
#pragma unroll
                for (int i = 0; i < DPT; ++i)
                    v[i] = (pending >> i) & 1u ? ld_volatile(p.status + (size_t)q[i] * RADIX + tid * DPT + i) : 0u;
                bool progress = false;
#pragma unroll
                for (int i = 0; i < DPT; ++i) {
                    if (((pending >> i) & 1u) && (v[i] & (ST_AGG | ST_INC))) {
                        progress = true;
                        excl[i] += v[i] & ST_VALUE;
                        if ((v[i] & ST_INC) || q[i] == td.firstTile) pending &= ~(1u << i);
                        else --q[i];
                    }
                }
                if (!progress) {
                    if (++it > spin_limit) {
                        atomicOr(&p.ctrl[CTRL_ERR], ERR_TIMEOUT);  // give up: short prefixes (stay in bounds)
                        break;
                    }
                    if (it > 32) __nanosleep(64);
                }
            }
            if (owner) {
#pragma unroll
                for (int i = 0; i < DPT; ++i) {
                    const int d = tid * DPT + i;
                    if (!first) st_volatile(p.status + (size_t)t * RADIX + d, ST_INC | ((excl[i] + cnt[i]) & ST_VALUE));
                    gbase[d] = td.segStart + p.seg_base[(size_t)td.seg * p.seg_base_stride + d] + excl[i] -
                               digit_start[d];
                }
            }
        }
        __syncthreads();
        for (uint32_t q = tid; q < td.len; q += OS_THREADS) {
            const KeyT k = skeys[q];
            const uint32_t v = svals[q];
            uint32_t d;
            if constexpr (VDIG) d = (v >> p.shift) & (uint32_t)(RADIX - 1);
            else d = (uint32_t)((k >> p.shift) & (KeyT)(RADIX - 1));
            const uint32_t dst = gbase[d] + q;
            BWT_DCHECK(dst - td.segStart < td.pad0, &p.ctrl[CTRL_ERR]);  // inside the tile's segment
            kout[dst] = k;
            p.vout[dst] = v;
        }
        __syncthreads();
    }
}

// ---- histograms ------------------------------------------------------------

// d = 8: byte histogram of every block. Each thread counts a run of 16
// consecutive bytes and adds whole runs of equal bytes, so run-heavy blocks
// do not serialise on one shared-memory counter.
__global__ void __launch_bounds__(256) k_hist_bytes(const uint8_t* __restrict__ S, const BlockInfo* __restrict__ blocks,
                                                    const TileDesc* __restrict__ tiles, uint32_t num_tiles,
                                                    const uint32_t* __restrict__ num_tiles_dev,
                                                    uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    if (num_tiles_dev) num_tiles = *num_tiles_dev;
    for (uint32_t t = blockIdx.x; t < num_tiles; t += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
        const TileDesc td = tiles[t];
        for (uint32_t c0 = threadIdx.x * 16; c0 < td.len; c0 += 256 * 16) {
            const uint32_t c1 = min(c0 + 16, td.len);
            uint32_t prev = S[td.start + c0], run = 1;
            for (uint32_t q = c0 + 1; q < c1; ++q) {
                const uint32_t b = S[td.start + q];
                if (b == prev) {
                    ++run;
                } else {
                    atomicAdd(&h[prev], run);
                    prev = b;
                    run = 1;
                }
            }
            atomicAdd(&h[prev], run);
        }
        __syncthreads();
        const uint32_t c = h[threadIdx.x];
        if (c) atomicAdd(&hist[(size_t)td.blk * 256 + threadIdx.x], c);
        __syncthreads();
    }
}

// d = 11: six digit histograms of the u64 prefixes (shifts 0, 11, .., 55).
template <int TILE>
__global__ void __launch_bounds__(256) k_hist_keys11(const uint8_t* __restrict__ S, const BlockInfo* __restrict__ blocks,
                                                     const TileDesc* __restrict__ tiles, uint32_t num_tiles,
                                                     const uint32_t* __restrict__ num_tiles_dev,
                                                     uint32_t* __restrict__ hist) {
    constexpr int RADIX = 2048, PASSES = 6;
    if (num_tiles_dev) num_tiles = *num_tiles_dev;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* h = reinterpret_cast<uint32_t*>(smem);
    uint8_t* sbytes = smem + PASSES * RADIX * 4;
    const int lane = threadIdx.x & 31;
    for (uint32_t t = blockIdx.x; t < num_tiles; t += gridDim.x) {
        for (int i = threadIdx.x; i < PASSES * RADIX; i += 256) h[i] = 0;
        const TileDesc td = tiles[t];
        const BlockInfo bi = blocks[td.blk];
        const uint32_t i0 = td.start - bi.off;
        const uint32_t shift = stage_tile_bytes(S, bi, i0, td.len, sbytes, threadIdx.x, 256);
        __syncthreads();
        for (uint32_t q0 = 0; q0 < td.len; q0 += 256) {
            const uint32_t q = q0 + threadIdx.x;
            const bool valid = q < td.len;
            const uint64_t k = valid ? pack8_smem(sbytes, shift + q) : 0ull;
#pragma unroll
            for (int ps = 0; ps < PASSES; ++ps) {
                const uint32_t d = valid ? (uint32_t)((k >> (11 * ps)) & (RADIX - 1)) : (uint32_t)RADIX;
                const uint32_t peers = match_label<12>(d);
                if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[ps * RADIX + d], (uint32_t)__popc(peers));
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < PASSES * RADIX; i += 256) {
            const uint32_t c = h[i];
            if (c) atomicAdd(&hist[(size_t)td.blk * PASSES * RADIX + i], c);
        }
        __syncthreads();
    }
}

// Exclusive scan of rows of `radix` counters (one CTA per row, grid-stride).
__global__ void __launch_bounds__(256) k_scan_rows(uint32_t* __restrict__ hist, int radix,
                                                   const uint32_t* __restrict__ num_rows_dev, uint32_t rows_mult,
                                                   uint32_t rows_host, uint32_t max_rows) {
    __shared__ uint32_t tmp[32];
    uint64_t r64 = num_rows_dev ? (uint64_t)(*num_rows_dev) * rows_mult : rows_host;
    const uint32_t rows = (uint32_t)(r64 < max_rows ? r64 : max_rows);
    const int per = radix / 256;
    for (uint32_t r = blockIdx.x; r < rows; r += gridDim.x) {
        uint32_t* row = hist + (size_t)r * radix;
        uint32_t v[16];
        uint32_t s = 0;
        for (int i = 0; i < per; ++i) {
            v[i] = row[threadIdx.x * per + i];
            s += v[i];
        }
        uint32_t total;
        uint32_t ex = block_exclusive_scan<256>(s, tmp, &total);
        for (int i = 0; i < per; ++i) {
            row[threadIdx.x * per + i] = ex;
            ex += v[i];
        }
    }
}

__global__ void k_zero_by_count(uint32_t* __restrict__ p, const uint32_t* __restrict__ count, uint32_t per_unit,
                                uint32_t max_words) {
    uint64_t n = (uint64_t)(*count) * per_unit;
    if (n > max_words) n = max_words;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = 0u;
}

template <typename KeyT, int RBITS, int TILE, bool FROM_S, bool VDIG>
struct OneSweepKernel {
    static void* fn() { return (void*)k_onesweep<KeyT, RBITS, TILE, FROM_S, VDIG>; }
    static size_t smem() { return OneSweepLayout<KeyT, RBITS, TILE, FROM_S>::TOTAL; }
};

struct KernelEntry {
    void* fn;
    size_t smem;
    int grid;
    int threads;
};

template <typename KeyT, int RBITS, int TILE, bool FROM_S, bool VDIG = false>
KernelEntry& entry() {
    static KernelEntry e = [] {
        KernelEntry x;
        x.fn = OneSweepKernel<KeyT, RBITS, TILE, FROM_S, VDIG>::fn();
        x.smem = OneSweepKernel<KeyT, RBITS, TILE, FROM_S, VDIG>::smem();
        cudaFuncSetAttribute(x.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)x.smem);
        x.threads = OsThreads<TILE>::value;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, x.fn, x.threads, x.smem);
        x.grid = std::max(1, per_sm) * num_sms();
        return x;
    }();
    return e;
}

template <typename KeyT, bool FROM_S>
KernelEntry* pick(int rbits, int tile) {
    if (rbits == 8) {
        if (tile == 1024) return &entry<KeyT, 8, 1024, FROM_S>();
        if (tile == 2048) return &entry<KeyT, 8, 2048, FROM_S>();
        if (tile == 4096) return &entry<KeyT, 8, 4096, FROM_S>();
    } else if (rbits == 11) {
        if (tile == 1024) return &entry<KeyT, 11, 1024, FROM_S>();
        if (tile == 2048) return &entry<KeyT, 11, 2048, FROM_S>();
        if (tile == 4096) return &entry<KeyT, 11, 4096, FROM_S>();
    }
    return nullptr;
}

// 10-bit digits: u32 rank keys of the doubling rounds only (two passes cover
// ranks below 2^20, i.e. blocks up to 1 MiB).
KernelEntry* pick_u32_10(int tile) {
    if (tile == 1024) return &entry<uint32_t, 10, 1024, false>();
    if (tile == 2048) return &entry<uint32_t, 10, 2048, false>();
    if (tile == 4096) return &entry<uint32_t, 10, 4096, false>();
    return nullptr;
}

KernelEntry* pick_vdig(int tile) {
    if (tile == 1024) return &entry<uint64_t, 8, 1024, false, true>();
    if (tile == 2048) return &entry<uint64_t, 8, 2048, false, true>();
    if (tile == 4096) return &entry<uint64_t, 8, 4096, false, true>();
    return nullptr;
}

KernelEntry* pick_any(int key_bytes, bool from_s, int rbits, int tile) {
    if (key_bytes == 8) return from_s ? pick<uint64_t, true>(rbits, tile) : pick<uint64_t, false>(rbits, tile);
    if (key_bytes == 4 && !from_s) return rbits == 10 ? pick_u32_10(tile) : pick<uint32_t, false>(rbits, tile);
    if (key_bytes == -8 && !from_s && rbits == 8) return pick_vdig(tile);  // u64 keys, digit from the value
    return nullptr;
}

}  // namespace

int num_sms() {
    static int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

int onesweep_grid(int key_bytes, bool from_s, int radix_bits, int tile) {
    KernelEntry* e = pick_any(key_bytes, from_s, radix_bits, tile);
    return e ? e->grid : 0;
}

size_t onesweep_smem(int key_bytes, bool from_s, int radix_bits, int tile) {
    KernelEntry* e = pick_any(key_bytes, from_s, radix_bits, tile);
    return e ? e->smem : 0;
}

cudaError_t launch_onesweep(int key_bytes, bool from_s, int radix_bits, int tile, const OneSweepParams& p, int grid,
                            cudaStream_t st) {
    KernelEntry* e = pick_any(key_bytes, from_s, radix_bits, tile);
    if (!e) return cudaErrorInvalidValue;
    if (grid <= 0 || grid > e->grid) grid = e->grid;
    OneSweepParams a = p;
    void* args[] = {&a};
    return cudaLaunchKernel(e->fn, dim3(grid), dim3(e->threads), args, e->smem, st);
}

cudaError_t launch_hist_bytes(const uint8_t* S, const BlockInfo* blocks, const TileDesc* tiles, uint32_t num_tiles,
                              uint32_t* hist, cudaStream_t st, const uint32_t* num_tiles_dev) {
    if (num_tiles == 0 && !num_tiles_dev) return cudaSuccess;
    const int grid = num_tiles_dev ? num_sms() * 8 : (int)std::min<uint32_t>(num_tiles, (uint32_t)num_sms() * 8);
    k_hist_bytes<<<grid, 256, 0, st>>>(S, blocks, tiles, num_tiles, num_tiles_dev, hist);
    return cudaGetLastError();
}

cudaError_t launch_hist_keys11(const uint8_t* S, const BlockInfo* blocks, const TileDesc* tiles, uint32_t num_tiles,
                               int tile, uint32_t* hist, cudaStream_t st, const uint32_t* num_tiles_dev) {
    if (num_tiles == 0 && !num_tiles_dev) return cudaSuccess;
    const size_t smem = 6 * 2048 * 4 + (size_t)tile + 48;
    static bool attr = [] {
        cudaFuncSetAttribute((void*)k_hist_keys11<4096>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             6 * 2048 * 4 + 4096 + 48);
        return true;
    }();
    (void)attr;
    const int grid = num_tiles_dev ? num_sms() * 4 : (int)std::min<uint32_t>(num_tiles, (uint32_t)num_sms() * 4);
    k_hist_keys11<4096><<<grid, 256, smem, st>>>(S, blocks, tiles, num_tiles, num_tiles_dev, hist);
    return cudaGetLastError();
}

cudaError_t launch_scan_rows(uint32_t* hist, int radix, const uint32_t* num_rows_dev, uint32_t rows_mult,
                             uint32_t rows_host, uint32_t max_rows, cudaStream_t st) {
    if (radix != 256 && radix != 1024 && radix != 2048 && radix != 4096) return cudaErrorInvalidValue;
    const int grid = num_rows_dev ? num_sms() * 8 : (int)std::max<uint32_t>(1, std::min<uint32_t>(rows_host, 65535));
    if (!num_rows_dev && rows_host == 0) return cudaSuccess;
    k_scan_rows<<<grid, 256, 0, st>>>(hist, radix, num_rows_dev, rows_mult, rows_host, max_rows);
    return cudaGetLastError();
}

cudaError_t launch_zero_by_count(uint32_t* p, const uint32_t* count, uint32_t words_per_unit, uint32_t max_words,
                                 cudaStream_t st) {
    k_zero_by_count<<<num_sms() * 4, 256, 0, st>>>(p, count, words_per_unit, max_words);
    return cudaGetLastError();
}

}  // namespace bwt
