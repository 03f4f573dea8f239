// Group naming, prefix-doubling rounds and the L-column gather.
//
// After the first sort the rotations are ordered by their first 8 bytes.
// Lexicographic naming (the paper's Section 2.1 names it among the GPU
// building blocks): every rotation's rank becomes the block-local sorted
// position of the first member of its group of equal keys, so ranks order
// groups and equal ranks mean equal prefixes. A prefix-doubling round with
// shift h (rotations already ordered by their first h bytes) re-sorts every
// group of size > 1 by key2 = rank[(i + h) mod n], which orders the group by
// its first 2h bytes, and renames. Within a group the rotations are kept in
// increasing index order between rounds (every sort is stable or breaks ties
// by the index), so groups that reach 2h >= n -- identical rotations -- end
// lower-index-first.
//
// Round structure (all gathers of a round finish before any rank is
// rewritten, so a round reads one consistent rank array):
//   gather (micro: thread per group; tiny/small/medium: warp per group) and
//   large_prologue (large groups, by tile)
//   -> sorts: micro (sorting network in registers), tiny (bitonic across a
//      warp's lanes), small (warp: 33..64 bitonic in registers by shuffles,
//      larger in shared memory), medium (CTA bitonic in shared memory),
//      large (segmented onesweep radix)
//   -> renames (fused into the small sorts; rename_large for large groups).
// Refined groups are appended to the next round's size-class bins. A group
// whose key2 are all equal cannot split: it keeps its order and ranks and is
// passed on whole (small and medium groups check first; large groups are
// flagged by the prologue and skipped by the radix and the rename). A rank
// is written only where it changes.
#include <algorithm>

#include "kernels.h"

namespace bwt {

namespace {

// The run of keys equal to K[k] inside a sorted range, found by one warp:
// each round probes 32 positions at once (first exponentially spaced, then
// evenly inside the bracket left), so a run of length r costs about
// 1 + log32(r) dependent global reads instead of 2 log2(r). All 32 lanes
// call and all return the result.

// First index f in [lo, k] with K[f] == key (K sorted on [lo, k], K[k] == key).
template <typename KeyT>
__device__ __forceinline__ uint32_t warp_run_start(const KeyT* __restrict__ K, uint32_t lo, uint32_t k, KeyT key) {
    const uint32_t lane = threadIdx.x & 31;
    int64_t a = (int64_t)lo - 1, b = k;  // K[a] != key (or a < lo), K[b] == key
    {
        const int64_t p = (int64_t)k - (int64_t)(1ull << lane);  // decreasing with the lane
        const bool eq = p > a && K[p] == key;
        const uint32_t m = __popc(__ballot_sync(0xffffffffu, eq));  // equal probes: lanes 0 .. m-1
        if (m > 0) b = (int64_t)k - (int64_t)(1ull << (m - 1));
        if (m < 32) a = max(a, (int64_t)k - (int64_t)(1ull << m));
    }
    while (b - a > 1) {
        const int64_t span = b - a;
        const int64_t p = a + 1 + (span - 1) * (int64_t)lane / 32;  // increasing, inside (a, b)
        const uint32_t eqm = __ballot_sync(0xffffffffu, K[p] == key);  // equal probes: a suffix of lanes
        if (eqm == 0u) {
            a = a + 1 + (span - 1) * 31 / 32;
        } else {
            const int l = __ffs(eqm) - 1;
            const int64_t nb = a + 1 + (span - 1) * l / 32;
            if (l > 0) a = a + 1 + (span - 1) * (l - 1) / 32;
            b = nb;
        }
    }
    return (uint32_t)b;
}

// First index e in (k, hi] with e == hi or K[e] != key (K sorted on [k, hi),
// K[k] == key).
template <typename KeyT>
__device__ __forceinline__ uint32_t warp_run_end(const KeyT* __restrict__ K, uint32_t k, uint32_t hi, KeyT key) {
    const uint32_t lane = threadIdx.x & 31;
    int64_t a = k, b = hi;  // K[a] == key; b == hi or K[b] != key
    {
        const int64_t p = (int64_t)k + (int64_t)(1ull << lane);  // increasing with the lane
        const bool eq = p < b && K[p] == key;
        const uint32_t m = __popc(__ballot_sync(0xffffffffu, eq));  // equal probes: lanes 0 .. m-1
        if (m > 0) a = (int64_t)k + (int64_t)(1ull << (m - 1));
        if (m < 32) b = min(b, (int64_t)k + (int64_t)(1ull << m));
    }
    while (b - a > 1) {
        const int64_t span = b - a;
        const int64_t p = a + 1 + (span - 1) * (int64_t)lane / 32;  // increasing, inside (a, b)
        const uint32_t eqm = __ballot_sync(0xffffffffu, K[p] == key);  // equal probes: a prefix of lanes
        const int m = __popc(eqm);
        if (m == 0) {
            b = a + 1;
        } else {
            const int64_t na = a + 1 + (span - 1) * (m - 1) / 32;
            if (m < 32) b = a + 1 + (span - 1) * m / 32;
            a = na;
        }
    }
    return (uint32_t)b;
}

// Carries of a sorted tile [start, start + len) inside the sorted range
// [lo, hi): the start of the run holding its first key and the end of the
// run holding its last key. Warp 0 calls (all lanes); lane 0 writes them.
template <typename KeyT>
__device__ __forceinline__ void tile_carries(const KeyT* __restrict__ K, uint32_t lo, uint32_t hi, uint32_t start,
                                             uint32_t len, uint32_t* s_carry) {
    const uint32_t last = start + len - 1;
    const KeyT k0 = K[start], k1 = K[last];
    uint32_t c0 = start, c1 = last + 1;
    if (start > lo && K[start - 1] == k0) c0 = warp_run_start<KeyT>(K, lo, start, k0);
    if (last + 1 < hi && K[last + 1] == k1) c1 = warp_run_end<KeyT>(K, last, hi, k1);
    if ((threadIdx.x & 31) == 0) {
        s_carry[0] = c0;
        s_carry[1] = c1;
    }
}

// ---- first naming ------------------------------------------------------------
// seg_bounds: every tile's segment [segStart, segStart + pad0) is a whole
// range of groups (its first element starts a group, its last ends one), so
// the carries never look past it; else the carries search the whole block.
// num_tiles_dev, when non-null, holds the tile count on the device. Tiles
// are taken in order from an atomic counter (zeroed before the launch), so
// the tiles in flight stay within a few blocks: the rank writes of a block
// land while its rank range is still in L2 (a fixed grid stride lets the
// CTAs drift apart over many tiles; at 1,200 blocks that doubled the DRAM
// traffic).
__global__ void __launch_bounds__(256) k_name_initial(const uint64_t* __restrict__ K, const uint32_t* __restrict__ SA,
                                                      const BlockInfo* __restrict__ blocks,
                                                      const TileDesc* __restrict__ tiles, uint32_t num_tiles,
                                                      const uint32_t* __restrict__ num_tiles_dev, bool seg_bounds,
                                                      uint32_t* __restrict__ rank, Bins bins, uint32_t* ctrl,
                                                      uint32_t* __restrict__ tile_counter) {
    // the tile's keys and SA entries (dynamic: 48 KB; the naming loop reads
    // SA from shared memory, so it needs no register array and unrolls by 2)
    extern __shared__ __align__(16) unsigned char name_smem[];
    uint64_t* sk = reinterpret_cast<uint64_t*>(name_smem);
    uint32_t* ssa = reinterpret_cast<uint32_t*>(name_smem + 4096 * 8);
    __shared__ uint32_t s_carry[2];
    __shared__ uint32_t s_t;
    __shared__ GroupDesc ebuf[8][NCLS * EMIT_BUF];
    if (ld_volatile(&ctrl[CTRL_ERR])) return;  // an earlier stage failed: SA is not a permutation
    WarpEmitter em;
    em.init(ebuf[threadIdx.x >> 5]);
    if (num_tiles_dev) num_tiles = *num_tiles_dev;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(tile_counter, 1u);
        __syncthreads();
        const uint32_t t = s_t;
        if (t >= num_tiles) break;
        const TileDesc td = tiles[t];
        const BlockInfo bi = blocks[td.blk];
        const uint32_t lo = seg_bounds ? td.segStart : bi.off;
        const uint32_t hi = seg_bounds ? td.segStart + td.pad0 : bi.off + bi.n;
#pragma unroll
        for (int it = 0; it < 16; ++it) {  // tiles hold at most 4096 keys
            const uint32_t q = it * 256u + threadIdx.x;
            if (q < td.len) {
                sk[q] = K[td.start + q];
                ssa[q] = SA[td.start + q];
            }
        }
        if (threadIdx.x < 32) tile_carries<uint64_t>(K, lo, hi, td.start, td.len, s_carry);
        __syncthreads();
        name_tile<uint64_t>(sk, td.len, td.start, s_carry[0], s_carry[1], ssa, bi, td.blk, rank, bins,
                            bi.n > 8u, NO_OLD_START, em, &ctrl[CTRL_ERR]);
        __syncthreads();
    }
    em.finish(bins, &ctrl[CTRL_ERR]);
}

// ---- round: key gathers ------------------------------------------------------
__global__ void __launch_bounds__(256) k_gather_micro(const uint32_t* __restrict__ SA, const uint32_t* __restrict__ rank,
                                                      const BlockInfo* __restrict__ blocks, Bins cur,
                                                      const uint32_t* __restrict__ depth, uint32_t* __restrict__ key2,
                                                      const LazyRanks lz) {
    const uint32_t h = *depth;
    const uint32_t count = bin_count(cur, 0);
    // one thread per member (a micro group has at most MICRO_MAX), so the
    // members' rank reads -- a search each where ranks are found on demand --
    // run side by side
    const uint64_t total = (uint64_t)count * MICRO_MAX;
    for (uint64_t x = blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t g = (uint32_t)(x / MICRO_MAX), e = (uint32_t)(x % MICRO_MAX);
        const GroupDesc gd = cur.list[0][g];
        if (e >= gd.len) continue;
        const BlockInfo bi = blocks[gd.blk];
        uint32_t r = SA[gd.start + e] + h;
        if (r >= bi.n) r -= bi.n;
        key2[gd.start + e] = r < bi.n ? rank_at(lz, rank, bi, gd.blk, r) : 0u;
    }
}

// tiny, small and medium groups: one warp per group
__global__ void __launch_bounds__(256) k_gather_small(const uint32_t* __restrict__ SA, const uint32_t* __restrict__ rank,
                                                      const BlockInfo* __restrict__ blocks, Bins cur,
                                                      const uint32_t* __restrict__ depth, uint32_t* __restrict__ key2,
                                                      const LazyRanks lz) {
    const uint32_t h = *depth;
    const uint32_t c1 = bin_count(cur, 1), c2 = bin_count(cur, 2), c3 = bin_count(cur, 3);
    const uint32_t total = c1 + c2 + c3;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    auto desc = [&](uint32_t g) {
        return g < c1 ? cur.list[1][g] : (g < c1 + c2 ? cur.list[2][g - c1] : cur.list[3][g - c1 - c2]);
    };
    // two groups a warp (g and g + nwarps), their chains of loads interleaved:
    // the gather is bound by the latency of descriptor -> SA -> rank
    for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < total; g += 2 * nwarps) {
        const uint32_t g1 = g + nwarps;
        const GroupDesc gd0 = desc(g);
        const GroupDesc gd1 = g1 < total ? desc(g1) : GroupDesc{0u, 0u, 0u, 0u};
        const BlockInfo b0 = blocks[gd0.blk];
        const BlockInfo b1 = blocks[gd1.blk];
        const uint32_t len = max(gd0.len, gd1.len);
        // U elements of each group a lane per step (medium groups run to
        // 2,048): all their SA loads, then all their rank gathers, in flight
        constexpr int U = 4;
        for (uint32_t e0 = lane; e0 < len; e0 += 32 * U) {
            uint32_t s0[U], s1[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t e = e0 + 32 * u;
                s0[u] = e < gd0.len ? SA[gd0.start + e] : 0u;
                s1[u] = e < gd1.len ? SA[gd1.start + e] : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t e = e0 + 32 * u;
                const bool v0 = e < gd0.len, v1 = e < gd1.len;
                uint32_t r0 = s0[u] + h, r1 = s1[u] + h;
                if (r0 >= b0.n) r0 -= b0.n;
                if (r1 >= b1.n) r1 -= b1.n;
                s0[u] = v0 && r0 < b0.n ? rank_at(lz, rank, b0, gd0.blk, r0) : 0u;
                s1[u] = v1 && r1 < b1.n ? rank_at(lz, rank, b1, gd1.blk, r1) : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t e = e0 + 32 * u;
                if (e < gd0.len) key2[gd0.start + e] = s0[u];
                if (e < gd1.len) key2[gd1.start + e] = s1[u];
            }
        }
    }
}

// One CTA: numbers the tiles of every large group (a block scan over 1,024
// groups at a time), then all threads write the tiles, each finding its
// tile's group by binary search over the scanned first tiles (a group of
// 900,000 rotations has 220 tiles: written by one thread they took most of
// the kernel's time).
__global__ void __launch_bounds__(1024) k_build_large_tiles(Bins cur, int tile, TileDesc* __restrict__ tiles,
                                                            uint32_t max_tiles, uint32_t* ctrl,
                                                            uint32_t* __restrict__ seg_varied) {
    __shared__ uint32_t tmp[32];
    __shared__ uint32_t s_keys;
    __shared__ uint32_t s_first[1024];  // first tile of each group of the chunk, relative to the chunk
    __shared__ GroupDesc s_gd[1024];
    if (threadIdx.x == 0) s_keys = 0;
    __syncthreads();
    const uint32_t n = bin_count(cur, CLS_LARGE);
    uint32_t running = 0, keys = 0;
    for (uint32_t base = 0; base < n; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        GroupDesc gd{0, 0, 0, 0};
        uint32_t nt = 0;
        if (i < n) {
            gd = cur.list[CLS_LARGE][i];
            nt = (gd.len + tile - 1) / tile;
            keys += gd.len;
            if (seg_varied) seg_varied[i] = 0u;  // set by the prologue if the group's key2 differ
        }
        uint32_t tot;
        s_first[threadIdx.x] = block_exclusive_scan<1024>(nt, tmp, &tot);  // non-decreasing
        s_gd[threadIdx.x] = gd;
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < tot; k += 1024) {
            uint32_t lo = 0, hi = 1024;  // the last group whose first tile is <= k (it has tiles)
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_first[mid] <= k) lo = mid; else hi = mid;
            }
            const GroupDesc g = s_gd[lo];
            const uint32_t j = k - s_first[lo], ti = running + k;
            if (ti < max_tiles) {
                TileDesc td;
                td.start = g.start + j * tile;
                td.len = min((uint32_t)tile, g.len - j * tile);
                td.seg = base + lo;
                td.firstTile = running + s_first[lo];
                td.segStart = g.start;
                td.blk = g.blk;
                td.pad0 = g.len;
                td.pad1 = 0;
                tiles[ti] = td;
            }
        }
        running += tot;
        __syncthreads();  // the chunk's tables are read before the next chunk rewrites them
    }
    keys = __reduce_add_sync(0xffffffffu, keys);
    if ((threadIdx.x & 31) == 0 && keys) atomicAdd(&s_keys, keys);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (running > max_tiles) {
            atomicOr(&ctrl[CTRL_ERR], ERR_CAPACITY);
            running = max_tiles;
        }
        ctrl[CTRL_NUM_LTILES] = running;
        ctrl[CTRL_LARGE_KEYS] = s_keys;
    }
}

template <int RBITS>
__global__ void __launch_bounds__(256) k_large_prologue(const uint32_t* __restrict__ SA,
                                                        const uint32_t* __restrict__ rank,
                                                        const BlockInfo* __restrict__ blocks,
                                                        const TileDesc* __restrict__ tiles,
                                                        const uint32_t* __restrict__ num_tiles,
                                                        const uint32_t* __restrict__ depth,
                                                        uint32_t* __restrict__ kbuf, uint32_t* __restrict__ vbuf,
                                                        uint32_t* __restrict__ hist, int passes,
                                                        uint32_t* __restrict__ seg_varied, const LazyRanks lz) {
    constexpr int RADIX = 1 << RBITS;
    const uint32_t h = *depth;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* sh = reinterpret_cast<uint32_t*>(smem);
    const int lane = threadIdx.x & 31;
    const uint32_t nt = *num_tiles;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) sh[i] = 0;
        __syncthreads();
        const TileDesc td = tiles[t];
        const BlockInfo bi = blocks[td.blk];
        // key2 of the group's first member: the group does not move this
        // round if every member has it
        uint32_t k0;
        {
            uint32_t r = SA[td.segStart] + h;
            if (r >= bi.n) r -= bi.n;
            k0 = r < bi.n ? rank_at(lz, rank, bi, td.blk, r) : 0u;
        }
        bool same = true;
        // PI elements a thread per step: their SA loads, then their rank
        // gathers, are all in flight at once
        constexpr int PI = 4;
        for (uint32_t q0 = 0; q0 < td.len; q0 += 256u * PI) {
            uint32_t sa[PI], k2[PI];
#pragma unroll
            for (int j = 0; j < PI; ++j) {
                const uint32_t q = q0 + j * 256u + threadIdx.x;
                sa[j] = q < td.len ? SA[td.start + q] : 0u;
            }
#pragma unroll
            for (int j = 0; j < PI; ++j) {
                const uint32_t q = q0 + j * 256u + threadIdx.x;
                k2[j] = 0u;
                if (q < td.len) {
                    uint32_t r = sa[j] + h;
                    if (r >= bi.n) r -= bi.n;
                    k2[j] = r < bi.n ? rank_at(lz, rank, bi, td.blk, r) : 0u;
                }
            }
#pragma unroll
            for (int j = 0; j < PI; ++j) {
                const uint32_t q = q0 + j * 256u + threadIdx.x;
                const bool valid = q < td.len;
                if (valid) {
                    kbuf[td.start + q] = k2[j];
                    if (vbuf) vbuf[td.start + q] = sa[j];
                    same &= k2[j] == k0;
                }
                for (int ps = 0; ps < passes; ++ps) {
                    const uint32_t d = valid ? ((k2[j] >> (ps * RBITS)) & (RADIX - 1)) : (uint32_t)RADIX;
                    const uint32_t peers = __match_any_sync(0xffffffffu, d);
                    if (valid && lane == __ffs(peers) - 1) atomicAdd(&sh[ps * RADIX + d], (uint32_t)__popc(peers));
                }
            }
        }
        if (__syncthreads_or(!same) && threadIdx.x == 0) seg_varied[td.seg] = 1u;
        for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) {
            const uint32_t c = sh[i];
            if (c) atomicAdd(&hist[(size_t)td.seg * passes * RADIX + i], c);
        }
        __syncthreads();
    }
}

// ---- round: small-group sorts + rename ------------------------------------------

// micro groups (2..4 rotations): one thread each, a 4-input sorting network
__global__ void __launch_bounds__(256) k_sort_micro(uint32_t* __restrict__ SA, const uint32_t* __restrict__ key2,
                                                    uint32_t* __restrict__ rank, const BlockInfo* __restrict__ blocks,
                                                    Bins cur, Bins next, const uint32_t* __restrict__ depth,
                                                    uint32_t* ctrl) {
    __shared__ GroupDesc ebuf[8][NCLS * EMIT_BUF];
    if (ld_volatile(&ctrl[CTRL_ERR])) return;
    const uint32_t new_depth = 2u * *depth;
    const uint32_t count = bin_count(cur, 0);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    WarpEmitter em;
    em.init(ebuf[threadIdx.x >> 5]);
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < count; base += stride) {
        const uint32_t g = base + lane;
        const bool valid = g < count;
        GroupDesc gd{0, 0, 0, 0};
        BlockInfo bi{0, 0};
        uint64_t c[4] = {~0ull, ~0ull, ~0ull, ~0ull};
        if (valid) {
            gd = cur.list[0][g];
            bi = blocks[gd.blk];
            for (uint32_t e = 0; e < gd.len && e < 4; ++e)
                c[e] = ((uint64_t)key2[gd.start + e] << 32) | SA[gd.start + e];
        }
        auto cx = [](uint64_t& a, uint64_t& b) {
            const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
            a = lo;
            b = hi;
        };
        cx(c[0], c[1]);
        cx(c[2], c[3]);
        cx(c[0], c[2]);
        cx(c[1], c[3]);
        cx(c[1], c[2]);
        bool want0 = false, want1 = false;
        uint32_t s0 = 0, l0 = 0, s1 = 0, l1 = 0;
        if (valid) {
            uint32_t gstart[4] = {0, 0, 0, 0};
            uint32_t cur_start = 0;
            for (uint32_t e = 0; e < gd.len && e < 4; ++e) {
                if (e > 0 && (uint32_t)(c[e] >> 32) != (uint32_t)(c[e - 1] >> 32)) cur_start = e;
                gstart[e] = cur_start;
            }
            int emitted = 0;
            for (uint32_t e = 0; e < gd.len && e < 4; ++e) {
                const uint32_t sa = (uint32_t)c[e];
                SA[gd.start + e] = sa;
                BWT_DCHECK(sa < bi.n, &ctrl[CTRL_ERR]);
                if (sa < bi.n && gstart[e] != 0) rank[bi.off + sa] = gd.start - bi.off + gstart[e];
                if (gstart[e] == e) {
                    uint32_t f = e + 1;
                    while (f < gd.len && f < 4 && gstart[f] == e) ++f;
                    if (f - e > 1 && new_depth < bi.n) {
                        if (emitted == 0) {
                            want0 = true;
                            s0 = gd.start + e;
                            l0 = f - e;
                        } else {
                            want1 = true;
                            s1 = gd.start + e;
                            l1 = f - e;
                        }
                        ++emitted;
                    }
                }
            }
        }
        em.emit(next, want0, s0, l0, gd.blk, &ctrl[CTRL_ERR]);
        em.emit(next, want1, s1, l1, gd.blk, &ctrl[CTRL_ERR]);
    }
    em.finish(next, &ctrl[CTRL_ERR]);
}

// tiny groups (5..32): one warp each, bitonic across the lanes
__global__ void __launch_bounds__(256) k_sort_tiny(uint32_t* __restrict__ SA, const uint32_t* __restrict__ key2,
                                                   uint32_t* __restrict__ rank, const BlockInfo* __restrict__ blocks,
                                                   Bins cur, Bins next, const uint32_t* __restrict__ depth,
                                                   uint32_t* ctrl) {
    __shared__ GroupDesc ebuf[8][NCLS * EMIT_BUF];
    if (ld_volatile(&ctrl[CTRL_ERR])) return;
    const uint32_t new_depth = 2u * *depth;
    const uint32_t count = bin_count(cur, 1);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    WarpEmitter em;
    em.init(ebuf[threadIdx.x >> 5]);
    for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < count; g += nwarps) {
        const GroupDesc gd = cur.list[1][g];
        const BlockInfo bi = blocks[gd.blk];
        const bool valid = lane < gd.len;
        const uint32_t k = gd.start + lane;
        uint64_t c = valid ? (((uint64_t)key2[k] << 32) | SA[k]) : ~0ull;
#pragma unroll
        for (uint32_t kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
            for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
                const uint64_t o = __shfl_xor_sync(0xffffffffu, c, j);
                const bool up = (lane & kk) == 0;
                const bool lower = (lane & j) == 0;
                c = (lower == up) ? (c < o ? c : o) : (c > o ? c : o);
            }
        }
        const uint32_t key = (uint32_t)(c >> 32), sa = (uint32_t)c;
        const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
        const bool head = valid && (lane == 0 || prev != key);
        const uint32_t hm = __ballot_sync(0xffffffffu, head);
        const uint32_t le = (2u << lane) - 1u;  // lanes <= lane (lane 31 wraps to all ones)
        const uint32_t start_lane = 31u - __clz(hm & le);
        const uint32_t above = hm & ~le;
        const uint32_t end = above ? (uint32_t)(__ffs(above) - 1) : gd.len;
        if (valid) {
            SA[k] = sa;
            BWT_DCHECK(!valid || sa < bi.n, &ctrl[CTRL_ERR]);
            if (sa < bi.n && start_lane != 0) rank[bi.off + sa] = gd.start - bi.off + start_lane;
        }
        const uint32_t len = end - lane;
        const bool want = head && len > 1 && new_depth < bi.n;
        em.emit(next, want, k, len, gd.blk, &ctrl[CTRL_ERR]);
    }
    em.finish(next, &ctrl[CTRL_ERR]);
}

template <int NT>
__device__ __forceinline__ void coop_sync() {
    if constexpr (NT == 32) __syncwarp(); else __syncthreads();
}

// Sorts comp[0..P) (P a power of two) by bitonic merging; NT threads
// cooperate (a warp or the CTA), t is the thread's index among them. Each
// step has P/2 compare-exchanges; thread t takes pairs t, t + NT, ..: pair
// p is (i, i + j) with i = p with a zero bit inserted at j's position.
template <int NT>
__device__ __forceinline__ void coop_bitonic(uint64_t* comp, uint32_t P, uint32_t t) {
    const uint32_t half = P >> 1;
    for (uint32_t kk = 2; kk <= P; kk <<= 1) {
        for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
            for (uint32_t pr = t; pr < half; pr += NT) {
                const uint32_t i = ((pr & ~(j - 1)) << 1) | (pr & (j - 1));
                const uint32_t ixj = i | j;
                const uint64_t a = comp[i], b = comp[ixj];
                const bool up = (i & kk) == 0;
                if ((a > b) == up) {
                    comp[i] = b;
                    comp[ixj] = a;
                }
            }
            coop_sync<NT>();
        }
    }
}

// Loads a group's (key2, SA) composites, sorts them, writes SA back, renames
// and emits refined groups. NT threads (a warp or the CTA) cooperate.
template <int NT>
__device__ __forceinline__ void sort_rename_group(uint64_t* comp, const GroupDesc& gd, const BlockInfo& bi,
                                                  uint32_t* __restrict__ SA, const uint32_t* __restrict__ key2,
                                                  uint32_t* __restrict__ rank, const Bins& next, uint32_t new_depth,
                                                  WarpEmitter& em, uint32_t* err, uint32_t t) {
    const uint32_t m = gd.len;
    uint32_t P = 32;
    while (P < m) P <<= 1;
    static_assert((NT == 32 ? SMALL_MAX : MED_MAX) <= 8 * NT, "a group fits 8 elements a thread");
    // A group whose members all have the same key2 cannot split: it stays in
    // index order with its ranks (every member already holds the group's
    // start) and only moves on to the next round. Periodic blocks keep such
    // groups of identical rotations for every round until 2h >= n.
    const uint32_t k0 = key2[gd.start];
    if (key2[gd.start + m - 1] == k0) {  // else the group splits for sure: no full check
        bool mine = true;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t i = t + j * NT;
            if (i < m) mine &= key2[gd.start + i] == k0;
        }
        bool same;
        if constexpr (NT == 32) same = __all_sync(0xffffffffu, mine);
        else same = __syncthreads_and(mine);
        if (same) {
            em.emit(next, t == 0 && new_depth < bi.n, gd.start, m, gd.blk, err);
            return;
        }
    }
    bool sorted = false;
    if constexpr (NT == 32) {
        if (P == 64) {
            // 33..64 elements: element e = r * 32 + t in register c[r]; the
            // bitonic network by shuffles (its one distance-32 step pairs a
            // lane's own two elements), then the result to shared memory
            uint64_t c0 = t < m ? (((uint64_t)key2[gd.start + t] << 32) | SA[gd.start + t]) : ~0ull;
            uint64_t c1 = t + 32 < m ? (((uint64_t)key2[gd.start + t + 32] << 32) | SA[gd.start + t + 32]) : ~0ull;
#pragma unroll
            for (uint32_t kk = 2; kk <= 64; kk <<= 1) {
#pragma unroll
                for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
                    if (j == 32) {  // kk == 64: both elements in the ascending half
                        const uint64_t lo = c0 < c1 ? c0 : c1, hi = c0 < c1 ? c1 : c0;
                        c0 = lo;
                        c1 = hi;
                    } else {
                        const uint64_t o0 = __shfl_xor_sync(0xffffffffu, c0, j);
                        const uint64_t o1 = __shfl_xor_sync(0xffffffffu, c1, j);
                        const bool lower = (t & j) == 0;
                        const bool up0 = (t & kk) == 0, up1 = ((t + 32) & kk) == 0;
                        c0 = (lower == up0) ? (c0 < o0 ? c0 : o0) : (c0 > o0 ? c0 : o0);
                        c1 = (lower == up1) ? (c1 < o1 ? c1 : o1) : (c1 > o1 ? c1 : o1);
                    }
                }
            }
            comp[t] = c0;
            comp[t + 32] = c1;
            __syncwarp();
            sorted = true;
        }
    }
    if (!sorted) {
        // up to 8 elements a thread (P <= 8 NT): all loads in flight before any store
        uint32_t lk[8], ls[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t i = t + j * NT;
            lk[j] = i < m ? key2[gd.start + i] : 0u;
            ls[j] = i < m ? SA[gd.start + i] : 0u;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t i = t + j * NT;
            if (i < P) comp[i] = i < m ? (((uint64_t)lk[j] << 32) | ls[j]) : ~0ull;
        }
        coop_sync<NT>();
        coop_bitonic<NT>(comp, P, t);
    }
    if constexpr (NT == 32) {
        // One warp: group heads by ballot, 32 elements a step. An element's
        // group starts at the last head at or before it (carried across
        // steps); each head closes the group before it, and the last group
        // is closed after the loop.
        const bool emit_ok = new_depth < bi.n;
        uint32_t last_head = 0;
        for (uint32_t i0 = 0; i0 < m; i0 += 32) {
            const uint32_t i = i0 + t;
            const bool valid = i < m;
            const uint64_t c = valid ? comp[i] : 0ull;
            const uint32_t key = (uint32_t)(c >> 32), sa = (uint32_t)c;
            const bool head = valid && (i == 0 || (uint32_t)(comp[i - 1] >> 32) != key);
            const uint32_t hm = __ballot_sync(0xffffffffu, head);
            const uint32_t lt = (1u << t) - 1u;  // lanes below t
            const uint32_t hle = hm & (lt | (1u << t));
            const uint32_t s = hle ? i0 + 31u - __clz(hle) : last_head;
            if (valid) {
                SA[gd.start + i] = sa;
                BWT_DCHECK(sa < bi.n, err);
                if (sa < bi.n && s != 0) rank[bi.off + sa] = gd.start - bi.off + s;
            }
            bool want = false;
            uint32_t ps = 0, len = 0;
            if (head && i > 0) {
                const uint32_t hlt = hm & lt;
                ps = hlt ? i0 + 31u - __clz(hlt) : last_head;
                len = i - ps;
                want = len > 1 && emit_ok;
            }
            em.emit(next, want, gd.start + ps, len, gd.blk, err);
            if (hm) last_head = i0 + 31u - __clz(hm);
        }
        const uint32_t len = m - last_head;
        em.emit(next, t == 0 && len > 1 && emit_ok, gd.start + last_head, len, gd.blk, err);
        __syncwarp();
        return;
    }
    for (uint32_t i0 = 0; i0 < m; i0 += NT) {
        const uint32_t i = i0 + t;
        const bool valid = i < m;
        bool want = false;
        uint32_t len = 0;
        if (valid) {
            const uint64_t c = comp[i];
            const uint32_t key = (uint32_t)(c >> 32), sa = (uint32_t)c;
            const bool head = (i == 0) || (uint32_t)(comp[i - 1] >> 32) != key;
            const uint32_t s = head ? i : smem_lower_bound<uint64_t>(comp, m, (uint64_t)key << 32);
            SA[gd.start + i] = sa;
            BWT_DCHECK(sa < bi.n, err);
                if (sa < bi.n && s != 0) rank[bi.off + sa] = gd.start - bi.off + s;
            if (head) {
                len = smem_lower_bound<uint64_t>(comp, m, (uint64_t)(key + 1) << 32) - i;
                want = len > 1 && new_depth < bi.n;
            }
        }
        em.emit(next, want, gd.start + i, len, gd.blk, err);
    }
    coop_sync<NT>();
}

// small groups (33..256): one warp each, bitonic in the warp's shared memory
__global__ void __launch_bounds__(256) k_sort_small(uint32_t* __restrict__ SA, const uint32_t* __restrict__ key2,
                                                    uint32_t* __restrict__ rank, const BlockInfo* __restrict__ blocks,
                                                    Bins cur, Bins next, const uint32_t* __restrict__ depth,
                                                    uint32_t* ctrl) {
    __shared__ uint64_t comp[8][SMALL_MAX];
    __shared__ GroupDesc ebuf[8][NCLS * EMIT_BUF];
    if (ld_volatile(&ctrl[CTRL_ERR])) return;
    const uint32_t new_depth = 2u * *depth;
    const uint32_t count = bin_count(cur, 2);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    WarpEmitter em;
    em.init(ebuf[warp]);
    for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < count; g += nwarps) {
        const GroupDesc gd = cur.list[2][g];
        const BlockInfo bi = blocks[gd.blk];
        sort_rename_group<32>(comp[warp], gd, bi, SA, key2, rank, next, new_depth, em, &ctrl[CTRL_ERR], lane);
    }
    em.finish(next, &ctrl[CTRL_ERR]);
}

// medium groups (257..2048): one CTA each, bitonic in shared memory
__global__ void __launch_bounds__(256) k_sort_med(uint32_t* __restrict__ SA, const uint32_t* __restrict__ key2,
                                                  uint32_t* __restrict__ rank, const BlockInfo* __restrict__ blocks,
                                                  Bins cur, Bins next, const uint32_t* __restrict__ depth,
                                                  uint32_t* ctrl) {
    __shared__ uint64_t comp[MED_MAX];
    __shared__ GroupDesc ebuf[8][NCLS * EMIT_BUF];
    if (ld_volatile(&ctrl[CTRL_ERR])) return;
    const uint32_t new_depth = 2u * *depth;
    const uint32_t count = bin_count(cur, 3);
    WarpEmitter em;
    em.init(ebuf[threadIdx.x >> 5]);
    for (uint32_t g = blockIdx.x; g < count; g += gridDim.x) {
        const GroupDesc gd = cur.list[3][g];
        const BlockInfo bi = blocks[gd.blk];
        sort_rename_group<256>(comp, gd, bi, SA, key2, rank, next, new_depth, em, &ctrl[CTRL_ERR], threadIdx.x);
    }
    em.finish(next, &ctrl[CTRL_ERR]);
}

// large groups after their radix sort: rename by tile (binary search in the
// tile in shared memory; one global search per tile end for runs that cross
// it) and emit refined groups
__global__ void __launch_bounds__(256) k_rename_large(const uint32_t* __restrict__ SA, const uint32_t* __restrict__ key2,
                                                      uint32_t* __restrict__ rank,
                                                      const BlockInfo* __restrict__ blocks,
                                                      const TileDesc* __restrict__ tiles,
                                                      const uint32_t* __restrict__ num_tiles, Bins next,
                                                      const uint32_t* __restrict__ depth,
                                                      const uint32_t* __restrict__ seg_varied, uint32_t* ctrl) {
    __shared__ uint32_t sk[4096];
    __shared__ uint32_t ssa[4096];
    __shared__ uint32_t s_carry[2];
    __shared__ GroupDesc ebuf[8][NCLS * EMIT_BUF];
    if (ld_volatile(&ctrl[CTRL_ERR])) return;
    const uint32_t new_depth = 2u * *depth;
    const uint32_t nt = *num_tiles;
    WarpEmitter em;
    em.init(ebuf[threadIdx.x >> 5]);
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const TileDesc td = tiles[t];
        const BlockInfo bi = blocks[td.blk];
        if (seg_varied[td.seg] == 0u) {
            // every key2 of the group is the same: the radix left it alone, it
            // does not split and its ranks stand; it moves on whole (once, from
            // its first tile); no shared memory is touched on this path
            em.emit(next, threadIdx.x == 0 && td.start == td.segStart && new_depth < bi.n, td.segStart, td.pad0,
                    td.blk, &ctrl[CTRL_ERR]);
            continue;
        }
        const uint32_t lo = td.segStart, hi = td.segStart + td.pad0;
#pragma unroll
        for (int it = 0; it < 16; ++it) {  // tiles hold at most 4096 keys
            const uint32_t q = it * 256u + threadIdx.x;
            if (q < td.len) {
                sk[q] = key2[td.start + q];
                ssa[q] = SA[td.start + q];
            }
        }
        if (threadIdx.x < 32) tile_carries<uint32_t>(key2, lo, hi, td.start, td.len, s_carry);
        __syncthreads();
        name_tile<uint32_t>(sk, td.len, td.start, s_carry[0], s_carry[1], ssa, bi, td.blk, rank, next,
                            new_depth < bi.n, td.segStart, em, &ctrl[CTRL_ERR]);
        __syncthreads();
    }
    em.finish(next, &ctrl[CTRL_ERR]);
}

// Tiles in order from an atomic counter (zeroed before the launch): the
// blocks whose bytes are gathered stay few, so their S stays in L2.
__global__ void __launch_bounds__(256) k_gather_L(const uint8_t* __restrict__ S, const uint32_t* __restrict__ SA,
                                                  const BlockInfo* __restrict__ blocks,
                                                  const TileDesc* __restrict__ tiles, uint32_t num_tiles,
                                                  uint8_t* __restrict__ L, int32_t* __restrict__ primary,
                                                  uint32_t* __restrict__ tile_counter, uint32_t* err) {
    __shared__ uint32_t s_t;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(tile_counter, 1u);
        __syncthreads();
        const uint32_t t = s_t;
        if (t >= num_tiles) break;
        const TileDesc td = tiles[t];
        const BlockInfo bi = blocks[td.blk];
        // four elements a thread per step: their SA loads, then their byte
        // gathers, are all in flight at once
        constexpr int PI = 4;
        for (uint32_t q0 = 0; q0 < td.len; q0 += 256u * PI) {
            uint32_t sa[PI];
            uint8_t c[PI];
#pragma unroll
            for (int j = 0; j < PI; ++j) {
                const uint32_t q = q0 + j * 256u + threadIdx.x;
                sa[j] = q < td.len ? SA[td.start + q] : 1u;
            }
#pragma unroll
            for (int j = 0; j < PI; ++j) {
                sa[j] &= ~SA_FINAL;
                BWT_DCHECK(q0 + j * 256u + threadIdx.x >= td.len || sa[j] < bi.n, err);
                const uint32_t src = sa[j] == 0 || sa[j] > bi.n ? bi.n - 1 : sa[j] - 1;
                c[j] = S[bi.off + src];
            }
#pragma unroll
            for (int j = 0; j < PI; ++j) {
                const uint32_t q = q0 + j * 256u + threadIdx.x;
                if (q < td.len) {
                    L[td.start + q] = c[j];
                    if (sa[j] == 0) primary[td.blk] = (int32_t)q + (int32_t)(td.start - bi.off);
                }
            }
        }
        __syncthreads();  // every thread has read s_t before it is replaced
    }
}

int grid_for(uint32_t units, uint32_t per_cta, int cap_per_sm) {
    const uint64_t want = (units + per_cta - 1) / per_cta;
    const uint64_t cap = (uint64_t)num_sms() * cap_per_sm;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, cap));
}

}  // namespace

constexpr size_t NAME_SMEM = 4096 * 8 + 4096 * 4;
constexpr int NAME_CTAS_PER_SM = 3;  // 48 KB dynamic + 10 KB static shared memory each

bool name_attr() {
    static const bool ok = cudaFuncSetAttribute((void*)k_name_initial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)NAME_SMEM) == cudaSuccess;
    return ok;
}

// Tile counters of the naming and the L gather (control words no radix pass
// uses); each launch zeroes its counter first.
constexpr int NAME_CTR = CTRL_TILE_CTR + 56, GATHER_L_CTR = CTRL_TILE_CTR + 57;

cudaError_t launch_name_initial(const uint64_t* K, const uint32_t* SA, const BlockInfo* blocks, const TileDesc* tiles,
                                uint32_t num_tiles, uint32_t* rank, Bins bins, uint32_t* ctrl, cudaStream_t st) {
    if (!num_tiles) return cudaSuccess;
    if (!name_attr()) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(ctrl + NAME_CTR, 0, 4, st);
    if (e != cudaSuccess) return e;
    k_name_initial<<<grid_for(num_tiles, 1, NAME_CTAS_PER_SM), 256, NAME_SMEM, st>>>(
        K, SA, blocks, tiles, num_tiles, nullptr, false, rank, bins, ctrl, ctrl + NAME_CTR);
    return cudaGetLastError();
}

cudaError_t launch_name_tiles(const uint64_t* K, const uint32_t* SA, const BlockInfo* blocks, const TileDesc* tiles,
                              const uint32_t* num_tiles_dev, bool seg_bounds, uint32_t* rank, Bins bins,
                              uint32_t* ctrl, cudaStream_t st) {
    if (!name_attr()) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(ctrl + NAME_CTR, 0, 4, st);
    if (e != cudaSuccess) return e;
    k_name_initial<<<num_sms() * NAME_CTAS_PER_SM, 256, NAME_SMEM, st>>>(K, SA, blocks, tiles, 0u, num_tiles_dev,
                                                                          seg_bounds, rank, bins, ctrl,
                                                                          ctrl + NAME_CTR);
    return cudaGetLastError();
}

cudaError_t launch_gather_small(const uint32_t* SA, const uint32_t* rank, const BlockInfo* blocks, Bins cur,
                                const uint32_t* depth, uint32_t* key2, const uint32_t* host_counts, cudaStream_t st,
                                int* launched, const LazyRanks& lz) {
    int g_micro = num_sms() * 8, g_warp = num_sms() * 16;
    if (host_counts) {
        g_micro = host_counts[0] ? grid_for(std::min(host_counts[0], 0x3fffffffu) * MICRO_MAX, 256, 8) : 0;
        const uint32_t n = host_counts[1] + host_counts[2] + host_counts[3];
        g_warp = n ? grid_for(n, 8, 16) : 0;
    }
    *launched = 0;
    if (g_micro) {
        k_gather_micro<<<g_micro, 256, 0, st>>>(SA, rank, blocks, cur, depth, key2, lz);
        ++*launched;
    }
    if (g_warp) {
        k_gather_small<<<g_warp, 256, 0, st>>>(SA, rank, blocks, cur, depth, key2, lz);
        ++*launched;
    }
    return cudaGetLastError();
}

cudaError_t launch_build_large_tiles(Bins cur, int tile, TileDesc* tiles, uint32_t max_tiles, uint32_t* ctrl,
                                     cudaStream_t st, uint32_t* seg_varied) {
    k_build_large_tiles<<<1, 1024, 0, st>>>(cur, tile, tiles, max_tiles, ctrl, seg_varied);
    return cudaGetLastError();
}

cudaError_t launch_large_prologue(const uint32_t* SA, const uint32_t* rank, const BlockInfo* blocks,
                                  const TileDesc* tiles, const uint32_t* num_tiles, const uint32_t* depth,
                                  uint32_t* kbuf, uint32_t* vbuf, uint32_t* hist, int radix_bits, int passes,
                                  uint32_t* seg_varied, cudaStream_t st, const LazyRanks& lz) {
    const size_t smem = (size_t)passes * (1u << radix_bits) * 4;
    const int grid = num_sms() * 8;
    if (radix_bits == 8) {
        k_large_prologue<8><<<grid, 256, smem, st>>>(SA, rank, blocks, tiles, num_tiles, depth, kbuf, vbuf, hist,
                                                     passes, seg_varied, lz);
    } else if (radix_bits == 10) {
        k_large_prologue<10><<<grid, 256, smem, st>>>(SA, rank, blocks, tiles, num_tiles, depth, kbuf, vbuf, hist,
                                                      passes, seg_varied, lz);
    } else if (radix_bits == 11) {
        static bool attr = [] {
            cudaFuncSetAttribute((void*)k_large_prologue<11>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 4 * 2048 * 4);
            return true;
        }();
        (void)attr;
        k_large_prologue<11><<<grid, 256, smem, st>>>(SA, rank, blocks, tiles, num_tiles, depth, kbuf, vbuf, hist,
                                                      passes, seg_varied, lz);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_sort_small(uint32_t* SA, uint32_t* key2, uint32_t* rank, const BlockInfo* blocks, Bins cur,
                              Bins next, const uint32_t* depth, const uint32_t* host_counts, uint32_t* ctrl,
                              cudaStream_t st, int* launched) {
    int g[4] = {num_sms() * 8, num_sms() * 16, num_sms() * 8, num_sms() * 8};
    if (host_counts) {
        g[0] = host_counts[0] ? grid_for(host_counts[0], 256, 8) : 0;
        g[1] = host_counts[1] ? grid_for(host_counts[1], 8, 16) : 0;
        g[2] = host_counts[2] ? grid_for(host_counts[2], 8, 8) : 0;
        g[3] = host_counts[3] ? grid_for(host_counts[3], 1, 8) : 0;
    }
    *launched = 0;
    if (g[0]) {
        k_sort_micro<<<g[0], 256, 0, st>>>(SA, key2, rank, blocks, cur, next, depth, ctrl);
        ++*launched;
    }
    if (g[1]) {
        k_sort_tiny<<<g[1], 256, 0, st>>>(SA, key2, rank, blocks, cur, next, depth, ctrl);
        ++*launched;
    }
    if (g[2]) {
        k_sort_small<<<g[2], 256, 0, st>>>(SA, key2, rank, blocks, cur, next, depth, ctrl);
        ++*launched;
    }
    if (g[3]) {
        k_sort_med<<<g[3], 256, 0, st>>>(SA, key2, rank, blocks, cur, next, depth, ctrl);
        ++*launched;
    }
    return cudaGetLastError();
}

cudaError_t launch_rename_large(const uint32_t* SA, const uint32_t* key2, uint32_t* rank, const BlockInfo* blocks,
                                const TileDesc* tiles, const uint32_t* num_tiles, Bins next, const uint32_t* depth,
                                const uint32_t* seg_varied, uint32_t* ctrl, cudaStream_t st) {
    k_rename_large<<<num_sms() * 4, 256, 0, st>>>(SA, key2, rank, blocks, tiles, num_tiles, next, depth, seg_varied,
                                                  ctrl);
    return cudaGetLastError();
}

cudaError_t launch_gather_L(const uint8_t* S, const uint32_t* SA, const BlockInfo* blocks, const TileDesc* tiles,
                            uint32_t num_tiles, uint8_t* L, int32_t* primary, uint32_t* ctrl, cudaStream_t st) {
    if (!num_tiles) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(ctrl + GATHER_L_CTR, 0, 4, st);
    if (e != cudaSuccess) return e;
    k_gather_L<<<grid_for(num_tiles, 1, 16), 256, 0, st>>>(S, SA, blocks, tiles, num_tiles, L, primary,
                                                           ctrl + GATHER_L_CTR, ctrl + CTRL_ERR);
    return cudaGetLastError();
}

// ---- control kernels --------------------------------------------------------

__global__ void k_reset_ctrl(uint32_t* ctrl, uint32_t spin, uint32_t withhold, uint32_t ntiles0) {
    for (int i = threadIdx.x; i < CTRL_WORDS; i += blockDim.x) ctrl[i] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        ctrl[CTRL_SPIN] = spin;
        ctrl[CTRL_WITHHOLD] = withhold;
        ctrl[CTRL_NTILES0] = ntiles0;
        ctrl[CTRL_DEPTH] = 8u;
    }
}

__device__ __forceinline__ bool any_groups(const uint32_t* c) {
    uint32_t a = 0;
#pragma unroll
    for (int i = 0; i < NCLS; ++i) a |= c[i];
    return a != 0u;
}

// After a round that read bins[par]: advance the depth if the round had
// work; in graph mode also count the round and set conditions from whether
// another round is due (bins[par ^ 1] holds groups, the prefix is below the
// largest block, no device error, fewer than 40 rounds): flags bit 0 sets
// the doubling loop's condition, bit 1 the next round's own condition (the
// loop body's second round), bit 2 counts the round.
__global__ void k_round_end(uint32_t* ctrl, int par, uint32_t max_n, cudaGraphConditionalHandle loop,
                            cudaGraphConditionalHandle next_round, int flags) {
    const uint32_t* cur = ctrl + CTRL_BINS + NCLS * par;
    const uint32_t* nxt = ctrl + CTRL_BINS + NCLS * (par ^ 1);
    if (any_groups(cur)) {
        ctrl[CTRL_DEPTH] *= 2u;
        ctrl[CTRL_ROUNDS] += 1u;
    }
    if (flags & 4) ctrl[CTRL_BODY_ITERS] += 1u;
    if (flags & 3) {
        const bool more = any_groups(nxt) && ctrl[CTRL_DEPTH] < max_n && ctrl[CTRL_ROUNDS] < 40u &&
                          ctrl[CTRL_ERR] == 0u;
        if (flags & 1) cudaGraphSetConditional(loop, more ? 1u : 0u);
        if (flags & 2) cudaGraphSetConditional(next_round, more ? 1u : 0u);
    }
}

__global__ void k_set_cond_initial(const uint32_t* ctrl, uint32_t max_n, cudaGraphConditionalHandle cond) {
    const bool more = any_groups(ctrl + CTRL_BINS) && ctrl[CTRL_DEPTH] < max_n && ctrl[CTRL_ERR] == 0u;
    cudaGraphSetConditional(cond, more ? 1u : 0u);
}

// Word copy into mapped pinned host memory by the SMs: a copy engine busy
// with a large transfer on another stream would hold a memcpy node back, and
// the graph with it.
__global__ void k_words_to_host(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

cudaError_t launch_words_to_host(uint32_t* host_dst_dev_ptr, const uint32_t* src, uint32_t words, cudaStream_t st) {
    if (!words) return cudaSuccess;
    k_words_to_host<<<std::min<uint32_t>((words + 255) / 256, 64), 256, 0, st>>>(host_dst_dev_ptr, src, words);
    return cudaGetLastError();
}

cudaError_t launch_reset_ctrl(uint32_t* ctrl, uint32_t spin, uint32_t withhold, uint32_t ntiles0, cudaStream_t st) {
    k_reset_ctrl<<<1, 128, 0, st>>>(ctrl, spin, withhold, ntiles0);
    return cudaGetLastError();
}

cudaError_t launch_round_end(uint32_t* ctrl, int par, uint32_t max_n, cudaGraphConditionalHandle loop,
                             cudaGraphConditionalHandle next_round, int flags, cudaStream_t st) {
    k_round_end<<<1, 1, 0, st>>>(ctrl, par, max_n, loop, next_round, flags);
    return cudaGetLastError();
}

cudaError_t launch_set_cond_initial(const uint32_t* ctrl, uint32_t max_n, cudaGraphConditionalHandle cond,
                                    cudaStream_t st) {
    k_set_cond_initial<<<1, 1, 0, st>>>(ctrl, max_n, cond);
    return cudaGetLastError();
}

}  // namespace bwt
