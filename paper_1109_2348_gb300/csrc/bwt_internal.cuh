// Internal types and device helpers of the GB300 BWT block sort.
//
// Positions are global indices into the concatenated batch (u32: a batch is
// under 2^32 bytes). Within block b, rotation i lives at global index
// blocks[b].off + i; `rank` is indexed that way. SA holds block-local
// rotation indices at global sorted positions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bwt {

// One radix tile: `len` consecutive keys at global position `start`, inside
// segment `seg` (a block for the first sort, a group for a doubling round).
// Tiles never straddle segments; a segment's tiles are consecutive and
// `firstTile` is the index of its first one (where look-back stops).
struct TileDesc {
    uint32_t start, len, seg, firstTile;
    uint32_t segStart, blk, pad0, pad1;
};

// A group of rotations whose sort keys are still equal: global positions
// [start, start + len) of block blk.
struct GroupDesc {
    uint32_t start, len, blk, pad;
};

struct BlockInfo {
    uint32_t off, n;
};

// Look-back status word: 2 flag bits + 30-bit count.
constexpr uint32_t ST_AGG = 1u << 30;
constexpr uint32_t ST_INC = 2u << 30;
constexpr uint32_t ST_VALUE = (1u << 30) - 1;

// Device error bits (ctrl[CTRL_ERR]).
constexpr uint32_t ERR_TIMEOUT = 1u;
constexpr uint32_t ERR_CAPACITY = 2u;
constexpr uint32_t ERR_INPUT = 4u;  // device-checked input out of range (the inverse's primary index)
constexpr uint32_t ERR_BOUNDS = 8u; // a bounds check of the debug build failed (an internal error)

// SA entries marked SA_FINAL (bit 31; blocks hold fewer than 2^31 bytes) are
// rows that the learned chunk sort left as groups of one: their place is
// final and their rank (the row itself) is not stored, but found on demand
// (LazyRanks below). Readers of SA mask the bit.
constexpr uint32_t SA_FINAL = 0x80000000u;

// Bounds checks of the debug build (-DBWT_DEBUG): index < n for every
// SA-derived index, destinations inside their segment. A failed check sets
// ERR_BOUNDS in the error word *err (the call then returns BWT_EINTERNAL) and
// the kernel goes on with the clamped index the release build uses; no
// kernel traps. In the release build the checks compile to nothing.
#ifdef BWT_DEBUG
#define BWT_DCHECK(cond, err)                                  \
    do {                                                       \
        if (!(cond)) atomicOr((err), ::bwt::ERR_BOUNDS);       \
    } while (0)
#else
#define BWT_DCHECK(cond, err) \
    do {                      \
    } while (0)
#endif

// Group size classes of a doubling round.
constexpr int NCLS = 5;
constexpr uint32_t MICRO_MAX = 4;     // one thread per group, sorting network in registers
constexpr uint32_t TINY_MAX = 32;     // one warp per group, bitonic across the lanes
constexpr uint32_t SMALL_MAX = 256;   // one warp per group, bitonic in shared memory
constexpr uint32_t MED_MAX = 2048;    // one CTA per group, bitonic in shared memory
// groups above MED_MAX (class 4, "large") are sorted by the segmented onesweep radix.
constexpr int CLS_LARGE = 4;

// Layout of the plan's device control words.
enum : int {
    CTRL_BINS = 0,          // [2][NCLS]: group counts per size class, double-buffered
    CTRL_NUM_LTILES = 10,   // tiles of the large-group radix in this round
    CTRL_ERR = 11,
    CTRL_ROUNDS = 12,       // doubling rounds executed
    CTRL_LARGE_KEYS = 13,   // keys in large groups this round
    CTRL_ACTIVE = 14,       // u64 (words 14, 15): rotations re-sorted, summed over rounds
    CTRL_SPIN = 16,         // spin limit for bounded waits
    CTRL_WITHHOLD = 17,     // debug: first tile withholds its look-back publish
    CTRL_DEPTH = 18,        // prefix length h the current round doubles
    CTRL_NTILES0 = 19,      // tiles of the first sort
    CTRL_BODY_ITERS = 20,   // graph mode: doubling rounds whose launches ran (a round skipped by its condition is not counted)
    CTRL_AUX0 = 21,         // learned: tiles of plain-routed blocks
    CTRL_AUX1 = 22,         // learned: tiles of bucketed blocks
    CTRL_TILE_CTR = 32,     // [64] atomic tile counters, one per radix pass
    CTRL_WORDS = 128
};

struct Bins {
    GroupDesc* list[NCLS];
    uint32_t cap[NCLS];
    uint32_t* count;                // -> ctrl + CTRL_BINS + NCLS * parity
    unsigned long long* active;     // -> ctrl + CTRL_ACTIVE
};

// ---- ranks after the learned first stage --------------------------------------
//
// Learned bucketing (Section 3.1's sort by a learned CDF) names each chunk of
// whole key-range buckets in one CTA. Where a block's rotations are nearly
// all distinct in their first 8 bytes, its rank array would be written in
// full (one scattered store a rotation) for the few reads the doubling rounds
// make, rank[(i + h) mod n] for the members i of groups. Such a block is
// "lazy": the chunk sort stores ranks only for group members and marks its
// groups of one SA_FINAL, and a rank read finds a rotation's row on demand:
// its bucket (from its 8-byte key), then a lower bound for the key inside the
// bucket's rows (already sorted). A row marked SA_FINAL is the rotation's
// rank; otherwise the rotation is a group member with its rank stored.
constexpr int LR_BUCKETS = 4096;  // learned buckets (the library's BWT_BUCKETS)
constexpr int IDX_BITS = 16;      // splitter index on a key's first two bytes
constexpr int IDX_CELLS = 1 << IDX_BITS;
constexpr int IDX_WORDS = IDX_CELLS + 8;  // u16 entries (first[IDX_CELLS] = #splitters), padded to 16 bytes

// Bucket of a key: #{j : spl[j] <= key}. first[c] = #{j : spl[j] < c << 48}
// narrows the search to the splitters that share the key's first two bytes
// (the ones below all count, the ones above none).
__device__ __forceinline__ uint32_t bucket_of(const uint64_t* spl, const uint16_t* first, uint64_t key) {
    const uint32_t c = (uint32_t)(key >> (64 - IDX_BITS));
    uint32_t lo = first[c], hi = first[c + 1];
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (spl[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

struct LazyRanks {
    const uint32_t* lazy = nullptr;      // [block] 1: ranks of groups of one are not stored (null: none)
    const uint8_t* S = nullptr;          // the batch's bytes
    const uint32_t* SA = nullptr;        // rows (SA_FINAL-marked)
    const uint32_t* route = nullptr;     // [block] 0 learned buckets, 2 equal-width buckets
    const uint32_t* starts = nullptr;    // [block][LR_BUCKETS] block-relative first row of every bucket
    const uint64_t* splitters = nullptr; // learned splitters
    const uint16_t* index = nullptr;     // their two-byte-prefix index
    uint32_t own_cap = 0;                // largest bucket the chunk sorts name (larger: named in full)
};

// The 8-byte big-endian key of rotation j of a block (cyclic).
__device__ __forceinline__ uint64_t rotation_key(const uint8_t* __restrict__ S, BlockInfo bi, uint32_t j) {
    uint64_t k = 0;
    if ((uint64_t)j + 8 <= bi.n) {  // no wrap: eight independent loads
#pragma unroll
        for (int t = 0; t < 8; ++t) k = (k << 8) | S[bi.off + j + t];
        return k;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        uint32_t q = j + t;
        while (q >= bi.n) q -= bi.n;
        k = (k << 8) | S[bi.off + q];
    }
    return k;
}

static __device__ __noinline__ uint32_t lazy_rank_lookup(const LazyRanks lz, const uint32_t* __restrict__ rank, BlockInfo bi,
                                                  uint32_t blk, uint32_t j) {
    const uint64_t key = rotation_key(lz.S, bi, j);
    const uint32_t b = lz.route[blk] == 2u ? (uint32_t)(key >> 52) : bucket_of(lz.splitters, lz.index, key);
    const uint32_t* st = lz.starts + (size_t)blk * LR_BUCKETS;
    uint32_t lo = st[min(b, (uint32_t)LR_BUCKETS - 1u)];
    uint32_t hi = b + 1 < (uint32_t)LR_BUCKETS ? st[b + 1] : bi.n;
    if (hi > bi.n || lo > hi || hi - lo > lz.own_cap) return rank[bi.off + j];  // named in full
    while (lo < hi) {  // first row of the bucket whose key is not below this one
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t r = lz.SA[bi.off + mid] & ~SA_FINAL;
        if (rotation_key(lz.S, bi, r < bi.n ? r : 0u) < key) lo = mid + 1; else hi = mid;
    }
    const uint32_t x = lo < bi.n ? lz.SA[bi.off + lo] : 0u;
    return (x & SA_FINAL) ? lo : rank[bi.off + j];
}

// rank[j] of block `blk`, stored or found.
__device__ __forceinline__ uint32_t rank_at(const LazyRanks& lz, const uint32_t* __restrict__ rank, BlockInfo bi,
                                            uint32_t blk, uint32_t j) {
    if (lz.lazy == nullptr || lz.lazy[blk] == 0u) return rank[bi.off + j];
    return lazy_rank_lookup(lz, rank, bi, blk, j);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of the warp whose label equals this lane's, for labels below
// 2^BITS: one ballot per label bit, each lane keeping the lanes that agree
// with it on that bit. All 32 lanes call. (The same set as match.any, at a
// few cheap instructions per bit.)
template <int BITS>
__device__ __forceinline__ uint32_t match_label(uint32_t label) {
    uint32_t m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const uint32_t bit = (label >> b) & 1u;
        m &= __ballot_sync(0xffffffffu, bit) ^ (bit - 1u);
    }
    return m;
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) {
    *reinterpret_cast<volatile uint32_t*>(p) = v;
}

// The 8 bytes sb[idx .. idx + 7] as a big-endian u64 (the rotation's sort
// key). sb must be 4-byte aligned and readable up to idx + 11: three aligned
// 32-bit words are funnel-shifted to the byte offset and byte-swapped.
__device__ __forceinline__ uint64_t pack8_smem(const uint8_t* sb, uint32_t idx) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(sb) + (idx >> 2);
    const uint32_t sh = (idx & 3u) * 8u;
    const uint32_t w0 = w[0], w1 = w[1], w2 = w[2];
    const uint32_t lo = __funnelshift_r(w0, w1, sh);  // bytes idx .. idx+3, first byte lowest
    const uint32_t hi = __funnelshift_r(w1, w2, sh);  // bytes idx+4 .. idx+7
    return ((uint64_t)__byte_perm(lo, 0, 0x0123) << 32) | __byte_perm(hi, 0, 0x0123);
}

// Stages the bytes of rotations [i0, i0 + len) of block bi and the 7 bytes
// that follow them (cyclically) in shared memory: byte q of that range lands
// at sb[shift + q], and the return value is shift (0..15). A range that ends
// at least 16 bytes before the block's end and starts no more than 15 bytes
// after S is read with 16-byte loads from the aligned addresses covering it
// (every load stays inside [S, end of the block)); other ranges are read byte
// by byte with shift 0. sb must be 16-byte aligned and hold len + 48 bytes.
// All `nthreads` threads call; the caller synchronises before reading sb.
__device__ __forceinline__ uint32_t stage_tile_bytes(const uint8_t* __restrict__ S, BlockInfo bi, uint32_t i0,
                                                     uint32_t len, uint8_t* sb, uint32_t tid, uint32_t nthreads) {
    const uint32_t need = len + 7;
    const uintptr_t a = reinterpret_cast<uintptr_t>(S + bi.off + i0);
    const uintptr_t a0 = a & ~(uintptr_t)15;
    if ((uint64_t)i0 + need + 16 <= bi.n && a0 >= reinterpret_cast<uintptr_t>(S)) {
        const uint32_t shift = (uint32_t)(a - a0);
        const uint32_t nvec = (shift + need + 15) >> 4;
        const uint4* src = reinterpret_cast<const uint4*>(a0);
        uint4* dst = reinterpret_cast<uint4*>(sb);
        for (uint32_t v = tid; v < nvec; v += nthreads) dst[v] = __ldg(src + v);
        return shift;
    }
    for (uint32_t q = tid; q < need; q += nthreads) {
        uint32_t pos = i0 + q;
        if (pos >= bi.n) pos = bi.n >= 8 ? pos - bi.n : pos % bi.n;
        sb[q] = S[bi.off + pos];
    }
    return 0;
}

// ---- single-pass scan of one 64-bit count per tile -------------------------
//
// Decoupled look-back: tile t publishes its own total (AGG) at once and its
// inclusive prefix (INC) when known; a later tile adds up predecessors'
// words until it meets an INC. Tiles must be started in scan order (a tile
// counter), so every predecessor is in flight or done. The scan restarts at
// segment starts: `first` is the first tile of t's segment. A status word is
// the value in bits 0..61 and the flag in bits 62..63; words start at zero.
constexpr uint64_t LB_AGG = 1ull << 62;
constexpr uint64_t LB_INC = 2ull << 62;
constexpr uint64_t LB_VAL = LB_AGG - 1;

__device__ __forceinline__ uint64_t ld_volatile64(const uint64_t* p) {
    return *reinterpret_cast<const volatile uint64_t*>(p);
}

__device__ __forceinline__ void st_volatile64(uint64_t* p, uint64_t v) {
    *reinterpret_cast<volatile uint64_t*>(p) = v;
}

// All 32 lanes of one warp call; returns the exclusive prefix of tile t in
// every lane. A wait that runs past spin_limit polls sets ERR_TIMEOUT in *err
// and counts the word as an inclusive zero (the result is then wrong but in
// range: callers bound every index they derive from it). withhold (a test
// knob): the first tile of the segment does not publish, so the next tile's
// wait runs out.
__device__ __forceinline__ uint64_t lookback_u64(uint64_t* status, uint32_t t, uint32_t first, uint64_t agg,
                                                 uint32_t spin_limit, uint32_t* err, uint32_t withhold = 0) {
    const uint32_t lane = threadIdx.x & 31;
    if (t == first) {
        if (lane == 0 && !withhold) st_volatile64(status + t, LB_INC | agg);
        return 0;
    }
    if (lane == 0) st_volatile64(status + t, LB_AGG | agg);
    uint64_t excl = 0;
    uint32_t end = t;  // predecessors end - 1, end - 2, ... still to add
    for (;;) {
        const int64_t q = (int64_t)end - 1 - lane;
        uint64_t v = LB_INC;  // before the segment: an inclusive zero
        if (q >= (int64_t)first) {
            v = ld_volatile64(status + q);
            uint32_t it = 0;
            while ((v & (LB_AGG | LB_INC)) == 0ull) {
                if (++it > spin_limit) {
                    atomicOr(err, ERR_TIMEOUT);
                    v = LB_INC;
                    break;
                }
                if (it > 32) __nanosleep(64);
                v = ld_volatile64(status + q);
            }
        }
        const uint32_t inc = __ballot_sync(0xffffffffu, (v & LB_INC) != 0ull);
        const int stop = inc ? __ffs(inc) - 1 : 31;  // nearest inclusive word, or the whole window
        uint64_t x = lane <= (uint32_t)stop ? (v & LB_VAL) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        excl += x;
        if (inc) break;
        end -= 32;
    }
    if (lane == 0) st_volatile64(status + t, LB_INC | ((excl + agg) & LB_VAL));
    return excl;
}

// Number of valid entries of bin c (a count past the capacity means entries
// were dropped and ERR_CAPACITY is set).
__device__ __forceinline__ uint32_t bin_count(const Bins& b, int c) {
    const uint32_t v = b.count[c];
    return v < b.cap[c] ? v : b.cap[c];
}

// Size class of a group.
__device__ __forceinline__ int size_class(uint32_t len) {
    return len <= MICRO_MAX ? 0 : len <= TINY_MAX ? 1 : len <= SMALL_MAX ? 2 : len <= MED_MAX ? 3 : 4;
}

// Append a group to the bin of its size class with one atomic per warp and
// class, and add its length to the active-rotation counter. All 32 lanes
// must call it; lanes with want = false add nothing.
__device__ __forceinline__ void emit_group(const Bins& bins, bool want, uint32_t start, uint32_t len,
                                           uint32_t blk, uint32_t* err) {
    const int lane = threadIdx.x & 31;
    const int cls = want ? size_class(len) : -1;
    const uint32_t any = __ballot_sync(0xffffffffu, want);
    if (any == 0) return;
    const uint32_t lsum = __reduce_add_sync(0xffffffffu, want ? len : 0u);
    if (lane == __ffs(any) - 1) atomicAdd(bins.active, (unsigned long long)lsum);
#pragma unroll
    for (int c = 0; c < NCLS; ++c) {
        uint32_t m = __ballot_sync(0xffffffffu, cls == c);
        if (m == 0) continue;
        int leader = __ffs(m) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&bins.count[c], (uint32_t)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (cls == c) {
            uint32_t slot = base + __popc(m & lanemask_lt());
            if (slot < bins.cap[c]) {
                bins.list[c][slot] = GroupDesc{start, len, blk, 0u};
            } else {
                atomicOr(err, ERR_CAPACITY);
            }
        }
    }
}

// Warp-buffered emission: each warp stages the groups it emits in shared
// memory, EMIT_BUF per size class, and reserves bin slots with one atomic per
// flush instead of one per emitting warp step; the active-rotation count is
// summed per lane and added once at the end. Every lane of the warp must make
// the same calls (warp-uniform control flow).
constexpr int EMIT_BUF = 16;

struct WarpEmitter {
    GroupDesc* buf;              // shared memory, [NCLS][EMIT_BUF]
    uint32_t n[NCLS];            // staged entries per class (warp-uniform)
    unsigned long long active;   // this lane's emitted rotations

    __device__ __forceinline__ void init(GroupDesc* warp_buf) {
        buf = warp_buf;
#pragma unroll
        for (int c = 0; c < NCLS; ++c) n[c] = 0;
        active = 0;
    }

    __device__ __forceinline__ void flush(const Bins& bins, int c, uint32_t* err) {
        const int lane = threadIdx.x & 31;
        __syncwarp();
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&bins.count[c], n[c]);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((uint32_t)lane < n[c]) {
            const uint32_t slot = base + lane;
            if (slot < bins.cap[c]) bins.list[c][slot] = buf[c * EMIT_BUF + lane];
            else atomicOr(err, ERR_CAPACITY);
        }
        n[c] = 0;
        __syncwarp();
    }

    __device__ __forceinline__ void emit(const Bins& bins, bool want, uint32_t start, uint32_t len, uint32_t blk,
                                         uint32_t* err) {
        if (__ballot_sync(0xffffffffu, want) == 0u) return;  // the common case: nothing to emit
        const int cls = want ? size_class(len) : -1;
        if (want) active += len;
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int c = 0; c < NCLS; ++c) {
            const uint32_t m = __ballot_sync(0xffffffffu, cls == c);
            if (m == 0) continue;
            const uint32_t cnt = __popc(m);
            if (n[c] + cnt > EMIT_BUF) flush(bins, c, err);
            if (cnt > EMIT_BUF) {  // more than the buffer holds: reserve and write directly
                const int leader = __ffs(m) - 1;
                uint32_t base = 0;
                if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(&bins.count[c], cnt);
                base = __shfl_sync(0xffffffffu, base, leader);
                if (cls == c) {
                    const uint32_t slot = base + __popc(m & lt);
                    if (slot < bins.cap[c]) bins.list[c][slot] = GroupDesc{start, len, blk, 0u};
                    else atomicOr(err, ERR_CAPACITY);
                }
                continue;
            }
            if (cls == c) buf[c * EMIT_BUF + n[c] + __popc(m & lt)] = GroupDesc{start, len, blk, 0u};
            n[c] += cnt;
        }
    }

    __device__ __forceinline__ void finish(const Bins& bins, uint32_t* err) {
#pragma unroll
        for (int c = 0; c < NCLS; ++c)
            if (n[c]) flush(bins, c, err);
        const unsigned long long tot = __reduce_add_sync(0xffffffffu, (uint32_t)active) +
                                       ((unsigned long long)__reduce_add_sync(0xffffffffu, (uint32_t)(active >> 32)) << 32);
        if ((threadIdx.x & 31) == 0 && tot) atomicAdd(bins.active, tot);
    }
};

// Block-wide exclusive scan of one value per thread; returns the prefix and
// writes the total to *total. `tmp` holds at least THREADS/32 words.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* tmp, uint32_t* total) {
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < WARPS ? tmp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < WARPS) tmp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    uint32_t warp_prefix = warp > 0 ? tmp[warp - 1] : 0u;
    *total = tmp[WARPS - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

template <typename T>
__device__ __forceinline__ uint32_t smem_lower_bound(const T* a, uint32_t n, T x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ uint32_t smem_upper_bound(const T* a, uint32_t n, T x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Names every element of one sorted tile: the tile's keys sit in sk[0..len)
// and its SA entries in sa_tile[0..len) (both in shared memory); its first
// run may have begun before the tile (it begins at carry_start) and its last
// run may continue after it (it ends at carry_end). Writes rank[rotation] =
// block-local start of the element's group and emits the groups of size > 1
// that start inside the tile. old_start: the global start of the group the
// tile was sorted from, whose members already hold it as their rank (their
// rank is written only where it changes), or NO_OLD_START for a first naming.
//
// Each of the NW warps walks its own range (an NW-th of the tile, rounded up
// to whole steps), 32 elements a step: the heads (an
// element whose key differs from its predecessor's, and element 0) come
// from one ballot, an element's group starts at the last head at or before
// it (carried across steps and, through shared memory, across warps), and
// the lane at a head emits the group that ends there; the group of the
// tile's last head is emitted after the walk. All NW warps of the CTA call
// (one barrier inside).
constexpr uint32_t NO_OLD_START = 0xffffffffu;

template <typename KeyT, int NW = 8>
__device__ __forceinline__ void name_tile(const KeyT* sk, uint32_t len, uint32_t tstart, uint32_t carry_start,
                                          uint32_t carry_end, const uint32_t* sa_tile, BlockInfo bi, uint32_t blk,
                                          uint32_t* __restrict__ rank, const Bins& bins, bool emit_ok,
                                          uint32_t old_start, WarpEmitter& em, uint32_t* err) {
    constexpr uint32_t NONE = 0xffffffffu;
    __shared__ uint32_t s_heads[2 * NW];  // per warp: first head, last head of its range (NONE if none)
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t span = ((len + NW * 32 - 1) / (NW * 32)) * 32;
    const uint32_t r0 = min(len, warp * span), r1 = min(len, r0 + span);
    auto is_head = [&](uint32_t q) { return q < r1 && (q == 0 || sk[q - 1] != sk[q]); };
    // 1. first and last head of the warp's range
    uint32_t fh = NONE, lh = NONE;
    for (uint32_t b = r0; b < r1; b += 32) {
        const uint32_t m = __ballot_sync(0xffffffffu, is_head(b + lane));
        if (m) {
            fh = b + __ffs(m) - 1;
            break;
        }
    }
    if (fh != NONE) {
        for (uint32_t b = r0 + ((r1 - 1 - r0) & ~31u);; b -= 32) {
            const uint32_t m = __ballot_sync(0xffffffffu, is_head(b + lane));
            if (m) {
                lh = b + 31 - __clz(m);
                break;
            }
            if (b <= fh) break;  // unreachable: fh itself is a head
        }
    }
    if (lane == 0) {
        s_heads[warp] = fh;
        s_heads[NW + warp] = lh;
    }
    __syncthreads();
    // 2. the last head before the range and the first head after it
    uint32_t last = NONE, next = NONE;
    for (uint32_t w = 0; w < warp; ++w)
        if (s_heads[NW + w] != NONE) last = s_heads[NW + w];
    for (uint32_t w = NW - 1; w > warp; --w)
        if (s_heads[w] != NONE) next = s_heads[w];
    // 3. rank every element; each head closes the group before it
    for (uint32_t b = r0; b < r1; b += 32) {
        const uint32_t q = b + lane;
        const bool valid = q < r1;
        const bool h = is_head(q);
        const uint32_t m = __ballot_sync(0xffffffffu, h);
        const uint32_t hle = m & (lt | (1u << lane));
        const uint32_t sq = hle ? b + 31 - __clz(hle) : last;  // start of q's group (tile-local)
        if (valid) {
            const uint32_t gs = sq == 0 ? carry_start : tstart + sq;
            const uint32_t sa = sa_tile[q];
            BWT_DCHECK(sa < bi.n && gs - bi.off < bi.n, err);
            if (sa < bi.n && gs != old_start) rank[bi.off + sa] = gs - bi.off;
        }
        bool want = false;
        uint32_t ps = 0;
        if (h && q > 0) {
            const uint32_t hlt = m & lt;
            ps = hlt ? b + 31 - __clz(hlt) : last;  // the closed group is [ps, q)
            want = emit_ok && q - ps > 1 && (ps > 0 || carry_start == tstart);
        }
        em.emit(bins, want, tstart + ps, q - ps, blk, err);
        if (m) last = b + 31 - __clz(m);
    }
    // 4. the tile's last group, if its head is in this range
    if (r0 < r1 && next == NONE && lh != NONE) {
        const uint32_t glen = carry_end - (tstart + lh);
        const bool want = lane == 0 && emit_ok && glen > 1 && (lh > 0 || carry_start == tstart);
        em.emit(bins, want, tstart + lh, glen, blk, err);
    }
}

}  // namespace bwt
