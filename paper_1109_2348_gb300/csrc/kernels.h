// Host-side launchers of the BWT kernels (implemented in radix.cu,
// doubling.cu). All take device pointers and a stream and return the CUDA
// launch error.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bwt_internal.cuh"

namespace bwt {

// ---- segmented onesweep LSD radix pass -----------------------------------

struct OneSweepParams {
    const void* kin;              // keys in (u64 or u32); unused when reading S
    const uint32_t* vin;          // values in
    void* kout;                   // keys out
    uint32_t* vout;               // values out
    const uint8_t* S;             // blocks (first pass of the first sort only)
    const BlockInfo* blocks;
    const TileDesc* tiles;
    const uint32_t* num_tiles;    // device count of tiles
    const uint32_t* seg_base;     // per segment, per digit: exclusive digit offset in the segment
    uint32_t seg_base_stride;     // words between consecutive segments' rows
    uint32_t* status;             // [tile][radix] look-back words, zeroed before the pass
    uint32_t* tile_counter;       // zeroed before the pass
    uint32_t* ctrl;               // device control words (spin limit, error)
    int shift;                    // digit = (key >> shift) & (radix - 1)
    // u32 passes of the doubling rounds: per segment, nonzero if its keys are
    // not all equal; the tiles of the other segments are skipped (null: none)
    const uint32_t* seg_varied = nullptr;
};

// key_bytes: 8 (u64 rotation prefixes), 4 (u32 doubling ranks) or -8 (u64
// keys whose digit is taken from the u32 value; radix_bits 8 only).
// from_s: build the u64 keys from the block bytes instead of reading kin.
cudaError_t launch_onesweep(int key_bytes, bool from_s, int radix_bits, int tile, const OneSweepParams& p,
                            int grid, cudaStream_t st);
int onesweep_grid(int key_bytes, bool from_s, int radix_bits, int tile);
size_t onesweep_smem(int key_bytes, bool from_s, int radix_bits, int tile);

// ---- 16-bit digits of the first sort (radix16.cu) ------------------------

// Keys per part of a 16-bit pass: parts never straddle blocks, and a part's
// per-digit counts fit 16 bits.
constexpr uint32_t PART16_KEYS = 61440;

// One stable 16-bit LSD pass (digit = (key >> shift) & 0xffff) over every
// block, as four launches: part histograms, prefix over each block's parts,
// prefix over the digits, scatter. kin == nullptr: the first pass, keys packed
// from S (values = rotation indices). parts: the part table (TileDesc with
// seg = blk); part_first[b] .. part_first[b + 1]: block b's parts. partcnt:
// [nparts][65536] u32, segtot: [nseg][65536] u32 (scratch). A destination
// outside its block (counts that disagree with the keys) is not written and
// sets ERR_CAPACITY in ctrl.
cudaError_t launch_first16_pass(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                                const uint8_t* S, const BlockInfo* blocks, const TileDesc* parts, uint32_t nparts,
                                const uint32_t* part_first, uint32_t nseg, int shift, uint32_t* partcnt,
                                uint32_t* segtot, uint32_t* ctrl, cudaStream_t st);
size_t scatter16_smem();

// ---- histograms of the first sort ---------------------------------------

// Byte histogram of every block (d = 8: every pass of the first sort has the
// block's byte histogram as its digit histogram, because the pass-p digit of
// rotation i is S[(i + 7 - p) mod n]). hist: [block][256], zeroed. With
// num_tiles_dev the tile count is read on the device (num_tiles ignored).
cudaError_t launch_hist_bytes(const uint8_t* S, const BlockInfo* blocks, const TileDesc* tiles,
                              uint32_t num_tiles, uint32_t* hist, cudaStream_t st,
                              const uint32_t* num_tiles_dev = nullptr);

// Per-pass digit histograms of the u64 rotation prefixes for radix_bits = 11:
// hist: [block][passes][2048], zeroed.
cudaError_t launch_hist_keys11(const uint8_t* S, const BlockInfo* blocks, const TileDesc* tiles,
                               uint32_t num_tiles, int tile, uint32_t* hist, cudaStream_t st,
                               const uint32_t* num_tiles_dev = nullptr);

// Exclusive scan of every row of `radix` counts, in place; rows = *num_rows_dev
// * rows_mult (or rows_host if num_rows_dev is null), at most max_rows.
cudaError_t launch_scan_rows(uint32_t* hist, int radix, const uint32_t* num_rows_dev, uint32_t rows_mult,
                             uint32_t rows_host, uint32_t max_rows, cudaStream_t st);

// Zero count * words_per_unit words (count read on the device).
cudaError_t launch_zero_by_count(uint32_t* p, const uint32_t* count, uint32_t words_per_unit, uint32_t max_words,
                                 cudaStream_t st);

// ---- naming, doubling rounds, L gather (doubling.cu) --------------------

// First naming after the u64 sort: rank of every rotation = start of its
// group of equal 8-byte prefixes; groups of size > 1 go to `bins` unless
// 8 >= n (then they are identical rotations and final).
cudaError_t launch_name_initial(const uint64_t* K, const uint32_t* SA, const BlockInfo* blocks,
                                const TileDesc* tiles, uint32_t num_tiles, uint32_t* rank, Bins bins,
                                uint32_t* ctrl, cudaStream_t st);

// The same with the tile count on the device. seg_bounds: every tile's
// segment [segStart, segStart + pad0) is a whole range of groups (tiles from
// launch_build_large_tiles), so the carries stay inside it and keys outside
// the segments are never read; else the carries search the tile's block.
cudaError_t launch_name_tiles(const uint64_t* K, const uint32_t* SA, const BlockInfo* blocks, const TileDesc* tiles,
                              const uint32_t* num_tiles_dev, bool seg_bounds, uint32_t* rank, Bins bins,
                              uint32_t* ctrl, cudaStream_t st);

// Round with prefix length h = *depth: key2[k] = rank[(SA[k] + h) mod n] for
// every element of the micro, tiny, small and medium groups in `cur`.
// Ranks are read through `lz` (stored, or found on demand after a learned
// first stage).
cudaError_t launch_gather_small(const uint32_t* SA, const uint32_t* rank, const BlockInfo* blocks, Bins cur,
                                const uint32_t* depth, uint32_t* key2, const uint32_t* host_counts, cudaStream_t st,
                                int* launched, const LazyRanks& lz);

// Builds the radix tile table of the large groups of `cur`, its count and
// the number of keys in large groups; zeroes seg_varied[group] when given.
cudaError_t launch_build_large_tiles(Bins cur, int tile, TileDesc* tiles, uint32_t max_tiles, uint32_t* ctrl,
                                     cudaStream_t st, uint32_t* seg_varied = nullptr);

// Large groups: gathers key2 into kbuf at the positions of SA and builds
// per-group digit histograms hist[group][passes][radix]. With vbuf it also
// copies SA there (needed only when one pass both reads and writes the
// values; with several passes the first reads SA itself). seg_varied[group]
// becomes nonzero if the group's key2 are not all equal.
cudaError_t launch_large_prologue(const uint32_t* SA, const uint32_t* rank, const BlockInfo* blocks,
                                  const TileDesc* tiles, const uint32_t* num_tiles, const uint32_t* depth,
                                  uint32_t* kbuf, uint32_t* vbuf, uint32_t* hist, int radix_bits, int passes,
                                  uint32_t* seg_varied, cudaStream_t st, const LazyRanks& lz);

// Micro, tiny, small and medium groups: sort by (key2, SA), rename, emit
// refined groups.
cudaError_t launch_sort_small(uint32_t* SA, uint32_t* key2, uint32_t* rank, const BlockInfo* blocks, Bins cur,
                              Bins next, const uint32_t* depth, const uint32_t* host_counts, uint32_t* ctrl,
                              cudaStream_t st, int* launched);

// Large groups after their radix sort: rename and emit refined groups; a
// group with seg_varied[group] == 0 (all key2 equal, skipped by the radix)
// is passed on unchanged.
cudaError_t launch_rename_large(const uint32_t* SA, const uint32_t* key2, uint32_t* rank, const BlockInfo* blocks,
                                const TileDesc* tiles, const uint32_t* num_tiles, Bins next, const uint32_t* depth,
                                const uint32_t* seg_varied, uint32_t* ctrl, cudaStream_t st);

// Control words: reset before a batch; advance after a round (and set the
// graph loop condition); set the condition before the loop.
cudaError_t launch_reset_ctrl(uint32_t* ctrl, uint32_t spin, uint32_t withhold, uint32_t ntiles0, cudaStream_t st);

// Copies `words` u32 from device memory to pinned host memory, written by a
// kernel (host_dst_dev_ptr: the device view of the host buffer), so that no
// copy engine is involved: stream-ordered, visible to the host once the
// stream has passed the launch.
cudaError_t launch_words_to_host(uint32_t* host_dst_dev_ptr, const uint32_t* src, uint32_t words, cudaStream_t st);
// flags: 1 = set the loop condition `loop`, 2 = set `next_round`, 4 = count
// the round (graph mode); both conditions get "another round is due".
cudaError_t launch_round_end(uint32_t* ctrl, int par, uint32_t max_n, cudaGraphConditionalHandle loop,
                             cudaGraphConditionalHandle next_round, int flags, cudaStream_t st);

cudaError_t launch_set_cond_initial(const uint32_t* ctrl, uint32_t max_n, cudaGraphConditionalHandle cond,
                                    cudaStream_t st);

// L[k] = S[(SA[k] + n - 1) mod n]; primary[b] = the k with SA[k] = 0.
// ctrl: its tile-counter word for the gather is zeroed and used.
cudaError_t launch_gather_L(const uint8_t* S, const uint32_t* SA, const BlockInfo* blocks, const TileDesc* tiles,
                            uint32_t num_tiles, uint8_t* L, int32_t* primary, uint32_t* ctrl, cudaStream_t st);

int num_sms();

}  // namespace bwt
