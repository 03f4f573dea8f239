// Plan object and the host-side pieces shared by plan.cu, graph.cu and
// learned.cu.
#pragma once

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "bwt.h"
#include "bwt_internal.cuh"

namespace bwt {

// Host-side NVTX range around the launches of one stage ("pack+radix[0]",
// "radix[p]", "name", "double[r]", "gather", "bucket_*", "mlp_*", ...); a
// profiler shows them on the host timeline (in graph mode they mark the
// capture). Without a profiler attached the calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    NvtxRange(const char* name, int index) {
        char b[64];
        std::snprintf(b, sizeof b, "%s[%d]", name, index);
        nvtxRangePushA(b);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Consecutive NVTX ranges through one function: next() closes the open
// range and opens another; the last one closes with the object.
struct NvtxStages {
    bool open = false;
    void next(const char* name) {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    ~NvtxStages() {
        if (open) nvtxRangePop();
    }
};

struct EvMeta {
    double bytes_per_key;
    bool first_sort;     // a pass of the first sort (also reported on its own)
    uint64_t keys_host;  // keys moved, when the host knows it
    int ctrl_word;       // else: the ctrl word holding it (read after the round), -1 if none
    uint64_t keys_dev = 0;
    bool resolved = false;
    bool chunk_sort = false;  // the learned bucketing's 256-thread chunk sort, not a radix pass
};

// One instantiated CUDA graph of a batch (BWT_F_GRAPH).
struct GraphEntry {
    std::vector<uint64_t> key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t launched = nullptr;  // recorded after its last launch
    uint64_t last_use = 0;
    // kernels of the graph outside the doubling loop, of one round without its
    // large-group section, and of that section; radix passes likewise
    uint64_t main_kernels = 0, round_kernels = 0, large_kernels = 0, main_radix = 0, large_radix = 0;
};

constexpr size_t kGraphCache = 4;

}  // namespace bwt

struct bwt_plan {
    int device = 0;
    bwt_plan_desc desc{};
    std::string model_path;
    int rbits = 8, tile = 4096;
    int round_bits = 0;  // digit width of the doubling rounds' radix (0 = by rank width: 8 or 10)
    uint32_t spin_limit = 0;
    int withhold = 0;

    // capacities
    uint64_t cap_n = 0;
    uint32_t cap_b = 0, cap_tiles0 = 0, cap_ltiles = 0;
    uint32_t bincap[bwt::NCLS] = {0, 0, 0, 0, 0};
    uint64_t cap_hist = 0, cap_status = 0;
    size_t device_bytes = 0;

    // device memory (plan-owned scratch)
    uint64_t* keys[2] = {nullptr, nullptr};
    uint32_t* vals[2] = {nullptr, nullptr};
    uint32_t* rank = nullptr;
    bwt::TileDesc* tiles0 = nullptr;
    bwt::TileDesc* ltiles = nullptr;
    bwt::BlockInfo* blocks = nullptr;
    uint32_t* hist = nullptr;
    uint32_t* status = nullptr;
    uint32_t* ctrl = nullptr;
    uint32_t* seg_varied = nullptr;  // [large groups] nonzero if a large group's key2 are not all equal
    bwt::GroupDesc* bins[2][bwt::NCLS] = {};

    // learned bucketing (allocated when a model is installed)
    uint64_t* splitters = nullptr;      // [BWT_SPLITTERS] sorted
    uint16_t* splitter_index = nullptr; // [65,544] first splitter of every two-byte key prefix
    uint64_t* splitters_flat = nullptr; // [BWT_SPLITTERS] equal-width fallback (top 12 key bits)
    uint32_t* bucket_count = nullptr;   // [2][block][BWT_BUCKETS] counts (learned, equal-width), then starts
    uint32_t* bucket_cursor = nullptr;  // [block][BWT_BUCKETS] slots taken so far (per chunk)
    uint16_t* chunk_map = nullptr;      // [block][BWT_BUCKETS] chunk of each bucket
    uint32_t* chunk_base = nullptr;     // [block][BWT_BUCKETS] block-relative start of each chunk
    uint32_t* route = nullptr;          // [block] 0 = learned buckets, 1 = plain radix, 2 = equal-width buckets
    uint32_t* route_first = nullptr;    // [2][block] first tile of each block in its route's tile table
    uint32_t* members = nullptr;        // [block] rotations the chunk sorts sent to the doubling rounds
    uint32_t* lazy = nullptr;           // [block] 1: ranks of groups of one are found on demand
    bwt::LazyRanks lazy_ranks;          // how this call's doubling rounds read ranks
    unsigned long long* bstats = nullptr;  // [2][block][5] overflow keys, overflow buckets, largest bucket,
                                           // sum of squared sizes, non-empty buckets
    bwt::TileDesc* tiles_aux = nullptr; // [2][tiles0]: tiles of plain-routed blocks, then of bucketed ones
    uint32_t* h_route = nullptr;
    unsigned long long* h_bstats = nullptr;
    uint32_t* hd_route = nullptr;       // device views of the two pinned buffers above (written by kernels)
    uint32_t* hd_bstats = nullptr;
    bool have_model = false;
    int chunk_sort_ctas = 1;            // resident chunk-sort CTAs per SM
    uint32_t learned_overflow_passes = 0;  // radix passes over the overflow buckets (index + key)

    // 16-bit digits of the first sort (allocated when radix_bits 16 is first chosen)
    bwt::TileDesc* parts16 = nullptr;    // [cap_parts] parts of up to PART16_KEYS keys, block by block
    uint32_t* part_first16 = nullptr;    // [cap_b + 1] first part of every block
    uint32_t* partcnt16 = nullptr;       // [cap_parts][65536] per-part digit counts, then prefixes
    uint32_t* segtot16 = nullptr;        // [cap_b][65536] per-block digit totals, then starts
    bwt::TileDesc* stage_parts[2] = {nullptr, nullptr};  // pinned staging of the part table
    uint32_t* stage_pfirst[2] = {nullptr, nullptr};
    uint32_t cap_parts = 0, nparts = 0;

    // GPU inverse (allocated on first use)
    uint32_t* inv_slots = nullptr;     // [6][cap_n / 16 + 3 cap_b + 4] sample walks and pointer jumping
    uint32_t* inv_items = nullptr;     // [2][cap_b + 1] prefixes of work items and of samples per block
    uint32_t* h_inv_items = nullptr;   // pinned staging (also the move-to-front chunk table)
    uint8_t* mtf_lists = nullptr;      // move-to-front scratch (allocated on first use)

    // pinned host staging
    uint32_t* h_ctrl = nullptr;
    uint32_t* hd_ctrl = nullptr;        // its device view (the graph path writes it with a kernel)
    bwt::TileDesc* h_tiles = nullptr;    // the staging slot of the last upload (block and tile tables)
    bwt::BlockInfo* h_blocks = nullptr;
    uint64_t* h_off = nullptr;
    // Two staging slots for the block and tile tables, each with an event
    // recorded after its upload, so a call overwrites a slot only once the
    // copy from it two uploads ago has run (no stream synchronisation).
    bwt::TileDesc* stage_tiles[2] = {nullptr, nullptr};
    bwt::BlockInfo* stage_blocks[2] = {nullptr, nullptr};
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    bool stage_used[2] = {false, false};
    int stage_next = 0;
    std::vector<uint64_t> tables_key;  // layout (tile size, offsets) now in the device tables; empty = unknown

    // end of the last asynchronous forward call: its status and statistics
    // are read from h_ctrl (and the learned counters) once this event has
    // completed
    cudaEvent_t done_ev = nullptr;
    bool pending = false;       // a call's status and statistics are still to be read
    bool pending_learned = false;

    // current batch
    uint32_t nb = 0, total = 0, max_n = 0, ntiles0 = 0;
    uint32_t* sa = nullptr;    // final SA buffer of the current batch
    uint32_t* key2 = nullptr;  // doubling keys, position-indexed
    uint32_t *kA = nullptr, *vA = nullptr, *kB = nullptr, *vB = nullptr;

    // timing
    std::vector<cudaEvent_t> events;
    std::vector<bwt::EvMeta> ev_meta;
    size_t ev_used = 0;
    double radix_bytes = 0;
    uint32_t pending_large_passes = 0;  // u32 passes enqueued whose key count is still on the device

    // CUDA graph cache: the most recently used graphs, one per (buffers,
    // block layout, radix settings); the counts describe the graph the last
    // call launched
    std::vector<bwt::GraphEntry> graphs;
    uint64_t graph_use = 0;
    uint64_t graph_main_kernels = 0, graph_round_kernels = 0, graph_large_kernels = 0;
    uint64_t graph_main_radix = 0, graph_large_radix = 0;
    uint64_t cap_large_kernels = 0, cap_large_radix = 0;  // one round's large-group section, as enqueued
    bool capturing = false;

    bwt_stats stats{};
    bwt_status last = BWT_OK;
};

namespace bwt {

bwt_status record_cuda(cudaError_t e, const char* what);
void free_plan_memory(bwt_plan* p);
void drop_graph(bwt_plan* p);
bwt_status prepare_batch(bwt_plan* p, const uint64_t* offsets, uint32_t nb, cudaStream_t st);
bwt_status upload_tables(bwt_plan* p, const uint64_t* off, uint32_t nb, cudaStream_t st);
Bins bins_of(bwt_plan* p, int par);
int round_radix_bits(const bwt_plan* p);
bwt_status reset_ctrl(bwt_plan* p, cudaStream_t st);
bwt_status enqueue_initial_sort(bwt_plan* p, const uint8_t* d_in, cudaStream_t st);
// One doubling round on bins[par]; records the kernels and radix passes of
// its large-group section (cap_large_kernels, cap_large_radix).
bwt_status enqueue_round(bwt_plan* p, int par, const uint32_t* host_counts, cudaStream_t st);
// Graph capture helper: an IF node on handle h appended to the graph `st`
// is capturing (after st's work so far), whose body `inner` then captures
// until cudaStreamEndCapture(inner).
bwt_status begin_if_capture(cudaStream_t st, cudaStream_t inner, cudaGraphConditionalHandle h);
bwt_status enqueue_naming(bwt_plan* p, const uint64_t* K, cudaStream_t st);
bwt_status finish_status(bwt_plan* p, cudaStream_t st);
// Status of the control words' error field as read into h_ctrl.
bwt_status status_of_ctrl(const bwt_plan* p);
// Waits for the last asynchronous forward call and fills in its status and
// statistics (a no-op when nothing is pending).
void resolve_pending(bwt_plan* p);
void collect_timing(bwt_plan* p);
bwt_status run_plain_host_loop(bwt_plan* p, const uint8_t* d_in, uint8_t* d_L, int32_t* d_primary, cudaStream_t st);
bwt_status run_doubling_host_loop(bwt_plan* p, cudaStream_t st);
bwt_status run_per_block(bwt_plan* p, const uint8_t* d_in, uint8_t* d_L, int32_t* d_primary, cudaStream_t st);
bwt_status run_graph(bwt_plan* p, const uint8_t* d_in, uint8_t* d_L, int32_t* d_primary, cudaStream_t st);
bwt_status run_learned(bwt_plan* p, const uint8_t* d_in, uint8_t* d_L, int32_t* d_primary, cudaStream_t st);
// Learned first stage (bucket count, device-side routing, scatter, chunk sorts
// with naming, overflow radix, plain radix of plain-routed blocks) with no
// host synchronisation, so it can be captured; ctrl must have been reset.
bwt_status enqueue_learned(bwt_plan* p, const uint8_t* d_in, cudaStream_t st);
// After the call has synchronised: routing and bucket statistics from the
// per-block counters the learned stage copied to the host.
void learned_stats(bwt_plan* p);
bwt_status load_model(bwt_plan* p, const char* path);
void graph_stats(bwt_plan* p);
bwt_status ensure_learned_buffers(bwt_plan* p);
// The two-byte-prefix index of the installed splitter table (synchronous).
bwt_status build_splitter_index(bwt_plan* p);
// Scratch of the 16-bit digit passes (a no-op once allocated).
bwt_status ensure_radix16(bwt_plan* p);

}  // namespace bwt
