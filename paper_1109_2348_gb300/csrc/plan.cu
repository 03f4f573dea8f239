// Host side of the C ABI: plan creation, argument checks and the launch
// sequence of one batch.
//
//   per batch:  histograms -> P onesweep passes over the u64 prefixes (the
//               first pass builds the keys from the bytes) -> naming ->
//               doubling rounds (gather, small-group sorts, large-group
//               radix, rename) until no group is left -> L gather.
//
// The host reads three group counts per doubling round to decide whether to
// go on; in BWT_F_GRAPH mode the same launches sit in a CUDA graph whose
// doubling loop is a conditional WHILE node evaluated on the device.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "bwt.h"
#include "kernels.h"
#include "plan_internal.h"

using namespace bwt;

static thread_local std::string g_cuda_err = "no error";
static std::mutex g_err_mu;
static std::string g_cuda_err_global = "no error";

bwt_status bwt::record_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return BWT_OK;
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_cuda_err_global = std::string(what) + ": " + cudaGetErrorString(e);
    return BWT_ECUDA;
}

#define CK(call)                                               \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return record_cuda(_e, #call);  \
    } while (0)

extern "C" const char* bwt_last_cuda_error(void) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    static thread_local std::string copy;
    copy = g_cuda_err_global;
    return copy.c_str();
}

extern "C" const char* bwt_status_string(bwt_status s) {
    switch (s) {
    case BWT_OK: return "BWT_OK";
    case BWT_EINVAL: return "BWT_EINVAL";
    case BWT_ENOMEM: return "BWT_ENOMEM";
    case BWT_ECAPACITY: return "BWT_ECAPACITY";
    case BWT_ECUDA: return "BWT_ECUDA";
    case BWT_ETIMEOUT: return "BWT_ETIMEOUT";
    case BWT_EMISMATCH: return "BWT_EMISMATCH";
    case BWT_ENOMODEL: return "BWT_ENOMODEL";
    case BWT_ETOOBIG: return "BWT_ETOOBIG";
    case BWT_EINTERNAL: return "BWT_EINTERNAL";
    }
    return "BWT_UNKNOWN";
}

namespace {

constexpr uint32_t kDefaultSpin = 1u << 24;  // ~1 s of polling with back-off

template <typename T>
bwt_status dev_alloc(T** p, size_t count, size_t* total) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        record_cuda(e, "cudaMalloc");
        *p = nullptr;
        return BWT_ENOMEM;
    }
    *total += count * sizeof(T);
    return BWT_OK;
}

template <typename T>
bwt_status host_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMallocHost((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        record_cuda(e, "cudaMallocHost");
        *p = nullptr;
        return BWT_ENOMEM;
    }
    return BWT_OK;
}

int bits_for(uint32_t max_value) {  // bits to hold 0..max_value
    int b = 0;
    while (b < 32 && (max_value >> b) != 0) ++b;
    return b;
}

bool valid_radix(int rb) { return rb == 8 || rb == 11 || rb == 16; }
bool valid_round_radix(int rb) { return rb == 8 || rb == 10 || rb == 11; }
bool valid_tile(int t) { return t == 1024 || t == 2048 || t == 4096; }

}  // namespace

// Digit width of the doubling rounds' large-group radix: the plan's choice,
// else whichever of 8 and 10 needs fewer passes over the batch's rank width,
// 8 on a tie. Measured on 64 x 900,000 mixed blocks (20-bit ranks): two
// 10-bit passes took 0.71 ms against 0.84 ms for three 8-bit ones; an 11-bit
// pass costs more than twice an 8-bit one.
int bwt::round_radix_bits(const bwt_plan* p) {
    if (p->round_bits) return p->round_bits;
    const int kbits = std::max(1, bits_for(p->max_n ? p->max_n - 1 : 0));
    return (kbits + 9) / 10 < (kbits + 7) / 8 ? 10 : 8;
}

void bwt::free_plan_memory(bwt_plan* p) {
    auto F = [](void* q) {
        if (q) cudaFree(q);
    };
    auto FH = [](void* q) {
        if (q) cudaFreeHost(q);
    };
    F(p->keys[0]); F(p->keys[1]); F(p->vals[0]); F(p->vals[1]); F(p->rank);
    F(p->tiles0); F(p->ltiles); F(p->blocks); F(p->hist); F(p->status); F(p->ctrl); F(p->seg_varied);
    for (int s = 0; s < 2; ++s)
        for (int c = 0; c < NCLS; ++c) F(p->bins[s][c]);
    F(p->parts16); F(p->part_first16); F(p->partcnt16); F(p->segtot16);
    for (int sl = 0; sl < 2; ++sl) {
        FH(p->stage_parts[sl]);
        FH(p->stage_pfirst[sl]);
    }
    F(p->splitters); F(p->splitter_index); F(p->splitters_flat); F(p->bucket_count); F(p->bucket_cursor); F(p->chunk_map); F(p->chunk_base); F(p->route); F(p->route_first); F(p->members); F(p->lazy); F(p->bstats); F(p->tiles_aux); F(p->inv_slots); F(p->inv_items); F(p->mtf_lists);
    drop_graph(p);
    FH(p->h_ctrl); FH(p->h_off);
    for (int s = 0; s < 2; ++s) {
        FH(p->stage_tiles[s]);
        FH(p->stage_blocks[s]);
        if (p->stage_ev[s]) cudaEventDestroy(p->stage_ev[s]);
    }
    if (p->done_ev) cudaEventDestroy(p->done_ev);
    FH(p->h_route); FH(p->h_bstats); FH(p->h_inv_items);
    for (auto& e : p->events) cudaEventDestroy(e);
    p->events.clear();
}

extern "C" bwt_status bwt_plan_create(const bwt_plan_desc* desc, int device, bwt_plan** out) {
    if (!out) return BWT_EINVAL;
    *out = nullptr;
    if (!desc || desc->max_blocks == 0 || desc->max_total_bytes == 0 || desc->max_total_bytes >= (1ull << 32) ||
        desc->max_block_bytes == 0 || desc->max_block_bytes >= (1u << 30))
        return BWT_EINVAL;
    if (desc->radix_bits != 0 && !valid_radix(desc->radix_bits)) return BWT_EINVAL;
    if (desc->tile_keys != 0 && !valid_tile(desc->tile_keys)) return BWT_EINVAL;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return BWT_EINVAL;
    CK(cudaSetDevice(device));

    bwt_plan* p = new bwt_plan();
    p->device = device;
    p->desc = *desc;
    p->model_path = desc->model_path ? desc->model_path : "";
    p->desc.model_path = nullptr;
    p->rbits = desc->radix_bits ? desc->radix_bits : 8;
    p->tile = desc->tile_keys ? desc->tile_keys : 4096;
    p->spin_limit = kDefaultSpin;
    const uint64_t N = desc->max_total_bytes;
    const uint32_t B = desc->max_blocks;
    p->cap_n = N;
    p->cap_b = B;
    p->cap_tiles0 = (uint32_t)((N + 1023) / 1024 + B);
    p->cap_ltiles = (uint32_t)(N / 1024 + N / (MED_MAX + 1) + 2);
    p->bincap[0] = (uint32_t)(N / 2 + 1);
    p->bincap[1] = (uint32_t)(N / (MICRO_MAX + 1) + 1);
    p->bincap[2] = (uint32_t)(N / (TINY_MAX + 1) + 1);
    p->bincap[3] = (uint32_t)(N / (SMALL_MAX + 1) + 1);
    p->bincap[4] = (uint32_t)(N / (MED_MAX + 1) + 1);
    const uint64_t large_groups = p->bincap[4];
    p->cap_hist = std::max<uint64_t>({(uint64_t)B * 6 * 2048, (uint64_t)B * 256, large_groups * 4 * 256,
                                      large_groups * 3 * 2048});
    p->cap_status = (uint64_t)std::max(p->cap_tiles0, p->cap_ltiles) * 2048;

    bwt_status s = BWT_OK;
    size_t total = 0;
    auto A = [&](bwt_status r) {
        if (s == BWT_OK && r != BWT_OK) s = r;
    };
    A(dev_alloc(&p->keys[0], N, &total));
    A(dev_alloc(&p->keys[1], N, &total));
    A(dev_alloc(&p->vals[0], N, &total));
    A(dev_alloc(&p->vals[1], N, &total));
    A(dev_alloc(&p->rank, N, &total));
    A(dev_alloc(&p->tiles0, p->cap_tiles0, &total));
    A(dev_alloc(&p->ltiles, p->cap_ltiles, &total));
    A(dev_alloc(&p->blocks, B, &total));
    A(dev_alloc(&p->hist, p->cap_hist, &total));
    A(dev_alloc(&p->status, p->cap_status, &total));
    A(dev_alloc(&p->ctrl, CTRL_WORDS, &total));
    A(dev_alloc(&p->seg_varied, (size_t)p->bincap[CLS_LARGE] + 1, &total));
    for (int par = 0; par < 2; ++par)
        for (int c = 0; c < NCLS; ++c) A(dev_alloc(&p->bins[par][c], p->bincap[c], &total));
    A(host_alloc(&p->h_ctrl, CTRL_WORDS));
    if (s == BWT_OK) {
        const cudaError_t e = cudaHostGetDevicePointer((void**)&p->hd_ctrl, p->h_ctrl, 0);
        if (e != cudaSuccess) s = record_cuda(e, "cudaHostGetDevicePointer");
    }
    for (int sl = 0; sl < 2; ++sl) {
        A(host_alloc(&p->stage_tiles[sl], p->cap_tiles0));
        A(host_alloc(&p->stage_blocks[sl], B));
        if (s == BWT_OK && cudaEventCreateWithFlags(&p->stage_ev[sl], cudaEventDisableTiming) != cudaSuccess)
            s = BWT_ECUDA;
    }
    p->h_tiles = p->stage_tiles[0];
    p->h_blocks = p->stage_blocks[0];
    if (s == BWT_OK && cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming) != cudaSuccess) s = BWT_ECUDA;
    A(host_alloc(&p->h_off, (size_t)B + 1));
    A(host_alloc(&p->h_inv_items, 2 * ((size_t)B + 1)));
    // the learned bucketing's tables and the 16-bit passes' scratch, so that
    // no forward call allocates
    if (s == BWT_OK && (desc->flags & BWT_F_LEARNED)) s = ensure_learned_buffers(p);
    if (s == BWT_OK && p->rbits == 16) s = ensure_radix16(p);
    p->device_bytes = total;
    if (s == BWT_OK && (desc->flags & BWT_F_TIMING)) {
        p->events.resize(512);
        for (auto& e : p->events) {
            if (cudaEventCreate(&e) != cudaSuccess) {
                s = BWT_ECUDA;
                break;
            }
        }
    }
    if (s == BWT_OK && (desc->flags & BWT_F_LEARNED) && !p->model_path.empty()) s = load_model(p, p->model_path.c_str());
    if (s != BWT_OK) {
        free_plan_memory(p);
        delete p;
        return s;
    }
    *out = p;
    return BWT_OK;
}

extern "C" bwt_status bwt_plan_destroy(bwt_plan* plan) {
    if (!plan) return BWT_OK;
    cudaSetDevice(plan->device);
    free_plan_memory(plan);
    delete plan;
    return BWT_OK;
}

extern "C" bwt_status bwt_plan_last_status(const bwt_plan* plan) {
    if (!plan) return BWT_EINVAL;
    resolve_pending(const_cast<bwt_plan*>(plan));
    return plan->last;
}

extern "C" bwt_status bwt_plan_stats(const bwt_plan* plan, bwt_stats* out) {
    if (!plan || !out) return BWT_EINVAL;
    resolve_pending(const_cast<bwt_plan*>(plan));
    *out = plan->stats;
    return BWT_OK;
}

bwt_status bwt::ensure_radix16(bwt_plan* p) {
    if (p->partcnt16) return BWT_OK;
    const uint64_t cap_parts = p->cap_n / PART16_KEYS + p->cap_b;
    if (cap_parts >= (1ull << 32)) return BWT_EINVAL;
    size_t total = 0;
    bwt_status s = BWT_OK;
    auto A = [&](bwt_status r) {
        if (s == BWT_OK && r != BWT_OK) s = r;
    };
    A(dev_alloc(&p->parts16, cap_parts, &total));
    A(dev_alloc(&p->part_first16, (size_t)p->cap_b + 1, &total));
    A(dev_alloc(&p->partcnt16, cap_parts * 65536, &total));
    A(dev_alloc(&p->segtot16, (size_t)p->cap_b * 65536, &total));
    for (int sl = 0; sl < 2; ++sl) {
        A(host_alloc(&p->stage_parts[sl], cap_parts));
        A(host_alloc(&p->stage_pfirst[sl], (size_t)p->cap_b + 1));
    }
    if (s != BWT_OK) {
        auto F = [](void* q) {
            if (q) cudaFree(q);
        };
        F(p->parts16); F(p->part_first16); F(p->partcnt16); F(p->segtot16);
        p->parts16 = nullptr;
        p->part_first16 = p->partcnt16 = p->segtot16 = nullptr;
        for (int sl = 0; sl < 2; ++sl) {
            if (p->stage_parts[sl]) cudaFreeHost(p->stage_parts[sl]);
            if (p->stage_pfirst[sl]) cudaFreeHost(p->stage_pfirst[sl]);
            p->stage_parts[sl] = nullptr;
            p->stage_pfirst[sl] = nullptr;
        }
        return s;
    }
    p->cap_parts = (uint32_t)cap_parts;
    p->device_bytes += total;
    return BWT_OK;
}

extern "C" bwt_status bwt_plan_set_radix(bwt_plan* plan, int radix_bits, int tile_keys) {
    if (!plan || !valid_radix(radix_bits) || !valid_tile(tile_keys)) return BWT_EINVAL;
    if (radix_bits == 16) {
        if (cudaSetDevice(plan->device) != cudaSuccess) return BWT_ECUDA;
        const bwt_status s = ensure_radix16(plan);
        if (s != BWT_OK) return s;
    }
    plan->rbits = radix_bits;
    plan->tile = tile_keys;
    drop_graph(plan);
    return BWT_OK;
}

extern "C" bwt_status bwt_plan_set_round_radix(bwt_plan* plan, int radix_bits) {
    if (!plan || (radix_bits != 0 && !valid_round_radix(radix_bits))) return BWT_EINVAL;
    plan->round_bits = radix_bits;
    drop_graph(plan);
    return BWT_OK;
}

extern "C" bwt_status bwt_plan_debug_waits(bwt_plan* plan, uint32_t spin_limit, int withhold_publish) {
    if (!plan) return BWT_EINVAL;
    plan->spin_limit = spin_limit ? spin_limit : kDefaultSpin;
    plan->withhold = withhold_publish ? 1 : 0;
    drop_graph(plan);
    return BWT_OK;
}

void bwt::drop_graph(bwt_plan* p) {
    for (auto& g : p->graphs) {
        if (g.launched) {
            cudaEventSynchronize(g.launched);  // its last launch may still run
            cudaEventDestroy(g.launched);
        }
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    p->graphs.clear();
}

// ---------------------------------------------------------------------------
// Argument checks and per-batch host tables.

bwt_status bwt::prepare_batch(bwt_plan* p, const uint64_t* offsets, uint32_t nb, cudaStream_t st) {
    if (nb == 0 || nb > p->cap_b || !offsets) return BWT_EINVAL;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, offsets);
    if (e != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) {
        // device offsets: read in stream order, which waits for the stream
        CK(cudaMemcpyAsync(p->h_off, offsets, sizeof(uint64_t) * (nb + 1), cudaMemcpyDefault, st));
        CK(cudaStreamSynchronize(st));
    } else {
        std::memcpy(p->h_off, offsets, sizeof(uint64_t) * (nb + 1));
    }
    const uint64_t* off = p->h_off;
    if (off[0] != 0) return BWT_EINVAL;
    for (uint32_t b = 0; b < nb; ++b) {
        if (off[b + 1] <= off[b]) return BWT_EINVAL;
        if (off[b + 1] - off[b] > p->desc.max_block_bytes) return BWT_EINVAL;
    }
    if (off[nb] > p->cap_n) return BWT_EINVAL;
    return upload_tables(p, off, nb, st);
}

// Block and first-sort tile tables for blocks off[b] .. off[b+1] (global
// positions as given), uploaded from pinned staging memory.
bwt_status bwt::upload_tables(bwt_plan* p, const uint64_t* off, uint32_t nb, cudaStream_t st) {
    const uint32_t T = (uint32_t)p->tile;
    std::vector<uint64_t> key;
    key.reserve((size_t)nb + 3);
    key.push_back(T);
    key.push_back((uint64_t)p->rbits);  // 16-bit digits add the part table
    key.push_back(nb);
    key.insert(key.end(), off, off + nb + 1);
    if (key == p->tables_key) return BWT_OK;  // the device tables already hold this layout
    p->tables_key.clear();
    // a staging slot is refilled only after the copy from it has run
    const int sl = p->stage_next;
    if (p->stage_used[sl]) CK(cudaEventSynchronize(p->stage_ev[sl]));
    p->h_tiles = p->stage_tiles[sl];
    p->h_blocks = p->stage_blocks[sl];
    uint32_t max_n = 0;
    uint32_t nt = 0;
    for (uint32_t b = 0; b < nb; ++b) {
        const uint32_t o = (uint32_t)off[b], n = (uint32_t)(off[b + 1] - off[b]);
        max_n = std::max(max_n, n);
        p->h_blocks[b] = BlockInfo{o, n};
        const uint32_t first = nt;
        for (uint32_t s = 0; s < n; s += T) {
            TileDesc td;
            td.start = o + s;
            td.len = std::min(T, n - s);
            td.seg = b;
            td.firstTile = first;
            td.segStart = o;
            td.blk = b;
            td.pad0 = n;
            td.pad1 = 0;
            p->h_tiles[nt++] = td;
        }
    }
    p->nb = nb;
    p->total = (uint32_t)(off[nb] - off[0]);
    p->max_n = max_n;
    p->ntiles0 = nt;
    CK(cudaMemcpyAsync(p->blocks, p->h_blocks, sizeof(BlockInfo) * nb, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(p->tiles0, p->h_tiles, sizeof(TileDesc) * nt, cudaMemcpyHostToDevice, st));
    p->nparts = 0;
    if (p->rbits == 16) {
        // parts of the 16-bit passes: up to PART16_KEYS consecutive rotations of one block
        TileDesc* hp = p->stage_parts[sl];
        uint32_t* hf = p->stage_pfirst[sl];
        uint32_t np = 0;
        for (uint32_t b = 0; b < nb; ++b) {
            const uint32_t o = (uint32_t)off[b], n = (uint32_t)(off[b + 1] - off[b]);
            hf[b] = np;
            for (uint32_t s0 = 0; s0 < n; s0 += PART16_KEYS) {
                if (np >= p->cap_parts) return BWT_EINVAL;
                hp[np++] = TileDesc{o + s0, std::min(PART16_KEYS, n - s0), b, hf[b], o, b, n, 0u};
            }
        }
        hf[nb] = np;
        p->nparts = np;
        CK(cudaMemcpyAsync(p->parts16, hp, sizeof(TileDesc) * np, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(p->part_first16, hf, sizeof(uint32_t) * (nb + 1), cudaMemcpyHostToDevice, st));
    }
    CK(cudaEventRecord(p->stage_ev[sl], st));
    p->stage_used[sl] = true;
    p->stage_next = sl ^ 1;
    p->tables_key = std::move(key);
    return BWT_OK;
}

Bins bwt::bins_of(bwt_plan* p, int par) {
    Bins b;
    for (int c = 0; c < NCLS; ++c) {
        b.list[c] = p->bins[par][c];
        b.cap[c] = p->bincap[c];
    }
    b.count = p->ctrl + CTRL_BINS + NCLS * par;
    b.active = reinterpret_cast<unsigned long long*>(p->ctrl + CTRL_ACTIVE);
    return b;
}

// Records an event pair around a radix launch when timing is on.
static cudaError_t timed_onesweep(bwt_plan* p, int key_bytes, bool from_s, const OneSweepParams& a,
                                  double bytes_per_key, uint64_t keys_host, int ctrl_keys_word, cudaStream_t st,
                                  int radix_bits = 0, bool first_sort = false) {
    const bool timing = !p->events.empty() && !p->capturing && p->ev_used + 2 <= p->events.size();
    if (timing) cudaEventRecord(p->events[p->ev_used], st);
    cudaError_t e = launch_onesweep(key_bytes, from_s, radix_bits ? radix_bits : p->rbits, p->tile, a, 0, st);
    if (timing) {
        cudaEventRecord(p->events[p->ev_used + 1], st);
        EvMeta m;
        m.bytes_per_key = bytes_per_key;
        m.first_sort = first_sort;
        m.keys_host = keys_host;
        m.ctrl_word = ctrl_keys_word;
        p->ev_meta.push_back(m);
        p->ev_used += 2;
    }
    p->stats.radix_launches++;
    p->stats.kernel_launches++;
    p->stats.radix_keys += keys_host;  // device-counted keys are added when the round's counts are read
    return e;
}

bwt_status bwt::reset_ctrl(bwt_plan* p, cudaStream_t st) {
    p->lazy_ranks = LazyRanks{};  // every rank stored, unless a learned first stage says otherwise
    CK(launch_reset_ctrl(p->ctrl, p->spin_limit, (uint32_t)p->withhold, p->ntiles0, st));
    p->stats.kernel_launches++;
    return BWT_OK;
}

// First sort: P passes over the u64 prefixes (the first pass builds the keys
// from the bytes), then naming into bins[0].
// The first sort with 16-bit digits: four reduce-then-scan passes (each four
// launches) over the part table, ending in buffer 1, then naming.
static bwt_status enqueue_initial_sort16(bwt_plan* p, const uint8_t* d_in, cudaStream_t st) {
    constexpr int P = 4;
    for (int ps = 0; ps < P; ++ps) {
        const bool timing = !p->events.empty() && !p->capturing && p->ev_used + 2 <= p->events.size();
        if (timing) cudaEventRecord(p->events[p->ev_used], st);
        NvtxRange nv(ps == 0 ? "pack+radix16" : "radix16", ps);
        CK(launch_first16_pass(ps == 0 ? nullptr : p->keys[(ps - 1) & 1], ps == 0 ? nullptr : p->vals[(ps - 1) & 1],
                               p->keys[ps & 1], p->vals[ps & 1], d_in, p->blocks, p->parts16, p->nparts,
                               p->part_first16, p->nb, 16 * ps, p->partcnt16, p->segtot16, p->ctrl, st));
        if (timing) {
            cudaEventRecord(p->events[p->ev_used + 1], st);
            EvMeta m{};
            m.bytes_per_key = ps == 0 ? 14.0 : 32.0;  // histogram key read (8) + scatter (12 + 12); S bytes first
            m.first_sort = true;
            m.keys_host = p->total;
            m.ctrl_word = -1;
            p->ev_meta.push_back(m);
            p->ev_used += 2;
        }
        p->stats.kernel_launches += 4;
        p->stats.radix_launches++;
        p->stats.radix_keys += p->total;
    }
    p->sa = p->vals[(P - 1) & 1];
    p->key2 = p->vals[P & 1];
    p->kA = reinterpret_cast<uint32_t*>(p->keys[P & 1]);
    p->vA = p->kA + p->cap_n;
    p->kB = reinterpret_cast<uint32_t*>(p->keys[(P - 1) & 1]);
    p->vB = p->kB + p->cap_n;
    return enqueue_naming(p, p->keys[(P - 1) & 1], st);
}

bwt_status bwt::enqueue_initial_sort(bwt_plan* p, const uint8_t* d_in, cudaStream_t st) {
    if (p->rbits == 16) return enqueue_initial_sort16(p, d_in, st);
    const int rb = p->rbits, RADIX = 1 << rb;
    const int P = (64 + rb - 1) / rb;
    const uint32_t nb = p->nb, nt = p->ntiles0;
    uint32_t* ctrl = p->ctrl;
    uint32_t seg_stride;
    if (rb == 8) {
        CK(cudaMemsetAsync(p->hist, 0, sizeof(uint32_t) * 256 * nb, st));
        CK(launch_hist_bytes(d_in, p->blocks, p->tiles0, nt, p->hist, st));
        CK(launch_scan_rows(p->hist, 256, nullptr, 0, nb, nb, st));
        seg_stride = 256;
    } else {
        CK(cudaMemsetAsync(p->hist, 0, sizeof(uint32_t) * 6 * 2048 * nb, st));
        CK(launch_hist_keys11(d_in, p->blocks, p->tiles0, nt, p->tile, p->hist, st));
        CK(launch_scan_rows(p->hist, 2048, nullptr, 0, nb * 6, nb * 6, st));
        seg_stride = 6 * 2048;
    }
    p->stats.kernel_launches += 2;
    // 8-bit digits: every pass gets its own look-back region (8 x 256 words a
    // tile fit the status array), all zeroed by one memset; 11-bit passes
    // reuse one region, zeroed before each
    const size_t region = (size_t)nt * RADIX;
    const bool one_memset = region * P <= p->cap_status;
    if (one_memset) CK(cudaMemsetAsync(p->status, 0, sizeof(uint32_t) * region * P, st));
    for (int ps = 0; ps < P; ++ps) {
        NvtxRange nv(ps == 0 ? "pack+radix" : "radix", ps);
        if (!one_memset) CK(cudaMemsetAsync(p->status, 0, sizeof(uint32_t) * region, st));
        OneSweepParams a{};
        a.kin = ps == 0 ? nullptr : p->keys[(ps - 1) & 1];
        a.vin = ps == 0 ? nullptr : p->vals[(ps - 1) & 1];
        a.kout = p->keys[ps & 1];
        a.vout = p->vals[ps & 1];
        a.S = d_in;
        a.blocks = p->blocks;
        a.tiles = p->tiles0;
        a.num_tiles = ctrl + CTRL_NTILES0;
        a.seg_base = p->hist + (rb == 8 ? 0 : ps * 2048);
        a.seg_base_stride = seg_stride;
        a.status = p->status + (one_memset ? region * ps : 0);
        a.tile_counter = ctrl + CTRL_TILE_CTR + ps;
        a.ctrl = ctrl;
        a.shift = ps * rb;
        CK(timed_onesweep(p, 8, ps == 0, a, ps == 0 ? 13.0 : 24.0, p->total, -1, st, 0, true));
    }
    p->sa = p->vals[(P - 1) & 1];
    p->key2 = p->vals[P & 1];
    p->kA = reinterpret_cast<uint32_t*>(p->keys[P & 1]);
    p->vA = p->kA + p->cap_n;
    p->kB = reinterpret_cast<uint32_t*>(p->keys[(P - 1) & 1]);
    p->vB = p->kB + p->cap_n;
    return enqueue_naming(p, p->keys[(P - 1) & 1], st);
}

bwt_status bwt::enqueue_naming(bwt_plan* p, const uint64_t* K, cudaStream_t st) {
    NvtxRange nv("name");
    CK(cudaMemsetAsync(p->ctrl + CTRL_BINS, 0, sizeof(uint32_t) * 2 * NCLS, st));
    CK(launch_name_initial(K, p->sa, p->blocks, p->tiles0, p->ntiles0, p->rank, bins_of(p, 0), p->ctrl, st));
    p->stats.kernel_launches++;
    return BWT_OK;
}

// One doubling round reading bins[par] and writing bins[par ^ 1]; the prefix
// length h sits in ctrl[CTRL_DEPTH]. host_counts: the three group counts when
// the host knows them (else null: persistent grids read them on the device).
bwt_status bwt::enqueue_round(bwt_plan* p, int par, const uint32_t* host_counts, cudaStream_t st) {
    NvtxRange nv("double", (int)p->stats.rounds);  // the round's index (0 while a graph is captured)
    const int kbits = bits_for(p->max_n - 1);
    const int rb = round_radix_bits(p), RADIX = 1 << rb;
    const int P2 = std::max(1, (kbits + rb - 1) / rb);
    uint32_t* ctrl = p->ctrl;
    const uint32_t* depth = ctrl + CTRL_DEPTH;
    Bins cur = bins_of(p, par), nxt = bins_of(p, par ^ 1);
    CK(cudaMemsetAsync(nxt.count, 0, sizeof(uint32_t) * NCLS, st));
    {
        int launched = 0;
        CK(launch_gather_small(p->sa, p->rank, p->blocks, cur, depth, p->key2, host_counts, st, &launched,
                               p->lazy_ranks));
        p->stats.kernel_launches += launched;
    }
    const bool large = !host_counts || host_counts[CLS_LARGE] > 0;
    const uint64_t k0 = p->stats.kernel_launches, r0 = p->stats.radix_launches;
    const uint32_t hist_cap = (uint32_t)std::min<uint64_t>(p->cap_hist, 0xffffffffu);
    const uint32_t status_cap = (uint32_t)std::min<uint64_t>(p->cap_status, 0xffffffffu);
    if (large) {
        const cudaStream_t ls = st;
        CK(launch_build_large_tiles(cur, p->tile, p->ltiles, p->cap_ltiles, ctrl, ls, p->seg_varied));
        CK(launch_zero_by_count(p->hist, cur.count + CLS_LARGE, (uint32_t)(P2 * RADIX), hist_cap, ls));
        // with one pass only, that pass would read and write SA in place: it
        // reads a copy instead
        CK(launch_large_prologue(p->sa, p->rank, p->blocks, p->ltiles, ctrl + CTRL_NUM_LTILES, depth, p->kA,
                                 P2 == 1 ? p->vA : nullptr, p->hist, rb, P2, p->seg_varied, ls, p->lazy_ranks));
        CK(launch_scan_rows(p->hist, RADIX, cur.count + CLS_LARGE, (uint32_t)P2, 0, (uint32_t)(p->cap_hist / RADIX),
                            ls));
        p->stats.kernel_launches += 4;
        for (int ps = 0; ps < P2; ++ps) {
            CK(launch_zero_by_count(p->status, ctrl + CTRL_NUM_LTILES, (uint32_t)RADIX, status_cap, ls));
            CK(cudaMemsetAsync(ctrl + CTRL_TILE_CTR + 16 + ps, 0, 4, ls));
            p->stats.kernel_launches++;
            OneSweepParams a{};
            const bool last = ps == P2 - 1;
            a.kin = ps == 0 ? p->kA : ((ps - 1) & 1 ? p->kA : p->kB);
            a.vin = ps == 0 ? (P2 == 1 ? p->vA : p->sa) : ((ps - 1) & 1 ? p->vA : p->vB);
            a.kout = last ? p->key2 : (ps & 1 ? p->kA : p->kB);
            a.vout = last ? p->sa : (ps & 1 ? p->vA : p->vB);
            a.blocks = p->blocks;
            a.tiles = p->ltiles;
            a.num_tiles = ctrl + CTRL_NUM_LTILES;
            a.seg_base = p->hist + ps * RADIX;
            a.seg_base_stride = (uint32_t)(P2 * RADIX);
            a.status = p->status;
            a.tile_counter = ctrl + CTRL_TILE_CTR + 16 + ps;
            a.ctrl = ctrl;
            a.shift = ps * rb;
            a.seg_varied = p->seg_varied;  // groups whose key2 are all equal do not move
            CK(timed_onesweep(p, 4, false, a, 16.0, 0, CTRL_LARGE_KEYS, ls, rb));
        }
        p->pending_large_passes = (uint32_t)P2;
    }
    const uint64_t k1 = p->stats.kernel_launches, r1 = p->stats.radix_launches;
    int launched = 0;
    CK(launch_sort_small(p->sa, p->key2, p->rank, p->blocks, cur, nxt, depth, host_counts, ctrl, st, &launched));
    p->stats.kernel_launches += launched;
    const uint64_t k2 = p->stats.kernel_launches;
    if (large) {
        CK(launch_rename_large(p->sa, p->key2, p->rank, p->blocks, p->ltiles, ctrl + CTRL_NUM_LTILES, nxt, depth,
                               p->seg_varied, ctrl, st));
        p->stats.kernel_launches++;
    }
    p->cap_large_kernels = (k1 - k0) + (p->stats.kernel_launches - k2);  // one round's large-group section
    p->cap_large_radix = r1 - r0;
    return BWT_OK;
}

bwt_status bwt::status_of_ctrl(const bwt_plan* p) {
    const uint32_t err = p->h_ctrl[CTRL_ERR];
    if (err & ERR_BOUNDS) return BWT_EINTERNAL;
    if (err & ERR_TIMEOUT) return BWT_ETIMEOUT;
    if (err & ERR_CAPACITY) return BWT_ECAPACITY;
    if (err & ERR_INPUT) return BWT_EINVAL;
    return BWT_OK;
}

bwt_status bwt::finish_status(bwt_plan* p, cudaStream_t st) {
    resolve_pending(p);  // the staging of h_ctrl below replaces an unread asynchronous result
    CK(cudaMemcpyAsync(p->h_ctrl, p->ctrl, sizeof(uint32_t) * CTRL_WORDS, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return status_of_ctrl(p);
}

void bwt::resolve_pending(bwt_plan* p) {
    if (!p->pending) return;
    p->pending = false;
    const cudaError_t e = cudaEventSynchronize(p->done_ev);
    if (e != cudaSuccess) {
        p->last = record_cuda(e, "cudaEventSynchronize");
        return;
    }
    p->last = status_of_ctrl(p);
    graph_stats(p);
    if (p->pending_learned) learned_stats(p);
    p->pending_learned = false;
    const uint64_t act = (uint64_t)p->h_ctrl[CTRL_ACTIVE] | ((uint64_t)p->h_ctrl[CTRL_ACTIVE + 1] << 32);
    p->stats.active_elements = act;
}

void bwt::collect_timing(bwt_plan* p) {
    for (size_t i = 0; i < p->ev_meta.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p->events[2 * i], p->events[2 * i + 1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        const EvMeta& m = p->ev_meta[i];
        if (m.chunk_sort) {
            p->stats.chunk_launches++;
            p->stats.chunk_ms += ms;
            continue;
        }
        const uint64_t keys = m.keys_host ? m.keys_host : m.keys_dev;
        p->stats.radix_ms += ms;
        p->radix_bytes += m.bytes_per_key * (double)keys;
        if (m.first_sort) {
            p->stats.first_launches++;
            p->stats.first_ms += ms;
            p->stats.first_bytes += m.bytes_per_key * (double)keys;
        }
    }
    p->ev_meta.clear();
    p->ev_used = 0;
}

static void resolve_large_keys(bwt_plan* p, uint32_t large_keys) {
    if (p->pending_large_passes) {
        p->stats.radix_keys += (uint64_t)p->pending_large_passes * large_keys;
        p->pending_large_passes = 0;
    }
    for (auto& m : p->ev_meta)
        if (m.ctrl_word >= 0 && !m.resolved) {
            m.keys_dev = large_keys;
            m.resolved = true;
        }
}

// Doubling rounds with the loop decided on the host (three counts read per
// round). Starts from bins[0] filled by the naming step.
bwt_status bwt::run_doubling_host_loop(bwt_plan* p, cudaStream_t st) {
    int par = 0;
    uint32_t depth = 8;
    // rounds of this batch (the statistic sums over the blocks of a
    // per-block call); doubling from 8 passes 2^32 after 29 rounds
    for (int round = 0; depth < p->max_n && round < 40; ++round) {
        CK(cudaMemcpyAsync(p->h_ctrl, p->ctrl, sizeof(uint32_t) * 24, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        resolve_large_keys(p, p->h_ctrl[CTRL_LARGE_KEYS]);
        if (p->h_ctrl[CTRL_ERR]) break;
        uint32_t counts[NCLS];
        uint64_t any = 0;
        for (int c = 0; c < NCLS; ++c) {
            counts[c] = std::min(p->h_ctrl[CTRL_BINS + NCLS * par + c], p->bincap[c]);
            any += counts[c];
        }
        if (any == 0) break;
        bwt_status s = enqueue_round(p, par, counts, st);
        if (s != BWT_OK) return s;
        CK(launch_round_end(p->ctrl, par, p->max_n, 0, 0, 0, st));  // advance the depth only
        p->stats.kernel_launches++;
        p->stats.rounds++;
        if (depth > 0x7fffffffu) break;
        depth *= 2;
        par ^= 1;
    }
    CK(cudaMemcpyAsync(p->h_ctrl + CTRL_LARGE_KEYS, p->ctrl + CTRL_LARGE_KEYS, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    resolve_large_keys(p, p->h_ctrl[CTRL_LARGE_KEYS]);
    return BWT_OK;
}

bwt_status bwt::run_plain_host_loop(bwt_plan* p, const uint8_t* d_in, uint8_t* d_L, int32_t* d_primary,
                                    cudaStream_t st) {
    bwt_status s;
    if ((s = reset_ctrl(p, st)) != BWT_OK) return s;
    if ((s = enqueue_initial_sort(p, d_in, st)) != BWT_OK) return s;
    if ((s = run_doubling_host_loop(p, st)) != BWT_OK) return s;
    NvtxRange nv("gather");
    CK(launch_gather_L(d_in, p->sa, p->blocks, p->tiles0, p->ntiles0, d_L, d_primary, p->ctrl, st));
    p->stats.kernel_launches++;
    return BWT_OK;
}

// Comparison mode: every block runs the whole launch chain on its own, one
// block after another (the batch's tables are rebuilt per block).
bwt_status bwt::run_per_block(bwt_plan* p, const uint8_t* d_in, uint8_t* d_L, int32_t* d_primary,
                              cudaStream_t st) {
    const uint32_t nb = p->nb;
    std::vector<uint64_t> off(p->h_off, p->h_off + nb + 1);
    uint64_t sub[2];
    for (uint32_t b = 0; b < nb; ++b) {
        CK(cudaStreamSynchronize(st));  // pinned staging tables are reused per block
        sub[0] = 0;
        sub[1] = off[b + 1] - off[b];
        bwt_status s = upload_tables(p, sub, 1, st);
        if (s != BWT_OK) return s;
        if ((s = run_plain_host_loop(p, d_in + off[b], d_L + off[b], d_primary + b, st)) != BWT_OK) return s;
        CK(cudaMemcpyAsync(p->h_ctrl, p->ctrl, sizeof(uint32_t) * CTRL_WORDS, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (p->h_ctrl[CTRL_ERR]) return status_of_ctrl(p);
    }
    return BWT_OK;
}

extern "C" bwt_status bwt_forward_batch(bwt_plan* p, const uint8_t* d_in, const uint64_t* offsets,
                                        uint32_t num_blocks, uint8_t* d_L, int32_t* d_primary, void* stream) {
    if (!p || !d_in || !offsets || !d_L || !d_primary) return BWT_EINVAL;
    if (cudaSetDevice(p->device) != cudaSuccess) return BWT_ECUDA;
    NvtxRange nv("bwt_forward_batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    p->pending = false;  // an unread result of an earlier call is superseded by this one
    p->pending_learned = false;
    std::memset(&p->stats, 0, sizeof(p->stats));
    p->radix_bytes = 0;
    p->pending_large_passes = 0;
    p->ev_meta.clear();
    p->ev_used = 0;
    bwt_status s = prepare_batch(p, offsets, num_blocks, st);
    if (s == BWT_OK && (const void*)d_in == (const void*)d_L) s = BWT_EINVAL;
    if (s != BWT_OK) {
        p->last = s;
        return s;
    }
    p->stats.radix_bits = (uint32_t)p->rbits;
    p->stats.round_radix_bits = (uint32_t)round_radix_bits(p);
    p->stats.tile_keys = (uint32_t)p->tile;
    const bool per_block = (p->desc.flags & BWT_F_PER_BLOCK_LAUNCH) != 0;
    const bool graph = !per_block && (p->desc.flags & BWT_F_GRAPH);
    const bool learned = !per_block && (p->desc.flags & BWT_F_LEARNED);
    if (graph) {
        // stream-ordered: enqueue the graph, then a copy of the control words
        // (by a kernel, not a copy engine: see launch_words_to_host) and an
        // event; status and statistics are read when asked for
        s = run_graph(p, d_in, d_L, d_primary, st);  // plain or learned first stage
        if (s == BWT_OK) {
            cudaError_t e = launch_words_to_host(p->hd_ctrl, p->ctrl, CTRL_WORDS, st);
            if (e == cudaSuccess) e = cudaEventRecord(p->done_ev, st);
            if (e == cudaSuccess) {
                p->pending = true;
                p->pending_learned = learned && p->h_bstats != nullptr;
                p->stats.radix_bytes = p->radix_bytes;
                p->last = BWT_OK;
                return BWT_OK;
            }
            s = record_cuda(e, "control-word copy / cudaEventRecord");
        }
        p->last = s;
        return s;
    }
    if (per_block) {
        s = run_per_block(p, d_in, d_L, d_primary, st);
    } else if (learned) {
        s = run_learned(p, d_in, d_L, d_primary, st);
    } else {
        s = run_plain_host_loop(p, d_in, d_L, d_primary, st);
    }
    if (s == BWT_OK) s = finish_status(p, st);
    else cudaStreamSynchronize(st);
    if (learned && s != BWT_ENOMODEL && p->h_bstats) learned_stats(p);
    if (!p->events.empty()) collect_timing(p);
    const uint64_t act = (uint64_t)p->h_ctrl[CTRL_ACTIVE] | ((uint64_t)p->h_ctrl[CTRL_ACTIVE + 1] << 32);
    p->stats.active_elements = act;
    p->stats.radix_bytes = p->radix_bytes;
    p->last = s;
    return s;
}
