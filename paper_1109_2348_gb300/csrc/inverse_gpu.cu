// Inverse BWT of a batch on the GPU.
//
// The transform is undone from L and the primary index alone (Section 3.1).
// F, the first column, is L sorted; FL[j] is the row whose rotation starts
// one position after row j's (the occurrence of F[j] in L, counted stably).
// From row r_0 = primary (rotation 0): S[i] = F[r_i] and r_{i+1} = FL[r_i].
//
// That walk is one dependent chain per block, so it is split:
//   1. one stable 8-bit radix pass over (L[k], k) gives F and FL (the plain
//      path's first-pass kernel with the digit taken from the top key byte);
//      they are packed as (FL << 8) | F, one load per step;
//   2. walkers start at every SMP-th row and at the primary row and walk FL
//      until the next such row (each row of a cycle is visited once); the
//      stride and the walkers in flight are set so that the blocks being
//      walked keep their tables in L2 (measured: stride 16 with 4 walkers a
//      lane at 4 CTAs per SM beat strides 8 to 64 and 6 or 8 walkers);
//   3. pointer jumping over the samples, with the list cut at the primary,
//      gives every sample on the primary's cycle its distance to the end,
//      hence its text offset;
//   4. the walks are repeated, writing S at those offsets.
// A periodic block S = u^k has k cycles of |u| rows; the primary's cycle
// gives u, and the block is u repeated.
#include <algorithm>
#include <cstring>
#include <vector>

#include "bwt.h"
#include "kernels.h"
#include "plan_internal.h"

using namespace bwt;

#define CKI(call)                                              \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return record_cuda(_e, #call);  \
    } while (0)

namespace {

constexpr uint32_t SMP = 16;     // every SMP-th row starts a walk
constexpr uint32_t WPT = 4;      // walkers per thread
constexpr uint32_t SL = 256 * WPT;  // samples per work item
constexpr uint32_t END = 0xffffffffu, INVALID = 0xfffffffeu;

struct InvCtx {
    const BlockInfo* blocks;
    const int32_t* primary;
    const uint32_t* items;  // [nb + 1] prefix of work items over the blocks (pointer jumping)
    const uint32_t* qbase;  // [nb + 1] prefix of sample counts (m_b + 1) over the blocks (walks)
    uint32_t nb;
    const void* P;          // (FL << 8) | F per row, global index: u32 for blocks under 2^24 bytes, else u64
    uint32_t* nxt;          // per sample slot: slot where its walk stops
    uint32_t* len;          // per sample slot: steps of its walk
    uint32_t* nx0;          // pointer jumping, first buffer: next slot (END at the primary, INVALID unused)
    uint32_t* dist0;        // pointer jumping, first buffer: steps to the end of the list
    uint8_t* out;
    uint32_t* ctrl;
};

// Sample slots of block b start at off / SMP + 3b: the blocks' ranges of
// m_b + 1 slots (m_b = ceil(n_b / SMP) strided rows plus the primary) never
// overlap.
__device__ __forceinline__ uint32_t slot_base(BlockInfo bi, uint32_t b) { return bi.off / SMP + 3u * b; }

// Last b with pre[b] <= k (pre[0] = 0, k < pre[nb]).
__device__ __forceinline__ uint32_t find_block(const uint32_t* pre, uint32_t nb, uint32_t k) {
    uint32_t lo = 0, hi = nb;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= k) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t block_of_item(const InvCtx& c, uint32_t k) { return find_block(c.items, c.nb, k); }

template <typename PT>
__global__ void k_inv_pack(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ fl, uint32_t total,
                           PT* __restrict__ P) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += gridDim.x * blockDim.x)
        P[j] = (PT)(((uint64_t)fl[j] << 8) | (keys[j] >> 56));
}

// Walks of every sample (WRITE = false: from its row to the next sample row,
// recording where and after how many steps it stops) or of the samples on
// the primary's cycle (WRITE = true: the same walks again, writing S at the
// sample's text offset). Walks differ a lot in length, so walkers are not
// tied to a work item: each warp takes ranges of CH sample ids from a global
// counter, and a lane starts its next walk as soon as one of its WALKERS
// walks ends. A walk is one dependent load per step; a walker holds only
// global row indices and counters, so many walks per SM are in flight.
// Runs only after the radix pass succeeded (FL is then a permutation of
// every block); nx/dd: the pointer-jumping result (WRITE only).
constexpr uint32_t CH = 64;
constexpr int WALKERS = 4;
constexpr int WALK_CTAS_PER_SM = 4;

template <bool WRITE, typename PT>
__global__ void __launch_bounds__(256, WALK_CTAS_PER_SM) k_inv_walks(InvCtx c, uint32_t Q,
                                                                     uint32_t* __restrict__ counter,
                                                                     const uint32_t* __restrict__ nx,
                                                                     const uint32_t* __restrict__ dd) {
    if (ld_volatile(&c.ctrl[CTRL_ERR]) & (ERR_TIMEOUT | ERR_CAPACITY)) return;
    const PT* __restrict__ P = static_cast<const PT*>(c.P);
    const uint32_t lane = threadIdx.x & 31, lt = lanemask_lt();
    uint32_t wq = 0, wq_end = 0;  // warp-uniform range of sample ids not started yet
    bool exhausted = false;
    // per walker: global row, its block's first row, then
    //   walk:  global row of the primary, sample slot, steps taken, block
    //   write: global text position, steps left
    uint32_t R[WALKERS], off[WALKERS], a[WALKERS], g[WALKERS], cnt[WALKERS], blk[WALKERS];
    bool act[WALKERS];
#pragma unroll
    for (int j = 0; j < WALKERS; ++j) act[j] = false;
    for (;;) {
        // start a walk in every idle slot, as long as samples are left
#pragma unroll
        for (int j = 0; j < WALKERS; ++j) {
            bool need = !act[j];
            for (;;) {
                const uint32_t mask = __ballot_sync(0xffffffffu, need && !exhausted);
                if (mask == 0u) break;
                if (wq == wq_end) {
                    uint32_t q0 = 0;
                    if (lane == 0) q0 = atomicAdd(counter, CH);
                    q0 = __shfl_sync(0xffffffffu, q0, 0);
                    if (q0 >= Q) {
                        exhausted = true;
                        break;
                    }
                    wq = q0;
                    wq_end = min(q0 + CH, Q);
                    continue;
                }
                const uint32_t take = min((uint32_t)__popc(mask), wq_end - wq);
                const uint32_t rk = __popc(mask & lt);
                if (need && rk < take) {
                    const uint32_t q = wq + rk;
                    const uint32_t b = find_block(c.qbase, c.nb, q);
                    const uint32_t s = q - c.qbase[b];
                    const BlockInfo bi = c.blocks[b];
                    const int32_t ps = c.primary[b];
                    if (ps < 0 || (uint32_t)ps >= bi.n) {
                        if (s == 0) atomicOr(&c.ctrl[CTRL_ERR], ERR_INPUT);
                    } else {
                        const uint32_t m = (bi.n + SMP - 1) / SMP, base = slot_base(bi, b), slot = base + s;
                        const uint32_t row = s < m ? s * SMP : (uint32_t)ps;
                        bool start;
                        if constexpr (!WRITE) {
                            start = !(s < m && row == (uint32_t)ps);  // the primary row walks as slot m
                            if (!start) c.nxt[slot] = INVALID;
                            a[j] = bi.off + (uint32_t)ps;
                            g[j] = slot;
                            cnt[j] = 0;
                            blk[j] = b;
                        } else {
                            start = nx[slot] == END;  // on the primary's cycle
                            if (start) {
                                a[j] = bi.off + dd[base + m] - dd[slot];  // cycle length - distance to the end
                                cnt[j] = c.len[slot];
                            }
                        }
                        if (start) {
                            R[j] = bi.off + row;
                            off[j] = bi.off;
                            act[j] = true;
                            need = false;
                        }
                    }
                }
                wq += take;
            }
        }
        bool any = false;
#pragma unroll
        for (int j = 0; j < WALKERS; ++j) any |= act[j];
        if (!__any_sync(0xffffffffu, any) && exhausted) break;
        // one step of every walk
        PT v[WALKERS];
#pragma unroll
        for (int j = 0; j < WALKERS; ++j) v[j] = act[j] ? P[R[j]] : (PT)0;
#pragma unroll
        for (int j = 0; j < WALKERS; ++j) {
            if (!act[j]) continue;
            const uint32_t nr = off[j] + (uint32_t)(v[j] >> 8);
            if constexpr (WRITE) {
                c.out[a[j]] = (uint8_t)(v[j] & 0xffu);
                ++a[j];
                R[j] = nr;
                if (--cnt[j] == 0) act[j] = false;
            } else {
                R[j] = nr;
                ++cnt[j];
                if (nr == a[j] || ((nr - off[j]) & (SMP - 1)) == 0) {
                    const BlockInfo bi = c.blocks[blk[j]];
                    const uint32_t base = slot_base(bi, blk[j]), m = (bi.n + SMP - 1) / SMP;
                    c.nxt[g[j]] = nr == a[j] ? base + m : base + (nr - off[j]) / SMP;
                    c.len[g[j]] = cnt[j];
                    act[j] = false;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_inv_jump_init(InvCtx c, uint32_t nitems) {
    for (uint32_t k = blockIdx.x; k < nitems; k += gridDim.x) {
        const uint32_t b = block_of_item(c, k);
        const BlockInfo bi = c.blocks[b];
        const int32_t prim_s = c.primary[b];
        if (prim_s < 0 || (uint32_t)prim_s >= bi.n) continue;
        const uint32_t m = (bi.n + SMP - 1) / SMP, base = slot_base(bi, b);
        const uint32_t s0 = (k - c.items[b]) * SL + threadIdx.x;
        for (uint32_t j = 0; j < WPT; ++j) {
            const uint32_t s = s0 + j * 256;
            if (s > m) break;
            const uint32_t g = base + s, t = c.nxt[g];
            c.nx0[g] = t == INVALID ? INVALID : (t == base + m ? END : t);
            c.dist0[g] = t == INVALID ? 0u : c.len[g];
        }
    }
}

// One pointer-jumping round: dist += dist[next], next = next[next].
__global__ void __launch_bounds__(256) k_inv_jump(InvCtx c, uint32_t nitems, const uint32_t* __restrict__ nx,
                                                  const uint32_t* __restrict__ dd, uint32_t* __restrict__ nx2,
                                                  uint32_t* __restrict__ dd2) {
    for (uint32_t k = blockIdx.x; k < nitems; k += gridDim.x) {
        const uint32_t b = block_of_item(c, k);
        const BlockInfo bi = c.blocks[b];
        const int32_t prim_s = c.primary[b];
        if (prim_s < 0 || (uint32_t)prim_s >= bi.n) continue;
        const uint32_t m = (bi.n + SMP - 1) / SMP, base = slot_base(bi, b);
        const uint32_t s0 = (k - c.items[b]) * SL + threadIdx.x;
        for (uint32_t j = 0; j < WPT; ++j) {
            const uint32_t s = s0 + j * 256;
            if (s > m) break;
            const uint32_t g = base + s, t = nx[g];
            if (t < INVALID) {
                dd2[g] = dd[g] + dd[t];
                nx2[g] = nx[t];
            } else {
                dd2[g] = dd[g];
                nx2[g] = t;
            }
        }
    }
}

// Periodic blocks: the primary's cycle covers one period; repeat it.
__global__ void k_inv_replicate(InvCtx c, const TileDesc* __restrict__ tiles, uint32_t ntiles,
                                const uint32_t* __restrict__ dd) {
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileDesc td = tiles[t];
        const BlockInfo bi = c.blocks[td.blk];
        const int32_t prim_s = c.primary[td.blk];
        if (prim_s < 0 || (uint32_t)prim_s >= bi.n) continue;
        const uint32_t m = (bi.n + SMP - 1) / SMP;
        const uint32_t cyc = dd[slot_base(bi, td.blk) + m];
        if (cyc == 0 || cyc >= bi.n) continue;
        const uint32_t q0 = td.start - bi.off;
        for (uint32_t q = threadIdx.x; q < td.len; q += blockDim.x)
            if (q0 + q >= cyc) c.out[td.start + q] = c.out[bi.off + (q0 + q) % cyc];
    }
}

}  // namespace

extern "C" bwt_status bwt_inverse_batch(bwt_plan* p, const uint8_t* d_L, const uint64_t* offsets,
                                        uint32_t num_blocks, const int32_t* d_primary, uint8_t* d_out,
                                        void* stream) {
    if (!p || !d_L || !offsets || !d_primary || !d_out || (const void*)d_L == (const void*)d_out) return BWT_EINVAL;
    bwt::NvtxRange nvtx_range("inverse");
    if (cudaSetDevice(p->device) != cudaSuccess) return BWT_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::memset(&p->stats, 0, sizeof(p->stats));
    bwt_status s = prepare_batch(p, offsets, num_blocks, st);
    if (s != BWT_OK) return p->last = s;
    const uint32_t nb = p->nb, nt = p->ntiles0, total = p->total;
    // work items and samples per block, and the sample-slot scratch (allocated on first use)
    uint32_t nitems = 0, Q = 0, max_m = 0;
    uint32_t* h_items = p->h_inv_items;
    uint32_t* h_qbase = p->h_inv_items + p->cap_b + 1;
    for (uint32_t b = 0; b < nb; ++b) {
        h_items[b] = nitems;
        h_qbase[b] = Q;
        const uint32_t m = (p->h_blocks[b].n + SMP - 1) / SMP;
        max_m = std::max(max_m, m);
        nitems += (m + 1 + SL - 1) / SL;
        Q += m + 1;
    }
    h_items[nb] = nitems;
    h_qbase[nb] = Q;
    const size_t slots = (size_t)(p->cap_n / SMP) + 3 * (size_t)p->cap_b + 4;
    if (!p->inv_slots) CKI(cudaMalloc(&p->inv_slots, sizeof(uint32_t) * 6 * slots));
    if (!p->inv_items) CKI(cudaMalloc(&p->inv_items, sizeof(uint32_t) * 2 * ((size_t)p->cap_b + 1)));
    CKI(cudaMemcpyAsync(p->inv_items, h_items, sizeof(uint32_t) * 2 * ((size_t)p->cap_b + 1),
                        cudaMemcpyHostToDevice, st));
    if ((s = reset_ctrl(p, st)) != BWT_OK) return p->last = s;

    // 1. F and FL: one stable pass over (L[k], k), digit = the top key byte
    CKI(cudaMemsetAsync(p->hist, 0, sizeof(uint32_t) * 256 * nb, st));
    CKI(launch_hist_bytes(d_L, p->blocks, p->tiles0, nt, p->hist, st));
    CKI(launch_scan_rows(p->hist, 256, nullptr, 0, nb, nb, st));
    CKI(cudaMemsetAsync(p->status, 0, sizeof(uint32_t) * (size_t)nt * 256, st));
    OneSweepParams a{};
    a.kout = p->keys[0];
    a.vout = p->vals[0];
    a.S = d_L;
    a.blocks = p->blocks;
    a.tiles = p->tiles0;
    a.num_tiles = p->ctrl + CTRL_NTILES0;
    a.seg_base = p->hist;
    a.seg_base_stride = 256;
    a.status = p->status;
    a.tile_counter = p->ctrl + CTRL_TILE_CTR;
    a.ctrl = p->ctrl;
    a.shift = 56;
    CKI(launch_onesweep(8, true, 8, p->tile, a, 0, st));
    const int sms = num_sms();
    // packed (FL << 8) | F: 4 bytes a row while block rows fit in 24 bits, so
    // twice as many blocks' tables stay in L2 during the walks
    const bool p32 = p->max_n <= (1u << 24);
    void* P = p->keys[1];
    if (p32) k_inv_pack<uint32_t><<<sms * 8, 256, 0, st>>>(p->keys[0], p->vals[0], total, (uint32_t*)P);
    else k_inv_pack<uint64_t><<<sms * 8, 256, 0, st>>>(p->keys[0], p->vals[0], total, (uint64_t*)P);

    // 2-4. walks, pointer jumping, writes
    InvCtx c{};
    c.blocks = p->blocks;
    c.primary = d_primary;
    c.items = p->inv_items;
    c.qbase = p->inv_items + p->cap_b + 1;
    c.nb = nb;
    c.P = P;
    c.nxt = p->inv_slots;
    c.len = p->inv_slots + slots;
    uint32_t* nxb[2] = {p->inv_slots + 2 * slots, p->inv_slots + 3 * slots};
    uint32_t* ddb[2] = {p->inv_slots + 4 * slots, p->inv_slots + 5 * slots};
    c.nx0 = nxb[0];
    c.dist0 = ddb[0];
    c.out = d_out;
    c.ctrl = p->ctrl;
    const int grid = std::max(1, std::min<int>(nitems, sms * 8));
    // walkers in flight: enough to hide latency, few enough that the blocks
    // being walked keep their tables in L2
    const int wgrid = sms * WALK_CTAS_PER_SM;
    uint32_t* counters = p->ctrl + CTRL_TILE_CTR + 60;  // zeroed by reset_ctrl; no radix pass of this call uses them
    if (p32) k_inv_walks<false, uint32_t><<<wgrid, 256, 0, st>>>(c, Q, counters, nullptr, nullptr);
    else k_inv_walks<false, uint64_t><<<wgrid, 256, 0, st>>>(c, Q, counters, nullptr, nullptr);
    k_inv_jump_init<<<grid, 256, 0, st>>>(c, nitems);
    int src = 0, rounds = 1;
    while ((1u << (rounds - 1)) < max_m + 2) ++rounds;  // >= log2(samples per block) + 1
    for (int i = 0; i < rounds; ++i, src ^= 1)
        k_inv_jump<<<grid, 256, 0, st>>>(c, nitems, nxb[src], ddb[src], nxb[src ^ 1], ddb[src ^ 1]);
    if (p32) k_inv_walks<true, uint32_t><<<wgrid, 256, 0, st>>>(c, Q, counters + 1, nxb[src], ddb[src]);
    else k_inv_walks<true, uint64_t><<<wgrid, 256, 0, st>>>(c, Q, counters + 1, nxb[src], ddb[src]);
    k_inv_replicate<<<std::max(1, std::min<int>(nt, sms * 8)), 256, 0, st>>>(c, p->tiles0, nt, ddb[src]);
    CKI(cudaGetLastError());
    p->stats.kernel_launches = 10 + rounds;
    p->stats.radix_launches = 1;
    p->stats.radix_keys = total;
    return p->last = finish_status(p, st);
}
