/*
 * bwt.h -- C ABI of the GB300 forward Burrows-Wheeler block sort.
 *
 * The operation (Section 3.1 of the paper: the forward transform "sorts the
 * rotations" of a block, after Burrows and Wheeler 1994):
 *   a block is n bytes S[0..n-1]; rotation i is S[i..n-1] S[0..i-1];
 *   SA = the permutation of 0..n-1 ordered by (rotation i as unsigned bytes,
 *        then i ascending), so identical rotations keep lower-index-first;
 *   L[k] = S[(SA[k] + n - 1) mod n] is the last column of the sorted matrix;
 *   primary = the row k with SA[k] = 0, i.e. where the original block sits.
 * There is no sentinel byte and no bzip2-specific pre-processing.
 *
 * Batches: num_blocks independent blocks concatenated in one byte buffer;
 * block b is in[offsets[b] .. offsets[b+1]). L uses the same layout and
 * primary[b] is block b's primary index (0-based, relative to the block).
 *
 * Memory: every pointer named d_* is device memory owned by the caller. The
 * plan owns all scratch; it is sized at plan creation from the descriptor
 * (including the learned bucketing's tables when BWT_F_LEARNED is set), so
 * bwt_forward_batch allocates nothing. bwt_inverse_batch and bwt_mtf_encode
 * allocate their extra scratch once, on their first call on the plan; the
 * MLP training calls allocate temporaries (each says so). All entry points
 * return a bwt_status and never abort the process; kernels never trap.
 * Device-side failures (a bounded wait that ran out, a capacity overflow) are
 * recorded in a device status word: the synchronous calls return it, and an
 * asynchronous bwt_forward_batch (BWT_F_GRAPH) leaves it for
 * bwt_plan_last_status.
 *
 * Thread safety and ordering: a plan may be used by one host thread at a
 * time, and its calls must run in order on the GPU (one stream, or streams
 * the caller orders with events): consecutive calls share the plan's scratch.
 */
#ifndef BWT_GB300_H
#define BWT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bwt_plan bwt_plan;

typedef enum {
    BWT_OK = 0,
    BWT_EINVAL = 1,     /* bad argument: NULL pointer, empty block, offsets not increasing, size over the plan's limits */
    BWT_ENOMEM = 2,     /* device or pinned host allocation failed at plan creation */
    BWT_ECAPACITY = 3,  /* a device-side work list overflowed (internal limit) */
    BWT_ECUDA = 4,      /* a CUDA runtime call failed; see bwt_last_cuda_error() */
    BWT_ETIMEOUT = 5,   /* a bounded device-side wait ran out; outputs are undefined */
    BWT_EMISMATCH = 6,  /* bwt_inverse_check: the inverse of L does not reproduce the block */
    BWT_ENOMODEL = 7,   /* BWT_F_LEARNED without a loaded splitter table */
    BWT_ETOOBIG = 8,    /* bwt_forward_block_noalloc: block larger than BWT_NOALLOC_MAX_BYTES */
    BWT_EINTERNAL = 9   /* a bounds check of the debug build (-DBWT_DEBUG) failed: an internal error; the
                           release build clamps the same indices and never reports it */
} bwt_status;

/* plan flags */
#define BWT_F_GRAPH            0x1u /* capture the whole batch in a CUDA graph and replay it when the
                                       block sizes repeat; the prefix-doubling loop is a device-side
                                       conditional WHILE node, so no host round trip per round */
#define BWT_F_LEARNED          0x2u /* learned-CDF bucketing before the exact sort (needs a model) */
#define BWT_F_PER_BLOCK_LAUNCH 0x4u /* comparison mode: sort block after block, one launch chain each */
#define BWT_F_TIMING           0x8u /* record CUDA events around every radix pass (see bwt_plan_stats) */

typedef struct {
    uint32_t max_blocks;       /* most blocks per call (>= 1) */
    uint64_t max_total_bytes;  /* most bytes per call, summed over blocks (< 2^32) */
    uint32_t max_block_bytes;  /* largest block (1 .. 2^30 - 1) */
    int radix_bits;            /* first sort's LSD digit width: 8, 11 or 16; 0 = the default (8) or the
                                  autotuned value. 16 adds about 4.3 bytes per byte of max_total_bytes
                                  plus 256 KB per block of scratch */
    int tile_keys;             /* keys per radix tile: 1024, 2048 or 4096; 0 = default (4096) */
    uint32_t flags;            /* BWT_F_* */
    const char* model_path;    /* splitter table for BWT_F_LEARNED (bwt_model_compile output); may be NULL */
} bwt_plan_desc;

/* Plan statistics of the last bwt_forward_batch call. */
typedef struct {
    uint32_t rounds;            /* prefix-doubling rounds executed (a batch shares its rounds; with
                                   BWT_F_PER_BLOCK_LAUNCH, summed over the blocks) */
    uint32_t radix_bits, tile_keys;
    uint64_t kernel_launches;   /* kernels launched (graph replays count the kernels they run) */
    uint64_t radix_launches;    /* onesweep radix-pass launches */
    uint64_t radix_keys;        /* keys moved by those launches, summed */
    double radix_ms;            /* their summed device time (only with BWT_F_TIMING) */
    double radix_bytes;         /* their algorithmic HBM bytes: 24 per u64 key (8 + 4 read, 8 + 4
                                   written), 13 for the first pass (1 byte read), 16 per u32 key;
                                   a 16-bit pass counts 32 (8 histogram read + 24), its first 14 */
    uint64_t active_elements;   /* rotations re-sorted by doubling rounds, summed over rounds */
    uint64_t buckets_overflowed;/* learned bucketing: buckets above the 3,328-rotation chunk (each
                                   sorted whole by one CTA up to 13,312 rotations, by the radix
                                   path beyond) */
    uint64_t keys_overflowed;   /* learned bucketing: keys in those buckets */
    uint32_t max_bucket;        /* learned bucketing: largest bucket */
    uint32_t graph_replayed;    /* 1 if the last call replayed a cached CUDA graph */
    uint32_t blocks_routed_plain; /* learned bucketing: blocks whose buckets overflowed too much and
                                     were sorted by the plain radix path instead */
    uint32_t blocks_routed_flat;  /* learned bucketing: blocks bucketed by equal-width splitters (the top
                                     12 key bits) because the learned buckets overflowed */
    uint64_t bucket_sq_sum;     /* learned bucketing: sum over all blocks and buckets of size^2 (the
                                   in-bucket sort work; smallest when buckets are even) */
    uint64_t buckets_nonempty;  /* learned bucketing: non-empty buckets over all blocks */
    uint32_t round_radix_bits;  /* digit width of the doubling rounds' radix */
    uint32_t pad2_;
    uint64_t first_launches;    /* the first sort's u64 passes alone (a subset of radix_launches) */
    double first_ms;            /* their summed device time (only with BWT_F_TIMING) */
    double first_bytes;         /* their algorithmic HBM bytes (13 per key for the first pass, 24 after) */
    uint64_t chunk_launches;    /* learned bucketing: timed launches of the 256-thread chunk sort (only
                                   with BWT_F_TIMING and without BWT_F_GRAPH) */
    double chunk_ms;            /* their summed device time */
    uint64_t chunk_keys;        /* learned bucketing: rotations in packed chunks (the ones that chunk
                                   sort sorts: the bucketed blocks' rotations outside over-full buckets) */
    double chunk_bytes;         /* their algorithmic HBM bytes: 16 per rotation (8-byte key and 4-byte
                                   index read, 4-byte SA entry written; ranks are stored only for
                                   rotations in groups of two or more) */
} bwt_stats;

/* Create a plan on CUDA device `device` (made current for the call). The plan
 * allocates all scratch for desc's limits (about 40 bytes per byte of
 * max_total_bytes). Returns BWT_EINVAL for bad limits, BWT_ENOMEM if the
 * allocation fails, BWT_ENOMODEL if BWT_F_LEARNED is set and model_path is
 * given but cannot be read (without model_path, install splitters with
 * bwt_plan_set_splitters before the first call). *out is NULL on failure. */
bwt_status bwt_plan_create(const bwt_plan_desc* desc, int device, bwt_plan** out);

/* Forward BWT of a batch (the definition at the top of this header).
 *   d_in        device, uint8[offsets[num_blocks]]: the blocks, concatenated.
 *   offsets     uint64[num_blocks + 1], offsets[0] = 0, strictly increasing
 *               (empty blocks are BWT_EINVAL). Host or device memory; device
 *               offsets are copied to the host in stream order, which waits
 *               for `stream` (pass host offsets to avoid that).
 *   num_blocks  1 .. max_blocks.
 *   d_L         device, uint8[offsets[num_blocks]]: the L column, same layout.
 *   d_primary   device, int32[num_blocks].
 *   stream      cudaStream_t to run on (NULL = the legacy default stream).
 * Argument errors are returned at once. The work is stream-ordered:
 *   - with BWT_F_GRAPH (and not BWT_F_PER_BLOCK_LAUNCH) the call only
 *     enqueues it -- the block and tile tables when the layout differs from
 *     the plan's last one, then the batch's CUDA graph -- and returns BWT_OK
 *     without waiting for the GPU (with host offsets). The device-side status
 *     and the statistics of the call are read by bwt_plan_last_status and
 *     bwt_plan_stats, which wait for the call's work to finish; they describe
 *     the most recent call only. Outputs are valid once the stream has
 *     reached the end of the call and bwt_plan_last_status is BWT_OK;
 *   - the other modes decide the doubling rounds on the host, synchronise
 *     `stream` and return the device-side status themselves.
 * d_in must not alias d_L. */
bwt_status bwt_forward_batch(bwt_plan* plan, const uint8_t* d_in, const uint64_t* offsets,
                             uint32_t num_blocks, uint8_t* d_L, int32_t* d_primary, void* stream);

/* Host-side check of one block: inverts L by the LF walk from `primary`
 * (Section 3.1: the inverse may start from any row) and compares the result
 * with `original`. All pointers are host memory of n bytes.
 * BWT_OK if it reproduces `original`; BWT_EMISMATCH if not, or if L is not a
 * permutation of `original`; BWT_EINVAL for n = 0, NULL pointers or a primary
 * outside [0, n). */
bwt_status bwt_inverse_check(const uint8_t* L, uint64_t n, int32_t primary, const uint8_t* original);

/* Inverse BWT of a batch on the device (Section 3.1: a block is recovered
 * from its L column and primary index alone).
 *   d_L         device, uint8[offsets[num_blocks]]: the L columns, concatenated.
 *   offsets     as in bwt_forward_batch (host or device memory).
 *   d_primary   device, int32[num_blocks]: the primary index of every block.
 *   d_out       device, uint8[offsets[num_blocks]]: receives the blocks.
 *   stream      cudaStream_t to run on (NULL = the legacy default stream).
 * Uses the plan's scratch plus about 1.5 bytes per byte of max_total_bytes
 * allocated on the first call. Returns BWT_EINVAL for bad arguments and for a primary
 * outside [0, n) (found on the device; that block's output is undefined).
 * The call synchronises `stream` before it returns. d_out must not alias
 * d_L. For any L that is a permutation of some block's bytes the result is
 * the block whose BWT (with this primary) is L. */
bwt_status bwt_inverse_batch(bwt_plan* plan, const uint8_t* d_L, const uint64_t* offsets, uint32_t num_blocks,
                             const int32_t* d_primary, uint8_t* d_out, void* stream);

/* ---- the stages after the block sort (Sections 3.2-3.4) ---------------
 * They take a plan for its scratch and its batch checks (offsets as in
 * bwt_forward_batch, host or device memory); they run on `stream` and
 * synchronise it before returning. */

/* Run-length encoding of a batch (Section 3.2, Fig. 1): every block becomes
 * its maximal runs, in order; runs never cross blocks.
 *   d_in       device, uint8[offsets[num_blocks]]: the blocks.
 *   d_chars    device, uint8[offsets[num_blocks]] (room for one run a byte):
 *              the byte of every run, block after block.
 *   d_lens     device, uint32[offsets[num_blocks]]: every run's length.
 *   d_run_off  device, uint64[num_blocks + 1]: block b's runs are
 *              [d_run_off[b], d_run_off[b + 1]); d_run_off[num_blocks] is the
 *              number of runs. */
bwt_status bwt_rle_encode(bwt_plan* plan, const uint8_t* d_in, const uint64_t* offsets, uint32_t num_blocks,
                          uint8_t* d_chars, uint32_t* d_lens, uint64_t* d_run_off, void* stream);

/* Run-length decoding (Section 3.2, Fig. 2), the inverse of bwt_rle_encode:
 * d_chars, d_lens and d_run_off as it writes them; `offsets` gives the
 * decoded blocks' layout; d_out (device, uint8[offsets[num_blocks]])
 * receives the blocks. Returns BWT_EINVAL if a length is zero or a block's
 * runs do not add up to its size (checked on the device; d_out is then
 * undefined). */
bwt_status bwt_rle_decode(bwt_plan* plan, const uint8_t* d_chars, const uint32_t* d_lens, const uint64_t* d_run_off,
                          const uint64_t* offsets, uint32_t num_blocks, uint8_t* d_out, void* stream);

/* Variable-length encoding of a batch (Section 3.4, Fig. 3): every byte c is
 * replaced by its codeword -- the low d_len[c] bits of d_code[c], 1 <= length
 * <= 32 -- written most significant bit first into a bit stream whose bit p
 * is bit 7 - (p mod 8) of byte p / 8; each block's stream starts at a byte
 * boundary and its last byte is padded with zero bits.
 *   d_code, d_len  device, uint32[256] and uint8[256]: the codeword table (a
 *                  precomputed table, as the paper proposes; any table works,
 *                  decodability is the caller's choice).
 *   d_out          device, 4-byte aligned, out_cap bytes; it must hold the
 *                  total stream rounded up to a multiple of 4 bytes (at most
 *                  4 * offsets[num_blocks] + 4).
 *   d_byte_off     device, uint64[num_blocks + 1]: block b's stream starts at
 *                  byte d_byte_off[b]; d_byte_off[num_blocks] is the total.
 *   d_block_bits   device, uint64[num_blocks]: the bits of every stream.
 * Returns BWT_EINVAL if a byte of the input has a length outside 1..32 (or
 * d_out is misaligned), BWT_ECAPACITY if out_cap is too small. */
bwt_status bwt_vle_encode(bwt_plan* plan, const uint8_t* d_in, const uint64_t* offsets, uint32_t num_blocks,
                          const uint32_t* d_code, const uint8_t* d_len, uint8_t* d_out, uint64_t out_cap,
                          uint64_t* d_byte_off, uint64_t* d_block_bits, void* stream);

/* Move-to-front encoding of a batch (Section 3.3): for every block a list of
 * the 256 byte values starts in ascending order; every byte is replaced by
 * its position in the list and then moved to the front.
 *   d_in   device, uint8[offsets[num_blocks]]; d_out: the same size (the
 *          positions). Uses the plan's first-sort tiles as chunks, plus about
 *          0.13 bytes per byte of max_total_bytes allocated on the first call. */
bwt_status bwt_mtf_encode(bwt_plan* plan, const uint8_t* d_in, const uint64_t* offsets, uint32_t num_blocks,
                          uint8_t* d_out, void* stream);

/* Free the plan and all its device and host memory. NULL is accepted. */
bwt_status bwt_plan_destroy(bwt_plan* plan);

/* ---- plan control and introspection (no paper counterpart) ----------- */

/* Status of the last call on this plan. For an asynchronous
 * bwt_forward_batch this waits until the call's work has finished on the GPU
 * (immediately, if the caller has synchronised) and returns its device-side
 * status: BWT_OK, BWT_ETIMEOUT, BWT_ECAPACITY or BWT_EINVAL. */
bwt_status bwt_plan_last_status(const bwt_plan* plan);

/* Copies the statistics of the last call into *out (waiting for an
 * asynchronous bwt_forward_batch to finish, as bwt_plan_last_status does). */
bwt_status bwt_plan_stats(const bwt_plan* plan, bwt_stats* out);

/* Changes the first sort's digit width (8, 11 or 16) and tile size (1024,
 * 2048, 4096) used by later calls; drops any cached graph. Choosing 16 the
 * first time allocates its scratch (BWT_ENOMEM if that fails; the plan keeps
 * its old width). With BWT_F_LEARNED, blocks routed to the plain sort take
 * 8-bit passes when the width is 16. */
bwt_status bwt_plan_set_radix(bwt_plan* plan, int radix_bits, int tile_keys);

/* Digit width (8, 10 or 11) of the segmented radix that sorts large groups
 * in the prefix-doubling rounds; 0 (the default) picks by the batch's rank
 * width: 10 when that takes fewer passes than 8 (ranks of 9-10, 17-20 or
 * 25-30 bits; blocks of 65,537 to 1,048,576 bytes have 17 to 20), else 8.
 * Drops any cached graph. Returns BWT_EINVAL for any other width. */
bwt_status bwt_plan_set_round_radix(bwt_plan* plan, int radix_bits);

/* Autotuner (no paper counterpart): times this batch for radix_bits in
 * {8, 11, 16} x tile_keys in {1024, 2048, 4096} (16 is skipped when its
 * scratch cannot be allocated), then for the rounds' digit width
 * in {8, 10, 11} (one untimed run, then `repeats` runs between CUDA events
 * on `stream`, for each candidate), keeps the fastest in the plan and
 * reports it through the out-pointers (any may be NULL). With cache_path,
 * the result is appended to that JSON-lines file under (GPU name, workload
 * signature = block count, total bytes, largest block, plan flags) and a
 * later call with the same signature reads it back instead of sweeping.
 * Arguments as for bwt_forward_batch; d_L and d_primary receive the output
 * of a final run with the chosen configuration (bwt_plan_stats describes it). */
bwt_status bwt_plan_autotune(bwt_plan* plan, const uint8_t* d_in, const uint64_t* offsets, uint32_t num_blocks,
                             uint8_t* d_L, int32_t* d_primary, void* stream, const char* cache_path, int repeats,
                             int* out_radix_bits, int* out_tile_keys, float* out_ms);

/* Test knob for the bounded device waits: `spin_limit` caps every wait loop
 * (0 = the built-in default of about one second); `withhold_publish` = 1 makes
 * the first tile of every radix pass, and of every single-pass scan of the
 * later stages (run-length encoding and decoding, variable-length encoding),
 * skip publishing its counts, so the look-back waits behind it run out and
 * the call reports BWT_ETIMEOUT. The GPU is never left waiting: each wait
 * gives up after `spin_limit` polls, and every index derived from a prefix
 * that gave up stays inside its buffer. */
bwt_status bwt_plan_debug_waits(bwt_plan* plan, uint32_t spin_limit, int withhold_publish);

/* ---- learned CDF model (the learned bucketing of BWT_F_LEARNED) -------
 *
 * The model approximates the CDF of rotation prefixes: input x = the 8
 * prefix bytes of a rotation, each normalised through the byte-value table
 * norm[256] (the CDF of byte values in the training data, midpoint rule:
 * norm[b] = (#bytes < b + #bytes == b / 2) / #bytes), target t = the
 * rotation's sorted row / n. It is an FP32 MLP 8 -> 32 -> 32 -> 1 with ReLU
 * after both hidden layers; its BWT_MLP_NPARAMS parameters are laid out
 * row-major as W1[32][8] | b1[32] | W2[32][32] | b2[32] | W3[32] | b3.
 * The loss of a batch of B samples is mean over samples of (y - t)^2.
 * A trained model is compiled into BWT_SPLITTERS sorted u64 splitters;
 * rotation key K (the 8-byte prefix, big-endian) goes to bucket
 * #{j : splitter[j] <= K}, one of BWT_BUCKETS. Because the bucket is a
 * monotone function of K, any sorted splitter table gives the exact
 * transform; the model only decides how even the buckets are. */
#define BWT_MLP_NPARAMS 1377
#define BWT_SPLITTERS 4095
#define BWT_BUCKETS 4096

/* y[s] = f(x[s]) for s < count. d_params: float[BWT_MLP_NPARAMS];
 * d_x: float[count][8]; d_y: float[count]. Device pointers, async. */
bwt_status bwt_mlp_forward(const float* d_params, const float* d_x, uint32_t count, float* d_y, void* stream);

/* Gradient of the batch loss with respect to every parameter (d_grad:
 * float[BWT_MLP_NPARAMS]) and the loss itself (d_loss: float[1], may be
 * NULL), over samples (d_x[s], d_t[s]), s < count. Deterministic reduction
 * order. Synchronises `stream`; allocates temporary device memory. */
bwt_status bwt_mlp_loss_grad(const float* d_params, const float* d_x, const float* d_t, uint32_t count,
                             float* d_grad, float* d_loss, void* stream);

/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8; Kingma and Ba 2015) at
 * step >= 1, in place on d_params, d_m, d_v (all float[BWT_MLP_NPARAMS]). */
bwt_status bwt_mlp_adam_step(float* d_params, const float* d_grad, float* d_m, float* d_v, uint32_t step, float lr,
                             void* stream);

/* Trains d_params in place with Adam over `epochs` passes of minibatches of
 * `batch` samples; epoch e visits samples d_order[e * count + 0 .. count - 1]
 * (a permutation supplied by the caller, so training is reproducible).
 * d_epoch_loss: float[epochs] mean batch loss per epoch (may be NULL).
 * Synchronises `stream`; allocates temporary device memory. */
bwt_status bwt_model_train(float* d_params, const float* d_x, const float* d_t, uint32_t count,
                           const uint32_t* d_order, uint32_t epochs, uint32_t batch, float lr, float* d_epoch_loss,
                           void* stream);

/* The byte-value normalisation table of n bytes of training data (device
 * pointers; d_norm: float[256]). Allocates and frees a temporary buffer. */
bwt_status bwt_model_byte_norm(const uint8_t* d_in, uint64_t n, float* d_norm, void* stream);

/* Training samples produced by the plain sorter: sorts the batch with the
 * plain path of `plan`, then for every s < count takes the row at global
 * sorted position d_pos[s] (< total bytes) and writes d_x[s] = the 8 prefix
 * bytes of that row's rotation mapped through d_norm and d_t[s] = its row
 * within its block / block size. Synchronises `stream`. */
bwt_status bwt_model_samples(bwt_plan* plan, const uint8_t* d_in, const uint64_t* offsets, uint32_t num_blocks,
                             const uint64_t* d_pos, uint32_t count, const float* d_norm, float* d_x, float* d_t,
                             void* stream);

/* Compiles trained parameters into BWT_SPLITTERS sorted splitters
 * (d_splitters, device u64): splitter j is found by bisection over the 64-bit
 * key space as the smallest key whose model output (bytes mapped through
 * d_norm) reaches (j + 1) / BWT_BUCKETS; the table is then sorted and every
 * run of equal splitters is spread evenly up to the next distinct one. */
bwt_status bwt_model_compile(const float* d_params, const float* d_norm, uint64_t* d_splitters, void* stream);

/* Installs a sorted splitter table (host or device memory, BWT_SPLITTERS
 * entries) in the plan; BWT_EINVAL if it is not non-decreasing. */
bwt_status bwt_plan_set_splitters(bwt_plan* plan, const uint64_t* splitters);

/* Model files: parameters, byte normalisation and compiled splitters (host
 * arrays). The file is an 8-byte tag "BWTMDL02", then BWT_MLP_NPARAMS
 * little-endian floats, 256 floats of norm, then BWT_SPLITTERS little-endian
 * u64. load returns BWT_ENOMODEL if the file is missing or malformed. */
bwt_status bwt_model_save(const char* path, const float* params, const float* norm, const uint64_t* splitters);
bwt_status bwt_model_load(const char* path, float* params, float* norm, uint64_t* splitters);

/* ---- forward BWT of one small block without device allocation --------
 *
 * The paper has no counterpart to this entry point. It is for callers that
 * cannot allocate device memory -- for instance a host framework that owns
 * the GPU's memory through its own pool and forbids allocations outside it,
 * or a latency-bound pipeline that cannot take the device synchronisation of
 * cudaMalloc / cudaFree -- and therefore cannot create a bwt_plan.
 *
 * It computes the same L and primary index as bwt_forward_batch for one
 * block of n bytes, 1 <= n <= BWT_NOALLOC_MAX_BYTES, with one CTA on the
 * current device and the caller's `stream`; it allocates nothing and does
 * not synchronise. Its scratch is a fixed array of 5 * BWT_NOALLOC_MAX_BYTES
 * u32 words (1.25 MiB) that lives in the library's device image: every GPU
 * that loads the library holds it until the process exits. Every call looks
 * up that array's device address on the current device (cudaGetSymbolAddress,
 * a host-side query); the first call on a device also loads the library's
 * device code there, so make that first call before any stream capture.
 *   d_in       device, uint8[n]: the block.
 *   d_L        device, uint8[n]: its L column.
 *   d_primary  device, int32[1]: its primary index.
 * No two of the three buffers may share a byte. Returns BWT_ETOOBIG if
 * n > BWT_NOALLOC_MAX_BYTES, BWT_EINVAL for n = 0, NULL or overlapping
 * buffers, BWT_ECUDA if the lookup or the launch fails. All calls share the one
 * scratch array, so calls whose kernels overlap on the GPU (other streams,
 * other host threads on the same device) race and give wrong results;
 * serialise them, e.g. on one stream. Each call writes every scratch word it
 * reads, so earlier calls' contents do no harm. */
#define BWT_NOALLOC_MAX_BYTES 65536
bwt_status bwt_forward_block_noalloc(const uint8_t* d_in, uint32_t n, uint8_t* d_L, int32_t* d_primary,
                                     void* stream);

/* Human-readable name of a status code (static string). */
const char* bwt_status_string(bwt_status s);

/* Text of the last CUDA error seen by any call in this process (static). */
const char* bwt_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BWT_GB300_H */
