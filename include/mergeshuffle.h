/*
 * mergeshuffle.h -- C ABI of the GB300 MergeShuffle library (libmergeshuffle.so).
 *
 * MergeShuffle (Bacher, Bodini, Hollender, Lumbroso, arXiv 1508.03167) permutes an array
 * uniformly at random: split it into q = 2^c base blocks, shuffle each block with Fisher-Yates
 * (Algorithm 1), then merge adjacent blocks level by level (Algorithm 2) with the random merge
 * of Algorithm 3 -- coins interleave the two halves until one runs out, and the leftovers are
 * placed by random insertion.
 *
 * Result definition ("MS-Philox v1"). The output is a pure function of (input, n, seed, B):
 *   - block split of the appendix listing: c = smallest integer with floor(n / 2^c) <= B,
 *     block i = [floor(n*i/2^c), floor(n*(i+1)/2^c));
 *   - merge r of level l joins blocks [2pr, 2pr+p) and [2pr+p, 2pr+2p), p = 2^l;
 *   - the merge interleaves the halves stably (coin t = 0: next unused element of the first half,
 *     1: of the second half) until a coin asks for an exhausted half at step T; the other half's
 *     remaining elements follow in order; then for i = T..N-1, swap positions i and m_i,
 *     m_i uniform in {0..i} (Algorithm 3's second loop);
 *   - coin t of merge (l, r) is bit t%32 of word (t/32)%4 of Philox4x32-10(counter =
 *     (t/128, r, 0x10000|l, 0), key = (lo32(seed), hi32(seed)));
 *   - a uniform draw in [0, R) for stream (tag, level, id, pos) takes b = ceil(log2 R) bits
 *     per attempt, floor(32/b) attempts per 32-bit word; word j is word pos%4 of
 *     Philox4x32-10((pos/4, id, tag<<16|level, j)); the first attempt below R is returned.
 *     Tags: 2 = merge tail (pos = position in the merged range), 3 = base-block Fisher-Yates
 *     (level 0, id = block index, pos = i of Algorithm 1).
 * The same definition is implemented independently by the CPU oracle of the test suite.
 * Changing B changes the result; the fusion depth, launch shape, stream and batching do not.
 *
 * Memory. The library never allocates device memory and never synchronises a stream unless
 * an entry point says so. The caller passes a device workspace of ms_workspace_bytes() bytes
 * (256-byte aligned); it holds the second ping-pong buffer of n*w bytes plus the plan scratch
 * of the merge levels (coin prefixes per 4096 steps, tail tables sized to the expected tails,
 * double-buffered so the next level is planned while one streams; fused level pairs add a
 * bitmap of n/8 bytes, exception lists and per-chunk range records). Total device footprint:
 * 2*n*w bytes + scratch (the scratch is about 0.4*n*w for 4-byte elements at n = 2^30).
 *
 * Streams. Each call enqueues on the caller's stream; the data-independent plan of the global
 * merge levels runs on a second stream at the caller's priority, paired with it (created on
 * first use, ordered with events) unless MS_FLAG_SINGLE_STREAM is set.
 *
 * Errors. Argument errors are returned synchronously. Launch failures return MS_ERR_CUDA
 * (the CUDA error is not cleared). Nothing traps on the device.
 */
#ifndef MERGESHUFFLE_H
#define MERGESHUFFLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MS_OK = 0,
  MS_ERR_INVALID = 1,     /* bad argument: n, w, B, pointer alignment, workspace too small */
  MS_ERR_UNSUPPORTED = 2, /* valid request this build does not handle (e.g. B > MS_MAX_B) */
  MS_ERR_NOMEM = 3,       /* a host-side staging allocation failed */
  MS_ERR_CUDA = 4,        /* a CUDA call or launch failed */
  MS_ERR_TIMEOUT = 5      /* reserved: no entry point returns it (no kernel of this library
                             waits on another CTA, a flag or a peer) */
} ms_status;

/* Largest cutoff B the shared-memory base-block kernel accepts. */
#define MS_MAX_B 4096u

/* cudaStream_t, passed as an opaque pointer (NULL = the legacy default stream). */
typedef void *ms_stream_t;

/* Flags (ms_params.flags). */
#define MS_FLAG_TAIL_SEQUENTIAL 0x1u /* merge tails: one thread per merge, in place (slow path;
                                        the result is identical) */
#define MS_FLAG_PROFILE 0x2u         /* time every kernel of the call with CUDA events on its
                                        stream; read with ms_profile_read */
#define MS_FLAG_GLOBAL_LEVELS 0x4u   /* run every HBM merge level through the global plan (no
                                        CTA-local levels; the result is identical) */
#define MS_FLAG_CTA_LEVELS 0x8u      /* small merge levels finish per CTA rather than per warp
                                        (the result is identical) */
#define MS_FLAG_PERM 0x10u           /* batch calls: fill every instance with its permutation of
                                        0..n_i-1 instead of shuffling it (w must be 4).
                                        ms_plan_info: describe the plan of ms_perm rather than
                                        ms_shuffle (ms_perm and ms_shuffle set or clear it
                                        themselves) */
#define MS_FLAG_WARP_LEVELS 0x40u    /* small merge levels run one warp per group of merges,
                                        global to global, instead of streamed spans (the
                                        result is identical) */
#define MS_FLAG_SINGLE_LEVELS 0x80u  /* one data pass per global merge level: no fusing of
                                        consecutive levels into one pass (the result is
                                        identical) */
#define MS_FLAG_PAIR_LEVELS 0x100u   /* fuse consecutive global levels into one data pass for
                                        every element width (by default only 16-byte elements,
                                        where the pass is bound by memory rather than by its
                                        instructions, and, for a shuffle of at least 2^28 bytes
                                        whose tile pass needs an odd number of passes after it,
                                        its last two global levels; the result is identical) */
#define MS_FLAG_CTA_TILES 0x200u     /* fused merge levels (fuse_depth > 0) run on the CTA-wide
                                        base-block kernel rather than the eight-warp tile kernel
                                        on 16-bit indices (the result is identical) */
#define MS_FLAG_LITERAL 0x400u       /* Algorithm 3 as printed: the in-place swapping merge, whose
                                        first-half elements leave in a rotated order (the
                                        result differs from the default stable interleave; same
                                        coins, break steps and insertions, so the same random
                                        bits). Single calls only (the batched form returns
                                        MS_ERR_UNSUPPORTED); runs every level through HBM
                                        (fuse_depth 0, one global pass per level). The oracle's
                                        literal mode gives the same permutation. */
#define MS_FLAG_FDR 0x800u           /* uniform draws (Algorithm 1's and the merge tails') by the
                                        Fast Dice Roller on each draw's own stream instead of
                                        rejection on ceil(log2 R)-bit slices: fewer random bits
                                        a draw, a different result ("MS-Philox-FDR", the
                                        oracle's FDR mode). ms_random_bits counts its bits.
                                        Single calls only (the batched form returns
                                        MS_ERR_UNSUPPORTED); runs with fuse_depth 0 and one
                                        global pass per level. */
#define MS_FLAG_BALANCED 0x1000u     /* every merge driven by a balanced word (the idea of the
                                        paper's Section 3): the halves' labels merged by the
                                        merge's own coins and insertions give a uniform word
                                        with exactly n1 zeros, and the data is interleaved
                                        stably by it, so no insertion moves an element (a
                                        different result, same random bits; the oracle's
                                        BALANCED mode). Not with MS_FLAG_LITERAL
                                        (MS_ERR_INVALID); single calls only; fuse_depth 0 and
                                        one global pass per level. */
#define MS_FLAG_SINGLE_STREAM 0x20u  /* enqueue every kernel on the caller's stream: no plan
                                        stream beside it (the result is identical). By default
                                        the data-independent plan of each global merge level
                                        runs on a second stream, at the caller's priority,
                                        paired with the caller's, one or two levels ahead; make
                                        the first call on a stream before capturing it into a
                                        CUDA graph */

typedef struct {
  uint32_t B;          /* cutoff: base blocks have at most B+1 elements (1 <= B <= MS_MAX_B);
                          0 = autotuned: taken from the tuning table (ms_resolve_params) */
  int32_t fuse_depth;  /* merge levels done in shared memory per tile; -1 = automatic */
  uint32_t flags;      /* MS_FLAG_* */
  uint32_t tile_bytes; /* shared-memory bytes per tile buffer for the automatic fusion depth;
                          0 = default (48 KiB) */
} ms_params;

/* The resolved execution plan of one call (informational; filled by ms_plan_info). */
typedef struct {
  uint64_t n;
  uint32_t w;
  uint32_t B;
  uint32_t c;            /* levels: q = 2^c base blocks */
  uint32_t fuse_depth;   /* d: levels 0..d-1 run in shared memory inside the base-block kernel */
  uint32_t hbm_levels;   /* c - d merge levels that stream through HBM */
  uint32_t passes;       /* HBM read+write passes over the array: 1 + hbm_levels (0 if n <= 1) */
  uint64_t tiles;        /* CTAs of the base-block kernel */
  uint64_t tile_max;     /* largest tile (elements) */
  size_t workspace_bytes;
  uint32_t kernel_launches; /* kernels this library launches for one call */
  uint32_t global_levels;   /* HBM levels that use the global plan and streaming gather; the
                               other hbm_levels - global_levels finish inside a CTA or a warp */
  uint32_t fused_pairs;     /* pairs of consecutive global levels sharing one data pass:
                               passes = 1 + hbm_levels - fused_pairs */
  uint32_t tile_smem;       /* dynamic shared memory of one CTA of the 16-bit tile kernel (the
                               base-block pass when fuse_depth > 0), bytes; 0 if that pass
                               runs another kernel */
} ms_plan;

/* Per-kernel-class timing accumulated over calls made with MS_FLAG_PROFILE. */
#define MS_PROFILE_KINDS 16
typedef struct {
  uint32_t kinds;                        /* number of valid entries */
  char names[MS_PROFILE_KINDS][24];      /* "leaf", "count", "scan", ..., "gather", ... */
  uint64_t launches[MS_PROFILE_KINDS];   /* launches recorded */
  double ms[MS_PROFILE_KINDS];           /* summed event-to-event milliseconds */
} ms_profile;

/*
 * Autotuner lookup. B = 0 in ms_params asks for the cutoff (and, where fuse_depth is -1 or the
 * level-mode flags are unset, the fusion depth and level mode) measured fastest for the call's
 * element width and size on a GB300. The paper leaves the cutoff open (its driver, Algorithm 2,
 * splits the array into 2^c nearly equal blocks, and the appendix listing takes the cutoff as a
 * parameter); B changes the result through c = min{c : floor(n / 2^c) <= B}, so the resolved
 * value is a pure function of (n, w, installed table) and a caller who needs to reproduce a
 * result records it.
 *   ms_tune_entry            one row: applies to calls of width w, single (batch = 0) or batched
 *                            (batch = 1), with ceil(log2 n) <= log2n_max (the smallest such
 *                            bucket wins; beyond every bucket the largest applies). For batched
 *                            calls n is the median instance size. B is a block size: a single
 *                            call of n > B resolves to B' = floor(n / 2^c) for the c whose
 *                            blocks are nearest to B by ratio (of the two around n / B), so
 *                            that its blocks stay near the measured size whatever n (a batch
 *                            keeps B itself). flags may hold
 *                            MS_FLAG_CTA_LEVELS, MS_FLAG_GLOBAL_LEVELS,
 *                            MS_FLAG_SINGLE_LEVELS and MS_FLAG_PAIR_LEVELS only.
 *   ms_resolve_params        replaces B = 0 in *inout by the table's choice for (n, w); other
 *                            fields are kept (fuse_depth only if it is not -1). MS_ERR_INVALID
 *                            for a bad w or a NULL pointer.
 *   ms_resolve_batch_params  the same for a batch of k sizes h_n (host array).
 *   ms_tune_install          replaces the process-wide table by a copy of count rows (count = 0:
 *                            back to the built-in table); MS_ERR_INVALID if a row is malformed.
 *                            Thread-safe; calls already resolved keep their parameters.
 *   ms_tune_table            copies up to cap rows of the current table to out (may be NULL) and
 *                            returns the number of rows.
 */
typedef struct {
  uint32_t w;
  uint32_t batch;
  uint32_t log2n_max;
  uint32_t B;
  int32_t fuse_depth;
  uint32_t flags;
} ms_tune_entry;
ms_status ms_resolve_params(uint64_t n, uint32_t w, ms_params *inout);
ms_status ms_resolve_batch_params(uint32_t k, const uint64_t *h_n, uint32_t w, ms_params *inout);
ms_status ms_tune_install(const ms_tune_entry *entries, uint32_t count);
uint32_t ms_tune_table(ms_tune_entry *out, uint32_t cap);

/* Default parameters: B = 1024, automatic fusion depth, no flags. */
void ms_default_params(ms_params *p);

/* Plan for (n, w, p); returns MS_ERR_INVALID / MS_ERR_UNSUPPORTED for bad arguments. */
ms_status ms_plan_info(uint64_t n, uint32_t w, const ms_params *p, ms_plan *out);

/* Workspace bytes ms_shuffle / ms_perm need for (n, w, p); 0 if the arguments are invalid. */
size_t ms_workspace_bytes(uint64_t n, uint32_t w, const ms_params *p);

/*
 * Permute d_data[0..n) in place, uniformly at random (Algorithm 2 of the paper), stream-ordered.
 *   d_data  device pointer to n elements of w bytes (w in {1, 2, 4, 8, 16}); w-byte aligned
 *           (16-byte aligned for w = 16). Elements are moved as opaque w-byte records. For
 *           w = 1 and 2 the call builds ms_perm's permutation for the same (n, seed, B) in the
 *           workspace (B = 0 resolves as for 4-byte elements), gathers the elements through it
 *           and copies them back: the same result, a 4-byte perm's time plus two passes.
 *   n       0 <= n <= 2^32 - 1 (the paper's 32-bit n); n <= 1 returns MS_OK and launches
 *           nothing.
 *   seed    64-bit key of every Philox stream.
 *   d_ws    device workspace of at least ms_workspace_bytes(n, w, p) bytes, 256-byte aligned;
 *           owned by the caller, contents ignored on entry, scratch on exit.
 *   p       parameters (NULL = ms_default_params).
 *   stream  CUDA stream; the call only enqueues work.
 */
ms_status ms_shuffle(void *d_data, uint64_t n, uint32_t w, uint64_t seed, void *d_ws,
                     size_t ws_bytes, const ms_params *p, ms_stream_t stream);

/*
 * Fill d_out[0..n) with a uniformly random permutation of 0..n-1 (the problem statement of the
 * paper's introduction): the result equals ms_shuffle applied to the identity with the same
 * (n, seed, B), but the first pass generates the identity instead of reading it.
 *   d_out   device pointer to n uint32 values, 4-byte aligned.
 *   Other arguments as for ms_shuffle with w = 4.
 */
ms_status ms_perm(uint32_t *d_out, uint64_t n, uint64_t seed, void *d_ws, size_t ws_bytes,
                  const ms_params *p, ms_stream_t stream);

/*
 * End-to-end form for callers whose data lives in host memory: copy h_data (n*w bytes; pinned
 * memory gives full copy bandwidth) into the device workspace, shuffle it there, copy it back,
 * and synchronise the stream before returning.
 *   d_ws   device workspace of at least ms_host_workspace_bytes(n, w, p) bytes (it holds both
 *          ping-pong buffers).
 */
size_t ms_host_workspace_bytes(uint64_t n, uint32_t w, const ms_params *p);
ms_status ms_shuffle_host(void *h_data, uint64_t n, uint32_t w, uint64_t seed, void *d_ws,
                          size_t ws_bytes, const ms_params *p, ms_stream_t stream);
ms_status ms_perm_host(uint32_t *h_out, uint64_t n, uint64_t seed, void *d_ws, size_t ws_bytes,
                       const ms_params *p, ms_stream_t stream);

/*
 * Batched form: k independent instances (the same w and B), instance i of n_i elements at device
 * pointer h_ptrs[i] (the pointer array itself lives in host memory), with seed h_seeds[i], or
 * base_seed + i when h_seeds is NULL. Each result equals the single call on that instance.
 *
 * Instances of at most 2^22 elements run in one persistent launch: every CTA takes whole
 * instances, largest first, from an atomic queue and finishes each alone (no CTA waits for
 * another). Larger instances (and those above 2^16 that are large against the batch's share
 * per CTA) run the single-instance path: one after another on the stream if there is one, else
 * forked onto up to four side streams that belong to the caller's stream (created on its first
 * batch with several such instances) and joined back into it before the call's work ends.
 * Nothing of the batch fails asynchronously, so there is no per-instance status array.
 *   ms_batch_workspace_bytes  device workspace for the batch (ping-pong buffers of the engine
 *                             instances, per-CTA scratch, the instance table, and one
 *                             single-instance workspace per side stream, sized for the largest
 *                             large instance).
 *   ms_batch_prepare          writes the instance table into d_ws (a host-to-device copy from
 *                             pageable memory; call it again whenever pointers, sizes or seeds
 *                             change).
 *   ms_batch_run              only enqueues kernels and memsets on the stream (so it can be
 *                             captured into a CUDA graph once prepared); arguments as for prepare.
 *   ms_shuffle_batch          prepare + run.
 * flags MS_FLAG_PERM: fill each instance with its permutation of 0..n_i-1 (w = 4).
 */
size_t ms_batch_workspace_bytes(uint32_t k, const uint64_t *h_n, uint32_t w, const ms_params *p);
ms_status ms_batch_prepare(uint32_t k, void *const *h_ptrs, const uint64_t *h_n, uint32_t w,
                           const uint64_t *h_seeds, uint64_t base_seed, void *d_ws,
                           size_t ws_bytes, const ms_params *p, ms_stream_t stream);
ms_status ms_batch_run(uint32_t k, void *const *h_ptrs, const uint64_t *h_n, uint32_t w,
                       const uint64_t *h_seeds, uint64_t base_seed, void *d_ws, size_t ws_bytes,
                       const ms_params *p, ms_stream_t stream);
ms_status ms_shuffle_batch(uint32_t k, void *const *h_ptrs, const uint64_t *h_n, uint32_t w,
                           const uint64_t *h_seeds, uint64_t base_seed, void *d_ws,
                           size_t ws_bytes, const ms_params *p, ms_stream_t stream);

/*
 * ms_perm_static -- ms_perm for callers that cannot allocate device memory.
 * (An addition of this library; the paper has no counterpart.)
 *
 * Some callers have device pointers for their own inputs and outputs but no way to obtain more
 * device memory: a plugin whose host application owns every device allocation, or code that runs
 * under a fixed device-memory budget with no allocator of its own. This entry point needs no
 * workspace argument: its scratch is a fixed MS_STATIC_SCRATCH_BYTES (16 MiB) array compiled
 * into the library, which every GPU that loads the library holds until the process exits.
 *   d_out   device pointer to n uint32 values (the caller's output), 4-byte aligned.
 *   n       at most MS_STATIC_MAX_N (2^21); larger n, or parameters whose plan needs more
 *           scratch than the array holds, return MS_ERR_UNSUPPORTED without touching the device.
 *   p, stream, seed  as for ms_perm; the result is identical to ms_perm's.
 * Set-up: the first call on each device looks up the array's device address (with that device
 * current) and caches it; make that first call before any stream capture.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library routine). All calls
 * on a device share the one array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU (different streams, or different host threads) race on it; serialise them.
 */
#define MS_STATIC_MAX_N (1ull << 21)
#define MS_STATIC_SCRATCH_BYTES (16ull << 20)
ms_status ms_perm_static(uint32_t *d_out, uint64_t n, uint64_t seed, const ms_params *p,
                         ms_stream_t stream);

/*
 * Random-bit accounting of ms_perm(n, seed) with parameters p (B = 0: autotuned, as ms_perm
 * resolves it): the random-bit model of Section 1 of arXiv 1508.03167, the count its Table 1
 * reports. Nothing is permuted; the counts follow from the coin and draw streams alone and
 * equal the CPU oracle's for the same (n, seed, B).
 *   h_out   host array of 8 uint64: [0] coin bits (T + 1 per merge: the coin that asks for an
 *           exhausted half is drawn and counted), [1] bits of Algorithm 1's draws, [2] bits of
 *           the merge tails' draws (a draw costs its tested slices times b = ceil(log2 R); with
 *           MS_FLAG_FDR in p->flags, the bits the Fast Dice Roller reads from its stream),
 *           [3] Algorithm 1's draws, [4] tail draws, [5] merges, [6] leftover positions
 *           (sum of N - T), [7] levels c.
 *   d_ws    device workspace of ms_random_bits_workspace(n, p) bytes, 256-byte aligned.
 * Enqueued on stream; the call waits for it (the counts are copied to the host).
 * Errors: MS_ERR_INVALID for bad arguments, MS_ERR_CUDA for a failed launch or copy.
 */
size_t ms_random_bits_workspace(uint64_t n, const ms_params *p);
ms_status ms_random_bits(uint64_t n, uint64_t seed, const ms_params *p, void *d_ws,
                         size_t ws_bytes, uint64_t *h_out, ms_stream_t stream);

/*
 * The Rao-Sandelius splitting process (the comparison workload of the paper: the introduction's
 * passage on splitting processes and the third row of Table 1), with a Fisher-Yates cutoff B.
 * Result definition "RS-Philox v1" (also implemented by the CPU oracle of the test suite):
 *   start with the segment [0, n); on split level l = 0, 1, ... every segment [s, e) with more
 *   than B elements takes the bit of each current position p -- bit p%32 of word (p/32)%4 of
 *   Philox4x32-10((p/128, 0, 4<<16 | l, 0)) -- and is split stably, bit 0 first; segments of at
 *   most B elements stay. Once none is above B, every segment [s, e) is shuffled by Algorithm 1
 *   with the uniform draws of stream (tag 5, level 0, id = s, pos = i) defined above.
 *   ms_rs_workspace_bytes  device workspace for (n, w, B): a second buffer of n*w bytes, the
 *                          bit counts of every planned level (n/128 + n/1024 bytes a level,
 *                          made at once before the first level) and of one more, two lists of active
 *                          segments (8 bytes each, at most n/(B+1)), 12 bytes of split data per
 *                          active segment and a bitmap of the segment starts (n/8 bytes);
 *                          0 for invalid arguments.
 *   ms_rs_shuffle          permute d_data[0..n) (w in {4, 8, 16}, w-byte aligned) in place;
 *                          1 <= B <= MS_MAX_B, n <= 2^32 - 1, d_ws 256-byte aligned.
 *   ms_rs_perm             fill d_out[0..n) with the permutation ms_rs_shuffle applies to the
 *                          identity (the first level generates it instead of reading it).
 * Each split level is one pass over the array. The planned number of levels (c + 1, made odd
 * by one more unless w = 4 and B <= 512, where the Fisher-Yates pass runs in place;
 * c = min{c : floor(n / 2^c) <= B}) leaves a segment above B only rarely for large B;
 * the call then synchronises the stream once to read whether one is left, and runs further
 * pairs of levels if so (at most 4096 levels: MS_ERR_UNSUPPORTED beyond). So unlike ms_shuffle
 * these calls wait for their stream and cannot be captured into a CUDA graph.
 * Errors: MS_ERR_INVALID for bad arguments, MS_ERR_UNSUPPORTED for B > MS_MAX_B, MS_ERR_CUDA for
 * a failed launch or copy.
 */
size_t ms_rs_workspace_bytes(uint64_t n, uint32_t w, uint32_t B);
ms_status ms_rs_shuffle(void *d_data, uint64_t n, uint32_t w, uint64_t seed, uint32_t B,
                        void *d_ws, size_t ws_bytes, ms_stream_t stream);
ms_status ms_rs_perm(uint32_t *d_out, uint64_t n, uint64_t seed, uint32_t B, void *d_ws,
                     size_t ws_bytes, ms_stream_t stream);

/*
 * Collect the timings of every launch recorded since the last reset (waits for the recorded
 * events; process-wide state, not thread-safe) and optionally reset the record.
 */
ms_status ms_profile_read(ms_profile *out, int reset);

/* Human-readable name of a status code (static storage). */
const char *ms_status_string(ms_status s);

/*
 * The CUDA error (a cudaError_t value, 0 = none) behind the calling thread's most recent
 * MS_ERR_CUDA from a single-call or batched entry point, and its description (static storage).
 * The library does not clear CUDA's own error state.
 */
int ms_last_cuda_error(void);
const char *ms_last_cuda_error_string(void);

/* Library version string (static storage). */
const char *ms_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MERGESHUFFLE_H */
