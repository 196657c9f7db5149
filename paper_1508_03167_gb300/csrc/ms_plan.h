// ms_plan.h -- host-side plan of one MergeShuffle call and the launch interface between the
// API translation unit and the kernel translation units. Pure host C++ (no device code).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace msk {

constexpr uint32_t kMaxB = 4096u;             // largest cutoff (base block <= B+1 elements)
constexpr uint32_t kMaxFuse = 9u;             // at most 2^9 base blocks per tile
constexpr uint32_t kMaxTileMerges = 256u;     // 2^(kMaxFuse-1)
constexpr uint32_t kChunk = 4096u;            // coin steps per HBM chunk (32 Philox blocks)
constexpr uint32_t kDefaultTileBytes = 48u * 1024u;
constexpr uint32_t kLocalSpanBytes = 32u * 1024u;  // staging of a local-mode merge level
constexpr uint32_t kLocalMaxMergesLog = 4u;        // at most 16 merges per local CTA
constexpr uint32_t kWarpMergeMax = 4096u;           // largest merge a single warp finishes
constexpr uint32_t kWarpSpanMax = 8192u;            // elements of a warp's span of merges
constexpr uint32_t kSmemLimit = 200u * 1024u; // dynamic shared memory budget of one CTA
constexpr uint32_t kSpanBytes = 32u * 1024u;  // span buffer of the streamed small-merge levels
constexpr uint32_t kSpanMaxMerges = 64u;      // merges per span at most
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kTileMaxDepth = 6u;        // tile kernel: at most 2^6 base blocks a tile
constexpr uint64_t kPairParityBytes = 1ull << 28;  // arrays from which a shuffle fixes its pass
                                                   // parity with a fused pair of levels
constexpr uint32_t kXBlock = 1024u;       // positions per block of a pair's exception rank index
constexpr uint32_t kXTileBlocks = 128u;   // blocks per tile of that index (one CTA counts one)

// Kernel classes timed by the optional profiler (MS_FLAG_PROFILE).
enum KernelKind : int {
  kKindLeaf = 0,
  kKindCount,
  kKindScan,
  kKindKscan,
  kKindHashClear,
  kKindInsert,
  kKindResolve,
  kKindGather,
  kKindTailSeq,
  kKindPatchRead,
  kKindPatchWrite,
  kKindLocal,
  kKindEngine,
  kKindPairGather,
  kKindExceptions,
  kKindNum
};

// Records a CUDA event pair around each launch when profiling is on (null = off).
struct Prof {
  virtual void begin(int kind, cudaStream_t s) = 0;
  virtual void end(cudaStream_t s) = 0;
  virtual ~Prof() = default;
};

// One HBM merge level (levels d..c-1).
struct LevelPlan {
  uint32_t level;  // l
  uint32_t M;      // merges: q >> (l+1)
  uint32_t Nmax;   // largest merge: ceil(n * 2^(l+1) / q)
  uint32_t J;      // chunks of kChunk steps per merge
  uint32_t kcap;   // capacity for tail steps summed over the level's merges
  uint32_t hbits;  // hash table of 2^hbits slots
  // local modes: every merge finishes inside one CTA or warp, 2^mlog merges at a time
  bool local;             // any of the three local modes below (else the global plan)
  bool warp_local;        // one warp per group of merges, global to global (ms_wlevel.cu)
  bool span;              // streamed spans with asynchronous prefetch (ms_span.cu)
                          // (local and neither: one CTA per span staged in shared memory)
  uint32_t span_threads;  // span mode: 128 or 256 threads a CTA
  uint32_t warp_bytes;    // warp mode: shared memory of one warp
  uint32_t mlog;
  uint32_t span_max;      // elements of the largest span (span mode: the span buffer)
  uint32_t ucap, tcap;    // coin words and precomputed tail draws a span or warp holds
  size_t smem;            // dynamic shared memory a CTA (span and CTA modes)
  // global levels fused in pairs: 1 = first level of a pair (its tail moves become exceptions
  // of the pair's single data pass), 2 = second level of a pair, 0 = unpaired
  uint32_t pair;
  uint32_t xcap;    // a pair's first level: entries of its exception lists (2 kcap), else 0
  uint32_t lcap;    // literal merge (MS_FLAG_LITERAL): laps cached per merge
};

struct Plan {
  uint64_t n = 0;
  uint32_t w = 0;
  uint32_t B = 0;
  uint32_t c = 0;
  uint64_t q = 0;
  uint32_t d = 0;            // fused levels
  uint64_t tiles = 0;
  uint32_t tile_max = 0;     // elements
  uint32_t leaf_max = 0;     // largest base block: ceil(n / q)
  uint32_t leaf_stride = 0;  // odd shared-memory stride of one base block (>= leaf_max)
  uint32_t buf0_elems = 0;   // first tile buffer: max(2^d * leaf_stride, tile_max)
  uint32_t dw = 0;           // fused levels done by single warps (the rest, d - dw <= 3, by the CTA)
  uint32_t ucap_w = 0, tcap_w = 0, ucap_c = 0, tcap_c = 0;  // per-group coin-word / draw capacity
  uint32_t aux_w = 0;        // bytes of one warp's auxiliary shared-memory region
  uint32_t fy_per_cta = 0;   // d = 0: base blocks per one-warp CTA of the Fisher-Yates kernel
  size_t leaf_smem = 0;      // dynamic shared memory of the base-block kernel
  // eight-warp tile kernel (ms_tile.cu) for the base blocks and levels 0..d-1, if it fits:
  // block stride of its Fisher-Yates layout, 16-bit entries of each of its two buffers, coin
  // words and tail draws of one level, output stride of one merge of level l, shared memory
  bool tile_mode = false;
  uint32_t tile_P = 0, tile_buf = 0, tile_wcap = 0, tile_tcap = 0;
  uint32_t tile_S[kTileMaxDepth] = {};
  size_t tile_smem = 0;
  uint32_t nlevels = 0;      // HBM levels
  LevelPlan levels[33];
  uint32_t flags = 0;
  Prof *prof = nullptr;
  // workspace layout (byte offsets from the workspace base). The plan scratch of the global
  // levels comes in plan_sets copies, plan_set_bytes apart: level j of the global levels uses
  // set j % plan_sets, so the plan of the next level can be built while this one streams.
  size_t off_buf = 0, off_zc = 0, off_minfo = 0, off_ctrl = 0, off_mv = 0, off_hkeys = 0,
         off_hvals = 0, off_pdst = 0, off_psrc = 0, off_ptmp = 0, off_ostart = 0, ws_bytes = 0;
  size_t plan_set_bytes = 0;
  uint32_t plan_sets = 0;
  // exception structures of a pair's first level (offsets within one copy; one copy per two
  // plan sets): per-block zero counts (one byte per 128 coins), the exception bitmap (one bit
  // per element), the input index of each tail patch's element (by patch), the same indices in
  // position order (by rank), the rank index (exceptions before every 1024 positions within
  // their tile of 2^17 positions, and before every tile), and, for every chunk of the pair's
  // second level, the record of the two ranges it reads (2 x 16 words)
  size_t off_zb = 0, off_xbits = 0, off_xsrc = 0, off_xval = 0, off_xbpre = 0, off_xtpre = 0;
  size_t off_xrange = 0;
  size_t exc_base = 0, exc_bytes = 0;
  // literal merge (MS_FLAG_LITERAL): per merge, the first step of each lap of the first half's
  // rotating queue and the zero coins before it (uint2), lcap entries a merge; and per coin word
  // of a level, the word and the zeros of its chunk's earlier words (uint2) (same copies)
  size_t off_laps = 0, off_ctab = 0;
  // balanced-word merge (MS_FLAG_BALANCED): one label byte per element and the chunk zero counts
  // of the labels (same copies)
  size_t off_labels = 0, off_zlab = 0;
  uint32_t units = 0;         // global-level units: single levels and fused pairs
  uint32_t hbm_passes = 0;    // data passes after the base-block pass
  uint32_t zc_cap = 0, minfo_cap = 0, kcap_max = 0, hbits_max = 0;
};

// Builds the plan; returns 0 on success, 1 for invalid arguments, 2 for unsupported ones.
int make_plan(uint64_t n, uint32_t w, uint32_t B, int32_t fuse_depth, uint32_t tile_bytes,
              uint32_t flags, Plan *out);

// Device pointers of one call, derived from the plan and the caller's buffers.
struct Buffers {
  void *data;       // caller's array (result lands here)
  void *other;      // ping-pong partner
  uint8_t *zb;
  uint32_t *xbits;
  uint32_t *xsrc;
  uint32_t *xval;
  uint32_t *xbpre;
  uint32_t *xtpre;
  uint4 *xrange;
  uint32_t *zc;
  uint4 *minfo;
  uint32_t *ctrl;
  uint32_t *mv;
  unsigned long long *hkeys;
  uint32_t *hvals;
  uint32_t *pdst;
  uint32_t *psrc;
  void *ptmp;
  uint32_t *ostart;  // first merge of every 1024 tail steps of a level (kscan), + one sentinel
  uint2 *laps;       // literal merge: lap table (see Plan::off_laps)
  uint2 *ctab;       // literal merge: coin word table of a level (see Plan::off_ctab)
  uint8_t *labels;   // balanced-word merge: label bytes of a level
  uint32_t *zlab;    // balanced-word merge: zeros before each chunk of labels
};

// 1- and 2-byte elements (w): tmp[i] = data[idx[i]] for i < n (ms_narrow.cu).
cudaError_t launch_narrow_gather(const void *data, const uint32_t *idx, void *tmp, uint64_t n,
                                 uint32_t w, int sms, cudaStream_t s);

// Lets `kern` launch with `smem` bytes of dynamic shared memory. The attribute is process-wide,
// so every caller sets the same value (the device's opt-in maximum less the kernel's static
// shared memory): threads launching the same kernel with different sizes never lower it under
// each other. The launch's own size still decides the occupancy.
template <typename K>
cudaError_t allow_dynamic_smem(K kern, size_t smem) {
  int dev = 0, mx = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  // the kernel's static shared memory comes out of the same opt-in budget
  const size_t room = static_cast<size_t>(mx) > fa.sharedSizeBytes
                          ? static_cast<size_t>(mx) - fa.sharedSizeBytes
                          : 0;
  if (smem > room) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(room));
}

// Kernel launchers (ms_leaf.cu, ms_level.cu). Return the launch error (cudaSuccess if none).
cudaError_t launch_leaf(const Plan &p, const void *in, void *out, bool perm, uint64_t seed,
                        cudaStream_t s);
// The eight-warp tile kernel (ms_tile.cu): base blocks and levels 0..d-1; out of place unless perm.
cudaError_t launch_tile(const Plan &p, const void *in, void *out, bool perm, uint64_t seed,
                        cudaStream_t s);
// A global level in two parts: the data-independent plan (coin counts, prefixes, break steps,
// tail draws and their replay on indices) and the data pass (streaming gather, tail patches).
cudaError_t launch_level_plan(const Plan &p, const LevelPlan &lv, const Buffers &b, uint64_t seed,
                              cudaStream_t s);
// The break step T (and Z_T, N - T) of every merge of one level into b.minfo (count + scan only:
// the random-bit accounting of ms_bits.cu).
cudaError_t launch_level_breaks(const Plan &p, const LevelPlan &lv, const Buffers &b,
                                uint64_t seed, cudaStream_t s);
cudaError_t launch_level_data(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                              const Buffers &b, uint64_t seed, cudaStream_t s);
// Two consecutive global levels fused into one data pass (b1: the first level's plan set, with
// its exception structures; b2: the second's). The plan builds both levels' plans and turns the
// first level's tail moves into exceptions; the data pass gathers the second level's output
// straight from the first level's input (unfused fallback, gated on the device, if the first
// level's tails overflowed its capacity).
cudaError_t launch_pair_plan(const Plan &p, const LevelPlan &lv1, const LevelPlan &lv2,
                             const Buffers &b1, const Buffers &b2, uint64_t seed, cudaStream_t s);
cudaError_t launch_pair_data(const Plan &p, const LevelPlan &lv1, const LevelPlan &lv2,
                             const void *in, void *out, const Buffers &b1, const Buffers &b2,
                             uint64_t seed, cudaStream_t s);
cudaError_t launch_local_level(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                               uint64_t seed, cudaStream_t s);
cudaError_t launch_warp_level(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                              uint64_t seed, cudaStream_t s);
cudaError_t launch_span_level(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                              uint64_t seed, cudaStream_t s);
size_t span_smem_bytes(uint32_t S, uint32_t w, uint32_t ucap, uint32_t tcap);
// Batch engine (ms_batch.cu): one persistent launch over a device table of instances.
cudaError_t launch_engine(uint32_t w, bool perm, const void *inst, uint32_t k, uint32_t *queue,
                          uint32_t B, void *scratch, size_t scratch_per_cta, uint32_t kcap,
                          uint32_t hbits, uint32_t grid, size_t smem, cudaStream_t s, Prof *prof);
size_t engine_inst_bytes();
constexpr uint64_t kEngineMaxN = 1ull << 22;   // largest instance the batch engine takes
constexpr uint32_t kEngineKcap = 8192;         // tail steps per merge replayed in parallel
constexpr uint32_t kEngineHbits = 14;          // hash slots per engine CTA
constexpr size_t kEngineSmem = 96 * 1024;      // dynamic shared memory of an engine CTA

}  // namespace msk
