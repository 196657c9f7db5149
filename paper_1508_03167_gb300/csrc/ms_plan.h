// ms_plan.h -- host-side plan of one MergeShuffle call and the launch interface between the
// API translation unit and the kernel translation units. Pure host C++ (no device code).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace msk {

constexpr uint32_t kMaxB = 4096u;             // largest cutoff (base block <= B+1 elements)
constexpr uint32_t kMaxFuse = 10u;            // at most 2^10 base blocks per tile
constexpr uint32_t kMaxTileMerges = 512u;     // 2^(kMaxFuse-1)
constexpr uint32_t kChunk = 4096u;            // coin steps per HBM chunk (32 Philox blocks)
constexpr uint32_t kDefaultTileBytes = 48u * 1024u;
constexpr uint32_t kSmemLimit = 200u * 1024u; // dynamic shared memory budget of one CTA
constexpr uint32_t kNone = 0xFFFFFFFFu;

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
  uint32_t unit_cap = 0;     // coin words per tile level (shared-memory arrays)
  size_t leaf_smem = 0;      // dynamic shared memory of the base-block kernel
  uint32_t nlevels = 0;      // HBM levels
  LevelPlan levels[33];
  uint32_t flags = 0;
  Prof *prof = nullptr;
  // workspace layout (byte offsets from the workspace base)
  size_t off_buf = 0, off_zc = 0, off_minfo = 0, off_ctrl = 0, off_mv = 0, off_hkeys = 0,
         off_hvals = 0, off_pdst = 0, off_psrc = 0, off_ptmp = 0, ws_bytes = 0;
  uint32_t zc_cap = 0, minfo_cap = 0, kcap_max = 0, hbits_max = 0;
  bool buffer_in_ws = true;  // false for the host form, where both buffers live in ws
};

// Builds the plan; returns 0 on success, 1 for invalid arguments, 2 for unsupported ones.
int make_plan(uint64_t n, uint32_t w, uint32_t B, int32_t fuse_depth, uint32_t tile_bytes,
              uint32_t flags, Plan *out);

// Device pointers of one call, derived from the plan and the caller's buffers.
struct Buffers {
  void *data;       // caller's array (result lands here)
  void *other;      // ping-pong partner
  uint32_t *zc;
  uint4 *minfo;
  uint32_t *ctrl;
  uint32_t *mv;
  unsigned long long *hkeys;
  uint32_t *hvals;
  uint32_t *pdst;
  uint32_t *psrc;
  void *ptmp;
};

// Kernel launchers (ms_leaf.cu, ms_level.cu). Return the launch error (cudaSuccess if none).
cudaError_t launch_leaf(const Plan &p, const void *in, void *out, bool perm, uint64_t seed,
                        cudaStream_t s);
cudaError_t launch_level(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                         const Buffers &b, uint64_t seed, cudaStream_t s);

}  // namespace msk
