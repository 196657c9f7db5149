// ms_rs.cu -- the Rao-Sandelius splitting process on the GPU (arXiv 1508.03167, the
// introduction's passage on splitting processes and the third row of Table 1), with a
// Fisher-Yates cutoff B: the comparison workload of MergeShuffle.
//
// Result definition (RS-Philox v1, implemented independently by the CPU oracle of the tests):
//   start with the single segment [0, n); on split level l = 0, 1, ... every segment [s, e) with
//   more than B elements draws the bit of each current position p (bit p mod 32 of word
//   (p / 32) mod 4 of Philox((p / 128, 0, (4 << 16) | l, 0))) and is split stably, the elements
//   with bit 0 first; segments of at most B elements keep their place. Once no segment has more
//   than B elements, each segment [s, e) is shuffled by Algorithm 1 with the uniform draws of
//   stream (tag 5, level 0, id = s, pos = i).
//
// One split level is one streaming pass over the array (read n*w, write n*w):
//   count   zeros among the bits of every 128-position block and 4096-position chunk (Philox
//           only, no array traffic), then an exclusive scan of the chunk counts; the bits depend
//           only on the seed and the positions, so the planned levels' counts are made by one
//           launch and one scan before the first level;
//   split   per active segment its zero count z (from the prefix) and its children: a child
//           larger than B joins the next level's active list (an ordered compaction: count,
//           single-CTA scan, write), and a split point s + z is marked in the boundary bitmap;
//           the data pass then sends position p of an active segment to s + (Z_p - Z_s) if its
//           bit is 0, else to s + z + (p - s) - (Z_p - Z_s); every other position is copied.
//           One CTA takes one chunk (the hardware balances the chunks over the SMs); for
//           elements up to 8 bytes it copies the chunk's rows into shared memory (cp.async)
//           while it sets up the chunk's bits and segments.
// After the planned levels (c + 1; made odd, so that the last one writes the workspace buffer,
// unless the Fisher-Yates pass can run in place: 4-byte rows, B <= 512) the host reads whether
// a segment above B is left and runs further pairs of levels if so.
// The Fisher-Yates pass takes the final segments from the boundary bitmap in batches of 32 on
// eight-warp CTAs: all warps make the draws, one lane per segment runs its swap chain on 16-bit
// local indices in shared memory, and a warp per segment writes it through them.
#include <algorithm>

#include "mergeshuffle.h"
#include "ms_common.cuh"
#include "ms_device.cuh"
#include "ms_merge.cuh"
#include "ms_plan.h"

namespace msk {
namespace {

constexpr uint32_t kTagRsCoin = 4u;
constexpr uint32_t kTagRsLeaf = 5u;
constexpr uint32_t kRsChunk = 4096u;                 // positions per chunk (32 Philox blocks)
constexpr uint32_t kRsChunkBlocks = kRsChunk / 128u;
constexpr uint32_t kRsThreads = 256u;
constexpr uint32_t kRsScanThreads = 1024u;
constexpr uint32_t kRsSegCap = 512u;  // active segments of one chunk staged at a time

struct RsArgs {
  uint64_t n;
  uint2 key;
  uint32_t level;
  uint32_t B;
  uint32_t nchunks;
  uint32_t *zc;        // nchunks + 1: zeros per chunk, then their exclusive prefix (total last)
  uint8_t *zb;         // 32 per chunk: zeros per 128-position block
  const uint2 *act;    // active segments (s, e) of this level, sorted by s
  const uint32_t *act_n;
  uint2 *nxt;          // next level's active segments
  uint32_t *nxt_n;
  uint32_t *zseg;      // per active segment: zeros among its bits
  uint32_t *zs;        // per active segment: zeros before its first position (Z_s)
  uint32_t *cnt;       // per active segment: children above B, then their exclusive prefix
  uint32_t *bnd;       // boundary bitmap: bit p set iff a final segment starts at p
  uint32_t *tsum;      // scan scratch: one sum per tile of kRsScanTile values
  uint32_t *cfirst;    // per chunk: the first active segment that ends after the chunk's start
};

__device__ __forceinline__ uint4 rs_block(uint2 key, uint32_t level, uint32_t blk) {
  return philox10(make_uint4(blk, 0u, (kTagRsCoin << 16) | level, 0u), key);
}

// zeros among the bits of positions [128*blk, min(128*blk + 128, limit))
__device__ __forceinline__ uint32_t rs_block_zeros(const uint4 &c, uint64_t base, uint64_t limit) {
  if (base >= limit) return 0u;
  const uint32_t valid = static_cast<uint32_t>(limit - base < 128ull ? limit - base : 128ull);
  uint32_t z = 0;
  z += __popc(~c.x & low_mask(min(valid, 32u)));
  z += __popc(~c.y & low_mask(valid > 32u ? min(valid - 32u, 32u) : 0u));
  z += __popc(~c.z & low_mask(valid > 64u ? min(valid - 64u, 32u) : 0u));
  z += __popc(~c.w & low_mask(valid > 96u ? valid - 96u : 0u));
  return z;
}

// Z_p: zeros among the bits of positions [0, p), p <= n (after the chunk scan)
__device__ uint32_t rs_zeros_before(const RsArgs &a, uint64_t p) {
  const uint64_t chunk = p / kRsChunk;
  uint32_t Z = a.zc[chunk] - a.zc[0];
  if (chunk >= a.nchunks) return Z;
  const uint32_t blk_in = static_cast<uint32_t>((p / 128u) % kRsChunkBlocks);
  const uint8_t *zb = a.zb + chunk * kRsChunkBlocks;
  for (uint32_t b = 0; b < blk_in; ++b) Z += zb[b];
  const uint32_t q = static_cast<uint32_t>(p & 127u);
  if (q) {
    const uint4 c = rs_block(a.key, a.level, static_cast<uint32_t>(p / 128u));
    const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (uint32_t k = 0; k < 4u; ++k) {
      const uint32_t lo = 32u * k;
      if (q > lo) Z += __popc(~w[k] & low_mask(min(q - lo, 32u)));
    }
  }
  return Z;
}

// zeros per 128-block and per chunk: one warp per chunk, one lane per block
__global__ void __launch_bounds__(kRsThreads) rs_count_kernel(RsArgs a) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = gridDim.x * (kRsThreads / 32u);
  for (uint32_t ch = (blockIdx.x * kRsThreads + threadIdx.x) >> 5; ch < a.nchunks; ch += warps) {
    const uint32_t blk = ch * kRsChunkBlocks + lane;
    const uint4 c = rs_block(a.key, a.level, blk);
    const uint32_t z = rs_block_zeros(c, 128ull * blk, a.n);
    a.zb[blk] = static_cast<uint8_t>(z);
    const uint32_t tot = warp_sum(z);
    if (lane == 0) a.zc[ch] = tot;
  }
}

// the zero counts of every planned level at once (they depend on the seed and the positions
// only): one warp per (level, chunk), one lane per block; level l's chunk counts go to
// zca[l * (nchunks + 1) + chunk], with a zero after its last chunk, so that one exclusive scan
// over all levels gives each level's prefix relative to its first entry (uint32 arithmetic
// wraps consistently: a level's own prefixes stay below 2^32)
__global__ void __launch_bounds__(kRsThreads) rs_count_all_kernel(RsArgs a, uint32_t levels,
                                                                 uint32_t *zca, uint8_t *zba) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t f = (static_cast<uint64_t>(blockIdx.x) * kRsThreads + threadIdx.x) >> 5;
  if (f >= static_cast<uint64_t>(levels) * a.nchunks) return;
  const uint32_t l = static_cast<uint32_t>(f / a.nchunks);
  const uint32_t ch = static_cast<uint32_t>(f - static_cast<uint64_t>(l) * a.nchunks);
  const uint32_t blk = ch * kRsChunkBlocks + lane;
  const uint4 c = rs_block(a.key, l, blk);
  const uint32_t z = rs_block_zeros(c, 128ull * blk, a.n);
  zba[(static_cast<uint64_t>(l) * a.nchunks) * kRsChunkBlocks + blk] = static_cast<uint8_t>(z);
  const uint32_t tot = warp_sum(z);
  uint32_t *const zl = zca + static_cast<uint64_t>(l) * (a.nchunks + 1u);
  if (lane == 0) {
    zl[ch] = tot;
    if (ch == 0) zl[a.nchunks] = 0u;
  }
}

// In-place exclusive scan of v[0..count) by one CTA, the total stored at *total (may alias
// v + count). Each thread sums a contiguous run, then a CTA scan of the run sums.
__device__ void cta_exclusive_scan(uint32_t *v, uint32_t count, uint32_t *total) {
  __shared__ uint32_t scratch[33];
  const uint32_t per = (count + kRsScanThreads - 1u) / kRsScanThreads;
  const uint32_t lo = min(threadIdx.x * per, count);
  const uint32_t hi = min(lo + per, count);
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; ++i) s += v[i];
  uint32_t tot;
  uint32_t run = block_exclusive_scan(s, scratch, &tot);
  for (uint32_t i = lo; i < hi; ++i) {
    const uint32_t x = v[i];
    v[i] = run;
    run += x;
  }
  if (threadIdx.x == 0) *total = tot;
}

// Exclusive scan of v[0..count) over the whole grid, in three kernels: every CTA sums a tile of
// kRsScanTile values (tile_sums), one CTA scans the tile sums (the total goes to *total), then
// every CTA rescans its tile from its offset. count is *count_dev if given, else count_host.
constexpr uint32_t kRsScanTile = 16u * kRsThreads;

__device__ __forceinline__ uint32_t scan_count(const uint32_t *count_dev, uint32_t count_host) {
  return count_dev ? *count_dev : count_host;
}

__global__ void __launch_bounds__(kRsThreads) rs_scan_reduce_kernel(const uint32_t *v,
                                                                    const uint32_t *count_dev,
                                                                    uint32_t count_host,
                                                                    uint32_t *tile_sums) {
  __shared__ uint32_t red[kRsThreads / 32u];
  const uint32_t count = scan_count(count_dev, count_host);
  const uint32_t ntiles = (count + kRsScanTile - 1u) / kRsScanTile;
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    uint32_t sum = 0;
    for (uint32_t i = t * kRsScanTile + threadIdx.x; i < min((t + 1u) * kRsScanTile, count);
         i += kRsThreads)
      sum += v[i];
    sum = warp_sum(sum);
    if ((threadIdx.x & 31u) == 0u) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x < 32u) {
      uint32_t x = threadIdx.x < kRsThreads / 32u ? red[threadIdx.x] : 0u;
      x = warp_sum(x);
      if (threadIdx.x == 0u) tile_sums[t] = x;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kRsScanThreads) rs_scan_tiles_kernel(uint32_t *tile_sums,
                                                                       const uint32_t *count_dev,
                                                                       uint32_t count_host,
                                                                       uint32_t *total) {
  const uint32_t count = scan_count(count_dev, count_host);
  cta_exclusive_scan(tile_sums, (count + kRsScanTile - 1u) / kRsScanTile, total);
}

__global__ void __launch_bounds__(kRsThreads) rs_scan_down_kernel(uint32_t *v,
                                                                  const uint32_t *count_dev,
                                                                  uint32_t count_host,
                                                                  const uint32_t *tile_sums) {
  __shared__ uint32_t scratch[33];
  const uint32_t count = scan_count(count_dev, count_host);
  const uint32_t ntiles = (count + kRsScanTile - 1u) / kRsScanTile;
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // thread i takes the 16 consecutive values [16 i, 16 i + 16) of the tile
    const uint32_t lo = t * kRsScanTile + 16u * threadIdx.x;
    uint32_t x[16], sum = 0;
#pragma unroll
    for (uint32_t u = 0; u < 16u; ++u) {
      x[u] = lo + u < count ? v[lo + u] : 0u;
      sum += x[u];
    }
    uint32_t tot;
    uint32_t run = tile_sums[t] + block_exclusive_scan(sum, scratch, &tot);
#pragma unroll
    for (uint32_t u = 0; u < 16u; ++u) {
      if (lo + u < count) v[lo + u] = run;
      run += x[u];
    }
  }
}

// per active segment: its zeros, Z_s, its children above B; the split point joins the bitmap
__global__ void __launch_bounds__(kRsThreads) rs_children_kernel(RsArgs a) {
  const uint32_t na = *a.act_n;
  for (uint32_t k = blockIdx.x * kRsThreads + threadIdx.x; k < na; k += gridDim.x * kRsThreads) {
    const uint2 sg = a.act[k];
    const uint32_t Zs = rs_zeros_before(a, sg.x);
    const uint32_t z = rs_zeros_before(a, sg.y) - Zs;
    const uint32_t len = sg.y - sg.x;
    a.zs[k] = Zs;
    a.zseg[k] = z;
    a.cnt[k] = (z > a.B ? 1u : 0u) + (len - z > a.B ? 1u : 0u);
    if (z > 0u && z < len) {
      const uint32_t p = sg.x + z;
      atomicOr(&a.bnd[p >> 5], 1u << (p & 31u));
    }
  }
}

__global__ void __launch_bounds__(kRsThreads) rs_list_write_kernel(RsArgs a) {
  const uint32_t na = *a.act_n;
  for (uint32_t k = blockIdx.x * kRsThreads + threadIdx.x; k < na; k += gridDim.x * kRsThreads) {
    const uint2 sg = a.act[k];
    const uint32_t z = a.zseg[k];
    uint32_t o = a.cnt[k];
    if (z > a.B) a.nxt[o++] = make_uint2(sg.x, sg.x + z);
    if (sg.y - sg.x - z > a.B) a.nxt[o] = make_uint2(sg.x + z, sg.y);
  }
}

// per chunk: the first active segment that ends after the chunk's first position (one thread per
// chunk; the active segments are disjoint and sorted)
__global__ void __launch_bounds__(kRsThreads) rs_chunk_first_kernel(RsArgs a) {
  const uint32_t na = *a.act_n;
  for (uint32_t ch = blockIdx.x * kRsThreads + threadIdx.x; ch < a.nchunks;
       ch += gridDim.x * kRsThreads) {
    const uint64_t c0 = static_cast<uint64_t>(ch) * kRsChunk;
    uint32_t lo = 0, hi = na;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (a.act[mid].y <= c0) lo = mid + 1;
      else hi = mid;
    }
    a.cfirst[ch] = lo;
  }
}

// The data pass of one split level. A CTA takes a chunk of 4096 positions: warp 0 makes the
// chunk's bits and the zeros before each word, the active segments that overlap the chunk are
// staged in shared memory (in rounds of kRsSegCap), and every position goes to its place in its
// segment's split, or stays if no active segment holds it. Level 0 of a perm writes the
// positions themselves (nothing is read).
template <typename E, bool kPerm>
// (4-byte rows: eight CTAs an SM, 32 registers, as the shared memory allows)
__global__ void __launch_bounds__(kRsThreads, sizeof(E) == 4u ? 8 : (sizeof(E) == 8u ? 6 : 4))
    rs_split_kernel(RsArgs a, const E *in, E *out) {
  // elements up to 8 bytes: the chunk's rows are copied into shared memory (cp.async) while
  // the chunk's bits and segments are set up
  constexpr bool kStage = !kPerm && sizeof(E) <= 8u;
  __shared__ __align__(16) E sdata[kStage ? kRsChunk : 1u];
  __shared__ uint32_t cw[kRsChunk / 32u];
  __shared__ uint32_t zw[kRsChunk / 32u];
  __shared__ uint4 sg[kRsSegCap];  // (s, e, z, Z_s)
  __shared__ uint32_t s_first;
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint32_t na = *a.act_n;
  for (uint32_t ch = blockIdx.x; ch < a.nchunks; ch += gridDim.x) {
    const uint64_t c0 = static_cast<uint64_t>(ch) * kRsChunk;
    const uint64_t c1 = min(c0 + kRsChunk, a.n);
    if constexpr (kStage) {
      const uint32_t cnt = static_cast<uint32_t>(c1 - c0);
      const E *const src = in + c0;
      uint32_t i0 = 0;
      if ((reinterpret_cast<uintptr_t>(in) & 15u) == 0u) {
        constexpr uint32_t kPer = 16u / sizeof(E);
        const uint32_t nv = cnt / kPer;
        for (uint32_t i = tid; i < nv; i += kRsThreads)
          cp_async_elem(reinterpret_cast<uint4 *>(sdata) + i,
                        reinterpret_cast<const uint4 *>(src) + i);
        i0 = nv * kPer;
      }
      for (uint32_t i = i0 + tid; i < cnt; i += kRsThreads) cp_async_elem(sdata + i, src + i);
      cp_async_commit();
    }
    if (tid < 32u) {
      const uint4 c = rs_block(a.key, a.level, ch * kRsChunkBlocks + lane);
      cw[4u * lane + 0u] = c.x;
      cw[4u * lane + 1u] = c.y;
      cw[4u * lane + 2u] = c.z;
      cw[4u * lane + 3u] = c.w;
      const uint32_t z4 = __popc(~c.x) + __popc(~c.y) + __popc(~c.z) + __popc(~c.w);
      uint32_t ex = warp_inclusive_scan(z4) - z4;
      zw[4u * lane + 0u] = ex;
      ex += __popc(~c.x);
      zw[4u * lane + 1u] = ex;
      ex += __popc(~c.y);
      zw[4u * lane + 2u] = ex;
      ex += __popc(~c.z);
      zw[4u * lane + 3u] = ex;
    }
    if (tid == 0) s_first = a.cfirst[ch];
    __syncthreads();
    const uint32_t Zc = a.zc[ch] - a.zc[0];
    uint32_t k = s_first;
    uint64_t span_lo = c0;
    for (;;) {
      // stage the next round of segments that start before c1 (sorted: those form a prefix)
      uint32_t m = 0;
      for (uint32_t j0 = 0; j0 < kRsSegCap; j0 += kRsThreads) {
        const uint32_t j = j0 + tid;
        bool in_chunk = false;
        if (j < kRsSegCap && k + j < na) {
          const uint2 e = a.act[k + j];
          in_chunk = e.x < c1;
          // (s, e, A0 = s - Z_s, B1 = z + Z_s): bit 0 goes to A0 + Z_p, bit 1 to B1 + p - Z_p
          if (in_chunk) {
            const uint32_t Zs = a.zs[k + j];
            sg[j] = make_uint4(e.x, e.y, e.x - Zs, a.zseg[k + j] + Zs);
          }
        }
        if constexpr (kStage) cp_async_wait<0>();  // (the chunk's rows, before the barrier)
        const uint32_t got = static_cast<uint32_t>(__syncthreads_count(in_chunk));
        m += got;
        if (got < kRsThreads) break;  // (uniform: every thread sees the same count)
      }
      const bool last = (m < kRsSegCap) || (k + m >= na) || (a.act[k + m].x >= c1);
      const uint64_t span_hi = last ? c1 : min(static_cast<uint64_t>(sg[m - 1u].y), c1);
      // eight positions a thread per round (their loads in flight together), each to its place;
      // positions are 32-bit (n < 2^32), the thread's current segment is kept in registers
      constexpr uint32_t kU = 8u;
      const uint32_t lo32 = static_cast<uint32_t>(span_lo), hi32 = static_cast<uint32_t>(span_hi);
      const uint32_t cbase = static_cast<uint32_t>(c0);
      const uint32_t nlast = static_cast<uint32_t>(a.n - 1u);
      uint32_t j = 0;
      uint4 g = m ? sg[0] : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u);
      // (offsets from lo32 within the span stay below 4096: no 32-bit overflow near n = 2^32)
      const uint32_t span = hi32 - lo32;
      for (uint32_t o0 = tid; o0 < span; o0 += kU * kRsThreads) {
        const uint32_t p0 = lo32 + o0;
        E v[kU];
#pragma unroll
        for (uint32_t u = 0; u < kU; ++u) {
          const uint32_t p = p0 + u * kRsThreads;
          if (o0 + u * kRsThreads < span) {
            if constexpr (kPerm) v[u] = static_cast<E>(p);
            else if constexpr (kStage) v[u] = sdata[p - cbase];
            else v[u] = in[p];
          }
        }
#pragma unroll
        for (uint32_t u = 0; u < kU; ++u) {
          const uint32_t p = p0 + u * kRsThreads;
          if (o0 + u * kRsThreads >= span) break;
          while (g.y <= p && j < m) {
            ++j;
            g = j < m ? sg[j] : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u);
          }
          uint32_t dst = p;
          if (g.x <= p) {
            const uint32_t q = p - cbase;
            const uint32_t wv = cw[q >> 5];
            const uint32_t Zp = Zc + zw[q >> 5] + __popc(~wv & low_mask(q & 31u));
            dst = ((wv >> (q & 31u)) & 1u) ? g.w + p - Zp : g.z + Zp;
          }
          out[min(dst, nlast)] = v[u];
        }
      }
      if (last) break;
      k += m;
      span_lo = span_hi;
      __syncthreads();
    }
    __syncthreads();
  }
}

// Algorithm 1 on every final segment (at most B elements each; a segment starts at every set
// bit of the boundary bitmap and ends at the next one, or at n). CTAs of eight warps walk
// windows of kRsFyWinWords bitmap words; the eight warps read 256 of them at a time and add
// their segment starts, in order, to a shared list (all at once when they fit it). Each batch of `lanes` segments (segment k of the batch on lane k) then
// runs in three phases on 16-bit local indices in shared memory (stride P = 2 mod 64: the lanes'
// entries at one index sit in distinct banks):
//   draws   all eight warps (warp w: quads w, w + 8, ... of every segment) write the identity
//           and the draw of every position i >= 1 of stream (5, 0, s, i); a draw whose first
//           Philox word rejects every slice is queued by its thread and finished after the loop;
//   swaps   warp 0 runs each segment's chain i = L-1 .. 1 (one lane a segment), four steps
//           at a time: their eight reads together, values forwarded between the four in
//           registers, then their writes in the chain's order;
//   write   a warp per segment: out[s + i] = in[s + idx[i]], eight loads a lane in flight.
constexpr uint32_t kRsFyWinWords = 1024u;
constexpr uint32_t kRsFyInPlaceMax = 512u;  // largest final segment the in-place pass takes
constexpr uint32_t kRsFyWarps = 8u;
constexpr uint32_t kRsFyThreads = 32u * kRsFyWarps;
constexpr uint32_t kRsFyFail = 8u;  // queued second-word draws a thread

// One batch: the first kb starts of the list (cnt starts are waiting; the segment of start k
// ends at start k + 1, else at the next set bit of the bitmap).
template <typename E, bool kInPlace>
__device__ void rs_fy_batch(const E *in, E *out, uint64_t n, uint2 key, const uint32_t *bnd,
                            uint32_t P, const uint32_t *list, uint32_t kb, uint32_t cnt,
                            uint16_t *Abuf, uint16_t *Dbuf, uint16_t *F, uint32_t *sS,
                            uint32_t *sL) {
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint32_t warp = tid >> 5;
  if (warp == 0u && lane < kb) {
    const uint32_t s_pos = list[lane];
    uint64_t e = n;
    if (lane + 1u < cnt) {
      e = list[lane + 1u];
    } else {
      // the next start after s_pos in the bitmap (a later bit of its word, else a later word)
      const uint64_t nwords = (n + 31u) >> 5;
      const uint64_t w = static_cast<uint64_t>(s_pos) >> 5;
      uint32_t bw = bnd[w] & ~low_mask((s_pos & 31u) + 1u);
      uint64_t q = w;
      while (bw == 0u && ++q < nwords) bw = bnd[q];
      if (bw) e = (q << 5) + static_cast<uint32_t>(__ffs(static_cast<int>(bw)) - 1);
    }
    sS[lane] = s_pos;
    // (a final segment never exceeds B <= P - 2)
    const uint64_t len = min(e, n) - s_pos;
    sL[lane] = len < P - 2u ? static_cast<uint32_t>(len) : P - 2u;
  }
  __syncthreads();
  // draws
  if (lane < kb) {
    const uint32_t L = sL[lane], id = sS[lane];
    uint16_t *const A = Abuf + lane * P;
    uint16_t *const D = Dbuf + lane * P;
    uint16_t *const Fq = F + tid * kRsFyFail;
    const uint32_t nq = L ? ((L - 1u) >> 2) + 1u : 0u;
    uint32_t nf = 0;
#pragma unroll 2
    for (uint32_t qd = warp; qd < nq; qd += kRsFyWarps) {
      const uint4 blk = philox10(make_uint4(qd, id, kTagRsLeaf << 16, 0u), key);
      // slice width of the quad's ranges (positions 1..3 of quad 0 take the general draw)
      const uint32_t qb = 32u - __clz(4u * qd + 1u);
      const uint32_t qmask = 0xFFFFFFFFu >> (32u - qb);
#pragma unroll
      for (uint32_t v = 0; v < 4u; ++v) {
        const uint32_t pos = 4u * qd + v;
        if (pos < L) {
          A[pos] = static_cast<uint16_t>(pos);
          if (pos >= 1u) {
            uint32_t x;
            const uint32_t word = pick_word(blk, v);
            const bool ok = qd ? draw_first_word_b(word, pos + 1u, qb, qmask, 2u * qb, 3u * qb, x)
                               : draw_first_word(word, pos + 1u, x);
            if (ok) {
              D[pos] = static_cast<uint16_t>(x);
            } else if (nf < kRsFyFail) {
              Fq[nf++] = static_cast<uint16_t>(pos);
            } else {
              D[pos] = static_cast<uint16_t>(draw_continue(key, kTagRsLeaf, 0u, id, pos, pos + 1u));
            }
          }
        }
      }
    }
    // draws whose first word rejected every slice: words 1, 2, ... of their streams
    for (uint32_t e = 0; e < nf; ++e) {
      const uint32_t pos = Fq[e];
      D[pos] = static_cast<uint16_t>(draw_continue(key, kTagRsLeaf, 0u, id, pos, pos + 1u));
    }
  }
  __syncthreads();
  // swaps, i = L-1 .. 1, four steps a group (the draws clamped to the segment)
  if (warp == 0u && lane < kb) {
    const uint32_t L = sL[lane];
    uint16_t *const A = Abuf + lane * P;
    const uint16_t *const D = Dbuf + lane * P;
    fy_chain16(A, D, L);
  }
  __syncthreads();
  // the batch's rows through the indices, a warp per segment
  if constexpr (kInPlace) {
    // in place (4-byte rows, segments of at most 512 = 16 x 32 rows): the warp reads the whole
    // segment before it writes any of it back
    constexpr uint32_t kRowsAll = kRsFyInPlaceMax / 32u;
    for (uint32_t k = warp; k < kb; k += kRsFyWarps) {
      const uint32_t s_pos = sS[k], L = sL[k];
      const uint16_t *const A = Abuf + k * P;
      E v[kRowsAll];
#pragma unroll
      for (uint32_t u = 0; u < kRowsAll; ++u) {
        const uint32_t i = 32u * u + lane;
        if (i < L) v[u] = in[static_cast<uint64_t>(s_pos) + min(static_cast<uint32_t>(A[i]), L - 1u)];
      }
      __syncwarp();
#pragma unroll
      for (uint32_t u = 0; u < kRowsAll; ++u) {
        const uint32_t i = 32u * u + lane;
        if (i < L) out[static_cast<uint64_t>(s_pos) + i] = v[u];
      }
    }
    __syncthreads();
    return;
  }
  constexpr uint32_t kRows = sizeof(E) >= 16u ? 4u : 8u;
  for (uint32_t k = warp; k < kb; k += kRsFyWarps) {
    const uint32_t s_pos = sS[k], L = sL[k];
    const uint16_t *const A = Abuf + k * P;
    for (uint32_t i0 = 0; i0 < L; i0 += 32u * kRows) {
      E v[kRows];
#pragma unroll
      for (uint32_t u = 0; u < kRows; ++u) {
        const uint32_t i = i0 + 32u * u + lane;
        if (i < L) v[u] = in[static_cast<uint64_t>(s_pos) + min(static_cast<uint32_t>(A[i]), L - 1u)];
      }
#pragma unroll
      for (uint32_t u = 0; u < kRows; ++u) {
        const uint32_t i = i0 + 32u * u + lane;
        if (i < L) out[static_cast<uint64_t>(s_pos) + i] = v[u];
      }
    }
  }
  __syncthreads();
}

template <typename E, bool kInPlace>
__global__ void __launch_bounds__(kRsFyThreads, 3) rs_fy_kernel(const E *in, E *out, uint64_t n,
                                                            uint2 key, const uint32_t *bnd,
                                                            uint32_t P, uint32_t lanes) {
  extern __shared__ __align__(16) uint16_t fy_smem[];
  __shared__ uint32_t sS[32], sL[32], s_wt[kRsFyWarps];
  uint16_t *const Abuf = fy_smem;
  uint16_t *const Dbuf = fy_smem + lanes * P;
  uint32_t *const list = reinterpret_cast<uint32_t *>(fy_smem + ((2u * lanes * P + 1u) & ~1u));
  uint16_t *const F = reinterpret_cast<uint16_t *>(list + lanes + 32u * 32u + 32u);
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint32_t warp = tid >> 5;
  const uint64_t nwords = (n + 31u) >> 5;
  for (uint64_t w0 = static_cast<uint64_t>(blockIdx.x) * kRsFyWinWords; w0 < nwords;
       w0 += static_cast<uint64_t>(gridDim.x) * kRsFyWinWords) {
    uint32_t cnt = 0;  // starts waiting in the list (the same in every thread)
    for (uint32_t cw0 = 0; cw0 < kRsFyWinWords && w0 + cw0 < nwords; cw0 += 32u * kRsFyWarps) {
      // every warp reads one group of 32 bitmap words (eight reads in flight at once); groups
      // past the window or the array read as empty
      const uint64_t wi = w0 + cw0 + 32u * warp + lane;
      const uint32_t grp = (cw0 + 32u * warp < kRsFyWinWords && wi < nwords) ? bnd[wi] : 0u;
      const uint32_t c = static_cast<uint32_t>(__popc(grp));
      const uint32_t incl = warp_inclusive_scan(c);
      if (lane == 31u) s_wt[warp] = incl;
      __syncthreads();
      uint32_t base = 0, total = 0;
#pragma unroll
      for (uint32_t g = 0; g < kRsFyWarps; ++g) {
        const uint32_t t = s_wt[g];
        base += g < warp ? t : 0u;
        total += t;
      }
      // if the starts of all eight groups fit the list, every warp adds its group's starts at
      // once, behind the groups before it; otherwise (dense starts, small cutoffs) warp g adds
      // group g in round g
      const bool all = cnt + total <= lanes + 32u * 32u;
      const uint32_t rounds = all ? 1u : kRsFyWarps;
      for (uint32_t g = 0; g < rounds; ++g) {
        if (all || warp == g) {
          uint32_t word = grp;
          uint32_t pos = cnt + (all ? base : 0u) + incl - c;
          while (word) {
            list[pos++] = static_cast<uint32_t>(wi << 5) +
                          static_cast<uint32_t>(__ffs(static_cast<int>(word)) - 1);
            word &= word - 1u;
          }
        }
        __syncthreads();
        cnt += all ? total : s_wt[g];
        while (cnt > lanes) {  // (a full batch; the one after it supplies its last end)
          rs_fy_batch<E, kInPlace>(in, out, n, key, bnd, P, list, lanes, cnt, Abuf, Dbuf, F, sS, sL);
          if (warp == 0u) {
            for (uint32_t i = lane; i + lanes < cnt; i += 32u) {
              const uint32_t v = list[i + lanes];
              __syncwarp(__activemask());
              list[i] = v;
            }
          }
          __syncthreads();
          cnt -= lanes;
        }
      }
    }
    if (cnt) rs_fy_batch<E, kInPlace>(in, out, n, key, bnd, P, list, cnt, cnt, Abuf, Dbuf, F, sS,
                                     sL);
  }
}

__global__ void rs_init_kernel(RsArgs a, uint2 *act0, uint32_t *act0_n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    a.bnd[0] |= 1u;
    const bool split = a.n > a.B;
    if (split) act0[0] = make_uint2(0u, static_cast<uint32_t>(a.n));
    *act0_n = split ? 1u : 0u;
  }
}

}  // namespace
}  // namespace msk

namespace msk {
namespace {

__global__ void rs_iota_kernel(uint32_t *out, uint64_t n) {
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < n; i += gridDim.x * 256ull)
    out[i] = static_cast<uint32_t>(i);
}

size_t up256(size_t x) { return (x + 255u) & ~static_cast<size_t>(255u); }

// Workspace of one call: the ping-pong partner, the per-level bit counts, two active lists with
// their counts, the per-segment split data, and the boundary bitmap.
struct RsLayout {
  uint32_t nchunks = 0, maxact = 0;
  uint32_t plevels = 0;
  size_t buf = 0, zc = 0, zb = 0, zca = 0, zba = 0, act0 = 0, act1 = 0, ctl = 0, zseg = 0,
         zs = 0, cnt = 0, bnd = 0, tsum = 0, cfirst = 0, total = 0;
};

// whether the Fisher-Yates pass can run in place in the caller's buffer (4-byte rows, final
// segments of at most kRsFyInPlaceMax rows)
bool rs_fy_in_place(uint32_t w, uint32_t B) { return w == 4u && B <= kRsFyInPlaceMax; }

// planned split levels: c + 1 (segments then average at most B/2, so one above B is rare);
// unless the Fisher-Yates pass can run in place, made odd so that the last one writes the
// workspace buffer
uint32_t rs_planned_levels(uint64_t n, uint32_t w, uint32_t B) {
  if (n <= B) return 0u;
  uint32_t c = 0;
  while ((n >> c) > B) ++c;
  uint32_t levels = c + 1u;
  if (levels % 2u == 0u && !rs_fy_in_place(w, B)) ++levels;
  return levels;
}

RsLayout rs_layout(uint64_t n, uint32_t w, uint32_t B) {
  RsLayout L;
  L.nchunks = static_cast<uint32_t>((n + kRsChunk - 1u) / kRsChunk);
  L.maxact = static_cast<uint32_t>(n / (static_cast<uint64_t>(B) + 1u) + 2u);
  L.plevels = rs_planned_levels(n, w, B);
  const uint64_t nall = static_cast<uint64_t>(L.plevels) * (L.nchunks + 1ull);
  size_t off = 0;
  L.buf = off;
  off += up256(n * w);
  L.zc = off;
  off += up256((L.nchunks + 1ull) * 4u);
  L.zb = off;
  off += up256(static_cast<size_t>(L.nchunks) * kRsChunkBlocks);
  L.zca = off;
  off += up256(nall * 4u);
  L.zba = off;
  off += up256(static_cast<size_t>(L.plevels) * L.nchunks * kRsChunkBlocks);
  L.act0 = off;
  off += up256(L.maxact * 8ull);
  L.act1 = off;
  off += up256(L.maxact * 8ull);
  L.ctl = off;
  off += 256;
  L.zseg = off;
  off += up256(L.maxact * 4ull);
  L.zs = off;
  off += up256(L.maxact * 4ull);
  L.cnt = off;
  off += up256(L.maxact * 4ull);
  L.bnd = off;
  off += up256(((n + 31u) / 32u + 1u) * 4u);
  L.tsum = off;
  off += up256((std::max<uint64_t>(std::max<uint64_t>(L.maxact, L.nchunks), nall) / kRsScanTile +
                 2u) * 4u);
  L.cfirst = off;
  off += up256(L.nchunks * 4ull);
  L.total = off;
  return L;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

template <typename E>
cudaError_t rs_launch_split(const RsArgs &a, const void *in, void *out, bool perm, int sms,
                            cudaStream_t s) {
  // one CTA a chunk: the hardware balances the chunks over the SMs
  (void)sms;
  const unsigned grid = a.nchunks;
  if constexpr (sizeof(E) == 4) {
    if (perm) {
      rs_split_kernel<E, true><<<grid, kRsThreads, 0, s>>>(a, static_cast<const E *>(in),
                                                            static_cast<E *>(out));
      return cudaGetLastError();
    }
  }
  rs_split_kernel<E, false><<<grid, kRsThreads, 0, s>>>(a, static_cast<const E *>(in),
                                                         static_cast<E *>(out));
  return cudaGetLastError();
}

// one split level: bit counts and their scan (unless the planned levels' were made at once),
// the segments' splits and the next active list, then the data pass from `in` to `out`
cudaError_t rs_level(RsArgs a, uint32_t maxact, const void *in, void *out, uint32_t w,
                     bool perm, bool counted, int sms, cudaStream_t s) {
  const unsigned g_chunks =
      static_cast<unsigned>(std::min<uint64_t>((a.nchunks * 32ull + kRsThreads - 1) / kRsThreads,
                                               8ull * sms));
  const unsigned g_segs = static_cast<unsigned>(
      std::min<uint64_t>((maxact + kRsThreads - 1ull) / kRsThreads, 8ull * sms));
  const unsigned g_tiles = static_cast<unsigned>(std::min<uint64_t>(
      (std::max<uint64_t>(maxact, a.nchunks) + kRsScanTile - 1u) / kRsScanTile, 8ull * sms));
  if (!counted) {
    rs_count_kernel<<<g_chunks, kRsThreads, 0, s>>>(a);
    // exclusive prefix of the chunk zeros (the total after the last chunk)
    rs_scan_reduce_kernel<<<g_tiles, kRsThreads, 0, s>>>(a.zc, nullptr, a.nchunks, a.tsum);
    rs_scan_tiles_kernel<<<1, kRsScanThreads, 0, s>>>(a.tsum, nullptr, a.nchunks,
                                                      a.zc + a.nchunks);
    rs_scan_down_kernel<<<g_tiles, kRsThreads, 0, s>>>(a.zc, nullptr, a.nchunks, a.tsum);
  }
  rs_children_kernel<<<g_segs, kRsThreads, 0, s>>>(a);
  // the next active list: exclusive prefix of the children kept, its total is the list size
  rs_scan_reduce_kernel<<<g_tiles, kRsThreads, 0, s>>>(a.cnt, a.act_n, 0u, a.tsum);
  rs_scan_tiles_kernel<<<1, kRsScanThreads, 0, s>>>(a.tsum, a.act_n, 0u, a.nxt_n);
  rs_scan_down_kernel<<<g_tiles, kRsThreads, 0, s>>>(a.cnt, a.act_n, 0u, a.tsum);
  rs_list_write_kernel<<<g_segs, kRsThreads, 0, s>>>(a);
  rs_chunk_first_kernel<<<static_cast<unsigned>(std::min<uint64_t>(
                              (a.nchunks + kRsThreads - 1u) / kRsThreads, 8ull * sms)),
                          kRsThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (w) {
    case 4: return rs_launch_split<uint32_t>(a, in, out, perm, sms, s);
    case 8: return rs_launch_split<uint2>(a, in, out, perm, sms, s);
    default: return rs_launch_split<uint4>(a, in, out, perm, sms, s);
  }
}

template <typename E>
cudaError_t rs_launch_fy(const void *in, void *out, uint64_t n, uint2 key, const uint32_t *bnd,
                         uint32_t B, int sms, cudaStream_t s) {
  uint32_t P = B + 2u;
  while (P % 64u != 2u) ++P;
  // the lanes' index and draw regions (two of P 16-bit entries a lane) within kBudget
  constexpr uint32_t kBudget = 132u * 1024u;
  const uint32_t lanes = std::max<uint32_t>(1u, std::min<uint32_t>(32u, kBudget / (4u * P)));
  // the regions, the window's list of segment starts (the starts waiting plus one read of 32
  // bitmap words) and the threads' queues of second-word draws
  const size_t smem = ((2u * static_cast<size_t>(lanes) * P + 1u) & ~static_cast<size_t>(1u)) * 2u +
                      (lanes + 32u * 32u + 32u) * 4u + kRsFyThreads * kRsFyFail * 2u;
  // (in place only for 4-byte rows and final segments of at most kRsFyInPlaceMax: the planner
  // gives an even number of levels only then)
  if (in == out && (sizeof(E) != 4u || B > kRsFyInPlaceMax)) return cudaErrorInvalidValue;
  auto kern = rs_fy_kernel<E, false>;
  if constexpr (sizeof(E) == 4u) {
    if (in == out) kern = rs_fy_kernel<E, true>;
  }
  cudaError_t e = allow_dynamic_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRsFyThreads, smem);
  if (e != cudaSuccess) return e;
  const uint64_t windows = ((n + 31u) / 32u + kRsFyWinWords - 1u) / kRsFyWinWords;
  const uint64_t resident = static_cast<uint64_t>(std::max(per_sm, 1)) * sms;
  const unsigned grid = static_cast<unsigned>(std::max<uint64_t>(1u, std::min(windows, resident)));
  kern<<<grid, kRsFyThreads, smem, s>>>(static_cast<const E *>(in), static_cast<E *>(out), n, key,
                                        bnd, P, lanes);
  return cudaGetLastError();
}

thread_local cudaError_t g_rs_last_error = cudaSuccess;

bool rs_failed(cudaError_t e) {
  if (e != cudaSuccess) g_rs_last_error = e;
  return e != cudaSuccess;
}

ms_status rs_run(void *data, bool perm, uint64_t n, uint32_t w, uint64_t seed, uint32_t B,
                 void *ws, size_t ws_bytes, cudaStream_t s) {
  if (w != 4 && w != 8 && w != 16) return MS_ERR_INVALID;
  if (perm && w != 4) return MS_ERR_INVALID;
  if (B == 0 || n > 0xFFFFFFFFull) return MS_ERR_INVALID;
  if (B > MS_MAX_B) return MS_ERR_UNSUPPORTED;
  if (n <= 1) {
    if (perm && n == 1) {
      if (data == nullptr || reinterpret_cast<uintptr_t>(data) % 4 != 0) return MS_ERR_INVALID;
      if (rs_failed(cudaMemsetAsync(data, 0, 4, s))) return MS_ERR_CUDA;
    }
    return MS_OK;
  }
  const RsLayout L = rs_layout(n, w, B);
  if (data == nullptr || reinterpret_cast<uintptr_t>(data) % w != 0) return MS_ERR_INVALID;
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < L.total)
    return MS_ERR_INVALID;
  const int sms = sm_count();
  if (sms <= 0) return MS_ERR_CUDA;
  char *base = static_cast<char *>(ws);
  void *W = base + L.buf;
  uint32_t *ctl = reinterpret_cast<uint32_t *>(base + L.ctl);
  uint2 *act[2] = {reinterpret_cast<uint2 *>(base + L.act0), reinterpret_cast<uint2 *>(base + L.act1)};
  RsArgs a;
  a.n = n;
  a.key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  a.level = 0;
  a.B = B;
  a.nchunks = L.nchunks;
  a.zc = reinterpret_cast<uint32_t *>(base + L.zc);
  a.zb = reinterpret_cast<uint8_t *>(base + L.zb);
  a.zseg = reinterpret_cast<uint32_t *>(base + L.zseg);
  a.zs = reinterpret_cast<uint32_t *>(base + L.zs);
  a.cnt = reinterpret_cast<uint32_t *>(base + L.cnt);
  a.bnd = reinterpret_cast<uint32_t *>(base + L.bnd);
  a.tsum = reinterpret_cast<uint32_t *>(base + L.tsum);
  a.cfirst = reinterpret_cast<uint32_t *>(base + L.cfirst);
  if (rs_failed(cudaMemsetAsync(a.bnd, 0, ((n + 31u) / 32u + 1u) * 4u, s)) ||
      rs_failed(cudaMemsetAsync(ctl, 0, 256, s)))
    return MS_ERR_CUDA;
  rs_init_kernel<<<1, 32, 0, s>>>(a, act[0], ctl);
  if (rs_failed(cudaGetLastError())) return MS_ERR_CUDA;
  const uint32_t levels = L.plevels;
  uint32_t *const zca = reinterpret_cast<uint32_t *>(base + L.zca);
  uint8_t *const zba = reinterpret_cast<uint8_t *>(base + L.zba);
  if (levels > 0) {
    // the planned levels' zero counts, then one exclusive scan over all of them
    const uint64_t warps = static_cast<uint64_t>(levels) * L.nchunks;
    const uint32_t nall = levels * (L.nchunks + 1u);
    const unsigned g_tiles = static_cast<unsigned>(
        std::min<uint64_t>((nall + kRsScanTile - 1u) / kRsScanTile, 8ull * sms));
    rs_count_all_kernel<<<static_cast<unsigned>((warps * 32u + kRsThreads - 1u) / kRsThreads),
                          kRsThreads, 0, s>>>(a, levels, zca, zba);
    rs_scan_reduce_kernel<<<g_tiles, kRsThreads, 0, s>>>(zca, nullptr, nall, a.tsum);
    rs_scan_tiles_kernel<<<1, kRsScanThreads, 0, s>>>(a.tsum, nullptr, nall, ctl + 2);
    rs_scan_down_kernel<<<g_tiles, kRsThreads, 0, s>>>(zca, nullptr, nall, a.tsum);
    if (rs_failed(cudaGetLastError())) return MS_ERR_CUDA;
  }
  uint32_t lv = 0;
  auto run_levels = [&](uint32_t upto) -> bool {
    for (; lv < upto; ++lv) {
      RsArgs l = a;
      l.level = lv;
      l.act = act[lv % 2u];
      l.act_n = ctl + (lv % 2u);
      l.nxt = act[(lv + 1u) % 2u];
      l.nxt_n = ctl + ((lv + 1u) % 2u);
      const void *in = (lv % 2u == 0u) ? data : W;
      void *out = (lv % 2u == 0u) ? W : data;
      const bool counted = lv < levels;
      if (counted) {
        l.zc = zca + static_cast<uint64_t>(lv) * (L.nchunks + 1u);
        l.zb = zba + static_cast<uint64_t>(lv) * L.nchunks * kRsChunkBlocks;
      }
      if (rs_failed(rs_level(l, L.maxact, in, out, w, perm && lv == 0u, counted, sms, s)))
        return false;
    }
    return true;
  };
  if (!run_levels(levels)) return MS_ERR_CUDA;
  if (levels > 0) {
    // segments still above B after the planned levels: read the count and run pairs of levels
    for (;;) {
      uint32_t left = 0;
      if (rs_failed(cudaMemcpyAsync(&left, ctl + (lv % 2u), 4, cudaMemcpyDeviceToHost, s)) ||
          rs_failed(cudaStreamSynchronize(s)))
        return MS_ERR_CUDA;
      if (left == 0u) break;
      if (lv + 2u > 4096u) return MS_ERR_UNSUPPORTED;
      if (!run_levels(lv + 2u)) return MS_ERR_CUDA;
    }
  }
  // the data sits in W after an odd number of levels, in the caller's buffer after an even
  // number (the Fisher-Yates pass then runs in place); with no level at all it is the input
  const bool in_place = rs_fy_in_place(w, B);
  void *src = (lv % 2u == 1u) ? W : data;
  if (levels == 0) {
    void *dst0 = in_place ? data : W;
    if (perm) {
      rs_iota_kernel<<<static_cast<unsigned>(std::min<uint64_t>((n + 255u) / 256u, 8ull * sms)),
                       256, 0, s>>>(static_cast<uint32_t *>(dst0), n);
      if (rs_failed(cudaGetLastError())) return MS_ERR_CUDA;
    } else if (!in_place &&
               rs_failed(cudaMemcpyAsync(W, data, n * w, cudaMemcpyDeviceToDevice, s))) {
      return MS_ERR_CUDA;
    }
    src = dst0;
  }
  // Algorithm 1 on every final segment, from src into the caller's buffer
  cudaError_t e;
  switch (w) {
    case 4: e = rs_launch_fy<uint32_t>(src, data, n, a.key, a.bnd, B, sms, s); break;
    case 8: e = rs_launch_fy<uint2>(src, data, n, a.key, a.bnd, B, sms, s); break;
    default: e = rs_launch_fy<uint4>(src, data, n, a.key, a.bnd, B, sms, s); break;
  }
  return rs_failed(e) ? MS_ERR_CUDA : MS_OK;
}

}  // namespace
}  // namespace msk

extern "C" {

size_t ms_rs_workspace_bytes(uint64_t n, uint32_t w, uint32_t B) {
  if ((w != 4 && w != 8 && w != 16) || B == 0 || B > MS_MAX_B || n > 0xFFFFFFFFull) return 0;
  if (n <= 1) return 256;
  return msk::rs_layout(n, w, B).total;
}

ms_status ms_rs_shuffle(void *d_data, uint64_t n, uint32_t w, uint64_t seed, uint32_t B,
                        void *d_ws, size_t ws_bytes, ms_stream_t stream) {
  return msk::rs_run(d_data, false, n, w, seed, B, d_ws, ws_bytes,
                     static_cast<cudaStream_t>(stream));
}

ms_status ms_rs_perm(uint32_t *d_out, uint64_t n, uint64_t seed, uint32_t B, void *d_ws,
                     size_t ws_bytes, ms_stream_t stream) {
  return msk::rs_run(d_out, true, n, 4, seed, B, d_ws, ws_bytes,
                     static_cast<cudaStream_t>(stream));
}

}  // extern "C"
