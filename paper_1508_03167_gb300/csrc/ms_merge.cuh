// ms_merge.cuh -- device building blocks shared by the base-block, local-level and batch
// kernels: rejection draws from a given Philox word, warp / CTA groups, and one merge level of
// Algorithm 2 (arXiv 1508.03167) executed by a group over a region held in (or read from)
// memory, with the stable interleave of Algorithm 3 and its random-insertion tail.
#pragma once

#include "ms_common.cuh"
#include "ms_device.cuh"
#include "ms_plan.h"

namespace msk {
namespace {

constexpr int kLeafThreads = 256;
constexpr uint32_t kLeafWarps = kLeafThreads / 32;
constexpr uint32_t kGroupMerges = 16;  // merges per level of one group (warp: dw <= 5)

struct LeafArgs {
  const void *in;
  void *out;
  uint64_t n;
  uint64_t q;
  uint2 key;
  uint32_t c;
  uint32_t d;          // fused levels
  uint32_t dw;         // levels done by single warps
  uint32_t tile_max;   // elements of the largest tile
  uint32_t stride;     // odd stride of a base block in buffer 0
  uint32_t buf0;       // elements of buffer 0
  uint32_t ucap_w, tcap_w, ucap_c, tcap_c;  // coin-word / tail-draw capacities per group
  uint32_t aux_w;      // bytes of one warp's auxiliary region
};

// first 16-byte boundary at or after p
template <typename T>
__device__ __forceinline__ unsigned char *align16(T *p) {
  return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 15u) &
                                           ~static_cast<uintptr_t>(15u));
}

template <typename E>
__device__ __forceinline__ void swap_smem(E *a, uint32_t i, uint32_t j) {
  const E t = a[i];
  a[i] = a[j];
  a[j] = t;
}

// Algorithm 1's swap chain on 16-bit local indices: for i = L-1 down to 1, swap A[i] with
// A[D[i]] (each draw D[i] in [0, i], clamped into it). Four steps k0 > k1 > k2 > k3 at a time:
// their eight reads are made together, then each step takes its two values from the group's
// earlier writes to its targets where there were any (the later write wins), and the writes go
// out in the chain's order, so a group waits for one shared-memory read rather than four.
// Positions above a step are never a later step's target, so only the targets j0..j2 forward.
__device__ __forceinline__ void fy_chain16(uint16_t *A, const uint16_t *D, uint32_t L) {
  uint32_t i = L;
  while (i >= 5u) {
    const uint32_t k0 = i - 1u, k1 = i - 2u, k2 = i - 3u, k3 = i - 4u;
    const uint32_t j0 = min(static_cast<uint32_t>(D[k0]), k0);
    const uint32_t j1 = min(static_cast<uint32_t>(D[k1]), k1);
    const uint32_t j2 = min(static_cast<uint32_t>(D[k2]), k2);
    const uint32_t j3 = min(static_cast<uint32_t>(D[k3]), k3);
    const uint32_t c0 = A[k0], c1 = A[k1], c2 = A[k2], c3 = A[k3];
    const uint32_t v0 = A[j0], v1 = A[j1], v2 = A[j2], v3 = A[j3];
    const uint32_t x1 = k1 == j0 ? c0 : c1;
    const uint32_t y1 = j1 == j0 ? c0 : v1;
    const uint32_t x2 = k2 == j1 ? x1 : (k2 == j0 ? c0 : c2);
    const uint32_t y2 = j2 == j1 ? x1 : (j2 == j0 ? c0 : v2);
    const uint32_t x3 = k3 == j2 ? x2 : (k3 == j1 ? x1 : (k3 == j0 ? c0 : c3));
    const uint32_t y3 = j3 == j2 ? x2 : (j3 == j1 ? x1 : (j3 == j0 ? c0 : v3));
    A[k0] = static_cast<uint16_t>(v0);
    A[j0] = static_cast<uint16_t>(c0);
    A[k1] = static_cast<uint16_t>(y1);
    A[j1] = static_cast<uint16_t>(x1);
    A[k2] = static_cast<uint16_t>(y2);
    A[j2] = static_cast<uint16_t>(x2);
    A[k3] = static_cast<uint16_t>(y3);
    A[j3] = static_cast<uint16_t>(x3);
    i -= 4u;
  }
  for (; i >= 2u; --i) swap_smem(A, i - 1u, min(static_cast<uint32_t>(D[i - 1u]), i - 1u));
}

// Rejection draw in [0, R) from the slices of one word (R >= 2); false if every slice rejects.
__device__ __forceinline__ bool draw_from_word(uint32_t word, uint32_t R, uint32_t &x) {
  const uint32_t b = 32u - __clz(R - 1u);
  const uint32_t mask = (b == 32u) ? 0xFFFFFFFFu : ((1u << b) - 1u);
  const uint32_t first = word & mask;
  if (first < R) {  // the first slice accepts with probability >= 1/2
    x = first;
    return true;
  }
  // floor(32 / b): 32 / b is either exact (b a power of two) or at least 1/32 away from an
  // integer, far beyond the error of the fast reciprocal, so the truncation is exact
  const uint32_t slices = static_cast<uint32_t>(__fdividef(32.0f, static_cast<float>(b)));
  for (uint32_t u = 1; u < slices; ++u) {
    const uint32_t v = (word >> (u * b)) & mask;
    if (v < R) {
      x = v;
      return true;
    }
  }
  return false;
}

// Continuation of a draw whose word j = 0 rejected every slice: words j = 1, 2, ...
__device__ __noinline__ uint32_t draw_continue(uint2 key, uint32_t tag, uint32_t level,
                                               uint32_t id, uint32_t pos, uint32_t R) {
  for (uint32_t j = 1; j < (1u << 20); ++j) {
    const uint4 blk = philox10(make_uint4(pos >> 2, id, (tag << 16) | level, j), key);
    uint32_t x;
    if (draw_from_word(pick_word(blk, pos & 3u), R, x)) return x;
  }
  return 0u;
}

// Draw in [0, R) of stream (tag, level, id, pos) given its word j = 0.
__device__ __forceinline__ uint32_t draw_with_word0(uint2 key, uint32_t tag, uint32_t level,
                                                    uint32_t id, uint32_t pos, uint32_t R,
                                                    uint32_t word0) {
  if (R <= 1u) return 0u;
  uint32_t x;
  if (draw_from_word(word0, R, x)) return x;
  return draw_continue(key, tag, level, id, pos, R);
}

// The same draw for Algorithm 1's inner loop, where every lane draws at every step: the first
// four slices of a word are tested without branches (the first one below R wins, as above), so
// lanes rejecting their first slice do not split the warp, and the continuation is inlined.
__device__ __forceinline__ bool draw_from_word_flat(uint32_t word, uint32_t R, uint32_t &x) {
  const uint32_t b = 32u - __clz(R - 1u);
  const uint32_t mask = (b == 32u) ? 0xFFFFFFFFu : ((1u << b) - 1u);
  // floor(32 / b), exact as in draw_from_word
  const uint32_t slices = static_cast<uint32_t>(__fdividef(32.0f, static_cast<float>(b)));
  uint32_t best = 0xFFFFFFFFu;
#pragma unroll
  for (int u = 3; u >= 0; --u) {
    const uint32_t v = (word >> min(static_cast<uint32_t>(u) * b, 31u)) & mask;
    if (static_cast<uint32_t>(u) < slices && v < R) best = v;
  }
  if (best != 0xFFFFFFFFu) {
    x = best;
    return true;
  }
  for (uint32_t u = 4; u < slices; ++u) {
    const uint32_t v = (word >> (u * b)) & mask;
    if (v < R) {
      x = v;
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ uint32_t draw_with_word0_flat(uint2 key, uint32_t tag, uint32_t level,
                                                         uint32_t id, uint32_t pos, uint32_t R,
                                                         uint32_t word0) {
  if (R <= 1u) return 0u;
  uint32_t x;
  if (draw_from_word_flat(word0, R, x)) return x;
  for (uint32_t j = 1; j < (1u << 20); ++j) {
    const uint4 blk = philox10(make_uint4(pos >> 2, id, (tag << 16) | level, j), key);
    if (draw_from_word_flat(pick_word(blk, pos & 3u), R, x)) return x;
  }
  return 0u;
}

// The same draw from word 0 without the reciprocal: slice u = 1, 2, 3 exists for b <= 16, 10,
// 8 (floor(32/b) > u), so the first four slices need no division; the rest of the word (b <= 6)
// is tested in a loop. False if the whole word rejects.
__device__ __forceinline__ bool draw_first_word(uint32_t word, uint32_t R, uint32_t &x) {
  const uint32_t b = 32u - __clz(R - 1u);
  const uint32_t mask = 0xFFFFFFFFu >> (32u - b);
  const uint32_t v0 = word & mask;
  const uint32_t v1 = __funnelshift_rc(word, 0u, b) & mask;
  const uint32_t v2 = __funnelshift_rc(word, 0u, 2u * b) & mask;
  const uint32_t v3 = __funnelshift_rc(word, 0u, 3u * b) & mask;
  const bool a0 = v0 < R;
  const bool a1 = b <= 16u && v1 < R;
  const bool a2 = b <= 10u && v2 < R;
  const bool a3 = b <= 8u && v3 < R;
  x = a0 ? v0 : (a1 ? v1 : (a2 ? v2 : v3));
  if (a0 | a1 | a2 | a3) return true;
  if (b <= 6u) {
    const uint32_t slices = 32u / b;
    for (uint32_t u = 4; u < slices; ++u) {
      const uint32_t v = (word >> (u * b)) & mask;
      if (v < R) {
        x = v;
        return true;
      }
    }
  }
  return false;
}

// draw_first_word with the slice width b (and mask, 2b, 3b) computed by the caller, for a run of
// positions that share it: R - 1 in [4q, 4q + 3] with q >= 1 never crosses a power of two
// (those of 4 and above are multiples of 4), so one quad of Algorithm 1's positions shares b.
__device__ __forceinline__ bool draw_first_word_b(uint32_t word, uint32_t R, uint32_t b,
                                                  uint32_t mask, uint32_t b2, uint32_t b3,
                                                  uint32_t &x) {
  const uint32_t v0 = word & mask;
  const uint32_t v1 = __funnelshift_rc(word, 0u, b) & mask;
  const uint32_t v2 = __funnelshift_rc(word, 0u, b2) & mask;
  const uint32_t v3 = __funnelshift_rc(word, 0u, b3) & mask;
  const bool a0 = v0 < R;
  const bool a1 = b <= 16u && v1 < R;
  const bool a2 = b <= 10u && v2 < R;
  const bool a3 = b <= 8u && v3 < R;
  x = a0 ? v0 : (a1 ? v1 : (a2 ? v2 : v3));
  if (a0 | a1 | a2 | a3) return true;
  if (b <= 6u) {
    const uint32_t slices = 32u / b;
    for (uint32_t u = 4; u < slices; ++u) {
      const uint32_t v = (word >> (u * b)) & mask;
      if (v < R) {
        x = v;
        return true;
      }
    }
  }
  return false;
}

// Algorithm 1 (descending Fisher-Yates) on one base block of L elements in shared memory:
// for i = L-1 .. 1, swap blk[i] with blk[j], j uniform in {0..i} from the LEAF stream of block
// `id` at position i. Positions go in quads (one Philox block serves four of them), and the
// block of the next quad is computed while the current one is applied.
template <typename E>
__device__ __forceinline__ void fisher_yates_block(E *blk, uint32_t L, uint32_t id, uint2 key) {
  if (L < 2u) return;
  uint32_t quad = (L - 1u) >> 2;
  uint4 cur = philox10(make_uint4(quad, id, (kTagLeaf << 16), 0u), key);
  uint32_t i = L - 1u;
  for (;;) {
    const uint4 nxt =
        quad > 0 ? philox10(make_uint4(quad - 1u, id, (kTagLeaf << 16), 0u), key) : cur;
    const uint32_t lo = quad << 2;  // first position of this quad
#pragma unroll
    for (uint32_t v = 4; v-- > 0;) {
      const uint32_t pos = lo + v;
      if (pos <= i && pos >= 1u) {
        const uint32_t j =
            draw_with_word0_flat(key, kTagLeaf, 0u, id, pos, pos + 1u, pick_word(cur, v));
        swap_smem(blk, pos, j);
      }
    }
    if (quad == 0) break;
    --quad;
    i = lo - 1u;
    cur = nxt;
  }
}

// ---------------------------------------------------------------------------- groups ------
// A group is one warp (G = 1) or the whole CTA (G = kLeafWarps).
template <int G>
struct Group {
  static constexpr uint32_t kThreads = 32u * G;
  static __device__ __forceinline__ void sync() {
    if constexpr (G == 1) __syncwarp();
    else __syncthreads();
  }
  static __device__ __forceinline__ uint32_t tid() {
    if constexpr (G == 1) return threadIdx.x & 31u;
    else return threadIdx.x;
  }
  // exclusive scan of one value per thread of the group; *total gets the group sum
  static __device__ __forceinline__ uint32_t exscan(uint32_t v, uint32_t *scratch,
                                                    uint32_t *total) {
    if constexpr (G == 1) {
      const uint32_t incl = warp_inclusive_scan(v);
      *total = __shfl_sync(kFullMask, incl, 31);
      return incl - v;
    } else {
      return block_exclusive_scan(v, scratch, total);
    }
  }
};

// Per-group shared-memory views.
struct GroupSmem {
  uint32_t *cw;   // coin words of the level
  uint32_t *zp;   // exclusive zero prefix per coin word (over the group's level)
  uint16_t *mv;   // precomputed tail draws
  uint32_t ucap;  // capacity of cw / zp
  uint32_t tcap;  // capacity of mv
  // per merge (kGroupMerges entries): source bases of the halves (rebased by the merge's zero
  // prefix once T is known), destination base, first-half size, size, break step, leftover base,
  // packed tail prefix
  uint32_t *m_a, *m_b, *m_s, *m_n1, *m_N, *m_T, *m_lb, *m_off;
  uint32_t *scratch;  // 33 words for CTA-wide scans
};

// One merge level of Algorithm 2 over the group's region: 2^(gl-lam) merged runs of 2^lam base
// blocks become 2^(gl-lam-1) runs. lb = global index of the region's first base block; the
// tile-relative positions are relative to g0 (global position of the tile's first element).
// X is read as base blocks at stride P (padded) on level 0 of the warp phase, contiguous
// otherwise (X may also be global memory); Y is written contiguously. V (vcap elements, this
// group's own) is scratch for the tail patches: the level's input, dead once the gather is done.
template <int G, typename E>
__device__ __forceinline__ void merge_level(const LeafArgs &a, const GroupSmem &S, uint64_t lb,
                                            uint64_t leaf0, uint64_t g0, uint32_t lam,
                                            uint32_t gl, const E *X, uint32_t xcap, bool padded,
                                            E *Y, E *V, uint32_t vcap) {
  using Gp = Group<G>;
  constexpr uint32_t kT = Gp::kThreads;
  const uint32_t gt = Gp::tid();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t Mt = 1u << (gl - lam - 1u);
  const uint64_t rbase = lb >> (lam + 1u);  // global id of the region's first merge
  const uint32_t Nmax = static_cast<uint32_t>(((a.n << (lam + 1u)) + a.q - 1u) >> a.c);
  const uint32_t Wm = (Nmax + 31u) >> 5;    // coin words per merge
  const uint32_t BPM = (Nmax + 127u) >> 7;  // Philox blocks per merge
  const uint32_t U = Mt * Wm;
  // u / Wm as a multiply-high, exact for u, Wm < 2^16 (Wm = 1 is the identity)
  const uint32_t wm_magic = Wm > 1u ? static_cast<uint32_t>(0x100000000ull / Wm) + 1u : 0u;
  auto merge_of = [&](uint32_t u) { return Wm > 1u ? __umulhi(u, wm_magic) : u; };

  // ---- merge geometry
  for (uint32_t r = gt; r < Mt; r += kT) {
    const uint64_t L0 = lb + (static_cast<uint64_t>(r) << (lam + 1u));
    const uint64_t s = boundary(a.n, a.c, L0);
    const uint64_t mid = boundary(a.n, a.c, L0 + (1ull << lam));
    const uint64_t e = boundary(a.n, a.c, L0 + (2ull << lam));
    const uint32_t sl = static_cast<uint32_t>(s - g0);
    const uint32_t n1 = static_cast<uint32_t>(mid - s);
    S.m_s[r] = sl;
    S.m_n1[r] = n1;
    S.m_N[r] = static_cast<uint32_t>(e - s);
    S.m_T[r] = static_cast<uint32_t>(e - s);
    if (padded) {  // the halves are base blocks L0 and L0+1 of the tile at stride P
      const uint32_t k = static_cast<uint32_t>(L0 - leaf0);
      S.m_a[r] = k * a.stride;
      S.m_b[r] = (k + 1u) * a.stride;
    } else {
      S.m_a[r] = sl;
      S.m_b[r] = sl + n1;
    }
  }
  // ---- coin words
  for (uint32_t idx = gt; idx < Mt * BPM; idx += kT) {
    const uint32_t r = idx / BPM;
    const uint32_t jb = idx - r * BPM;
    const uint4 blk = coin_block(a.key, lam, static_cast<uint32_t>(rbase + r), jb);
    const uint32_t base = r * Wm + 4u * jb;
    if (4u * jb + 0u < Wm) S.cw[base + 0u] = blk.x;
    if (4u * jb + 1u < Wm) S.cw[base + 1u] = blk.y;
    if (4u * jb + 2u < Wm) S.cw[base + 2u] = blk.z;
    if (4u * jb + 3u < Wm) S.cw[base + 3u] = blk.w;
  }
  Gp::sync();

  // ---- zero counts per coin word and their exclusive prefix over the group's level
  {
    const uint32_t per = (U + kT - 1u) / kT;
    const uint32_t u0 = min(gt * per, U);
    const uint32_t u1 = min(u0 + per, U);
    uint32_t local = 0;
    for (uint32_t u = u0; u < u1; ++u) {
      const uint32_t r = merge_of(u);
      const uint32_t j = u - r * Wm;
      const uint32_t N = S.m_N[r];
      const uint32_t valid = (32u * j >= N) ? 0u : min(32u, N - 32u * j);
      const uint32_t z = __popc(~S.cw[u] & low_mask(valid));
      S.zp[u] = z;
      local += z;
    }
    uint32_t total;
    uint32_t excl = Gp::exscan(local, S.scratch, &total);
    for (uint32_t u = u0; u < u1; ++u) {
      const uint32_t z = S.zp[u];
      S.zp[u] = excl;
      excl += z;
    }
  }
  Gp::sync();

  // ---- break step T: the (n1+1)-th zero or the (n2+1)-th one, whichever comes first
  for (uint32_t u = gt; u < U; u += kT) {
    const uint32_t r = merge_of(u);
    const uint32_t j = u - r * Wm;
    const uint32_t N = S.m_N[r];
    if (32u * j >= N) continue;
    const uint32_t valid = min(32u, N - 32u * j);
    const uint32_t vm = low_mask(valid);
    const uint32_t word = S.cw[u];
    const uint32_t Zs = S.zp[u] - S.zp[r * Wm];
    const uint32_t Os = 32u * j - Zs;
    const uint32_t zeros = __popc(~word & vm);
    const uint32_t ones = valid - zeros;
    const uint32_t n1 = S.m_n1[r];
    const uint32_t n2 = N - n1;
    if (Zs <= n1 && n1 < Zs + zeros)
      atomicMin(&S.m_T[r], 32u * j + select_set_bit(~word & vm, n1 - Zs));
    if (Os <= n2 && n2 < Os + ones)
      atomicMin(&S.m_T[r], 32u * j + select_set_bit(word & vm, n2 - Os));
  }
  Gp::sync();

  // ---- per merge: rebased sources, leftover base, tail sizes (packed quads << 16 | length)
  uint32_t packed = 0;
  if (gt < Mt) {
    const uint32_t r = gt;
    const uint32_t T = S.m_T[r], N = S.m_N[r], n1 = S.m_n1[r];
    const uint32_t zbase = S.zp[r * Wm];
    const uint32_t A = S.m_a[r], B = S.m_b[r];
    // position t >= T takes the rest of the half that did not run out, in order; the coin at T
    // names the half that ran out (0: the first half)
    uint32_t lbase = 0;
    if (T < N) {
      const uint32_t bitT = (S.cw[r * Wm + (T >> 5)] >> (T & 31u)) & 1u;
      lbase = bitT ? A - (N - n1) : B - n1;
    }
    S.m_lb[r] = lbase;
    S.m_a[r] = A - zbase;  // A + Z with Z = zp[u] - zbase + (zeros below t in word u)
    S.m_b[r] = B + zbase;  // B + t - Z
    const uint32_t k = N - T;
    const uint32_t quads = k ? ((N - 1u) >> 2) - (T >> 2) + 1u : 0u;
    packed = (quads << 16) | k;
  }
  uint32_t total;
  {
    const uint32_t excl = Gp::exscan(packed, S.scratch, &total);
    if (gt < Mt) S.m_off[gt] = excl;
  }
  Gp::sync();

  // ---- stable interleave and leftover copy: one lane per position, so a warp covers one coin
  // word (32 consecutive outputs: conflict-free stores; the loads are two runs, one per half).
  // A warp takes four consecutive words at a time (one vector load of their coin words and one
  // of their prefixes; the merge's bases loaded once when all four lie in one merge) and issues
  // the four loads of its lanes before their stores.
  {
    constexpr uint32_t kWords = 4;
    const uint32_t wg = gt >> 5;
    const uint32_t lt = low_mask(lane);  // lanes below this one
    const bool vec =
        ((reinterpret_cast<uintptr_t>(S.cw) | reinterpret_cast<uintptr_t>(S.zp)) & 15u) == 0;
    for (uint32_t u0 = wg * kWords; u0 < U; u0 += G * kWords) {
      uint32_t cwv[kWords], zpv[kWords];
      if (vec && u0 + kWords <= U) {
        const uint4 c4 = *reinterpret_cast<const uint4 *>(S.cw + u0);
        const uint4 z4 = *reinterpret_cast<const uint4 *>(S.zp + u0);
        cwv[0] = c4.x; cwv[1] = c4.y; cwv[2] = c4.z; cwv[3] = c4.w;
        zpv[0] = z4.x; zpv[1] = z4.y; zpv[2] = z4.z; zpv[3] = z4.w;
      } else {
#pragma unroll
        for (uint32_t k = 0; k < kWords; ++k) {
          cwv[k] = u0 + k < U ? S.cw[u0 + k] : 0u;
          zpv[k] = u0 + k < U ? S.zp[u0 + k] : 0u;
        }
      }
      const uint32_t r0 = merge_of(u0);
      const bool one_merge = merge_of(min(u0 + kWords - 1u, U - 1u)) == r0;
      const uint32_t N0 = S.m_N[r0], T0 = S.m_T[r0], A0 = S.m_a[r0], B0 = S.m_b[r0],
                     L0 = S.m_lb[r0], s0 = S.m_s[r0];
      E v[kWords];
      uint32_t dst[kWords];
#pragma unroll
      for (uint32_t k = 0; k < kWords; ++k) {
        dst[k] = kNone;
        const uint32_t u = u0 + k;
        if (u < U) {
          uint32_t r = r0, N = N0, T = T0, aa = A0, bb = B0, lbase = L0, sb = s0;
          if (!one_merge) {
            r = merge_of(u);
            N = S.m_N[r]; T = S.m_T[r]; aa = S.m_a[r]; bb = S.m_b[r];
            lbase = S.m_lb[r]; sb = S.m_s[r];
          }
          const uint32_t t = 32u * (u - r * Wm) + lane;
          if (t < N) {
            const uint32_t word = cwv[k];
            const uint32_t z = zpv[k] + __popc(~word & lt);  // Z + zbase at t
            const uint32_t src =
                (t < T) ? (((word >> lane) & 1u) ? bb + t - z : aa + z) : lbase + t;
            v[k] = X[min(src, xcap - 1u)];  // clamp keeps the read inside the buffer
            dst[k] = sb + t;
          }
        }
      }
#pragma unroll
      for (uint32_t k = 0; k < kWords; ++k)
        if (dst[k] != kNone) Y[dst[k]] = v[k];
    }
  }

  // ---- tail draws, one Philox block per four consecutive positions
  const uint32_t Q = total >> 16;
  const uint32_t K = total & 0xFFFFu;
  const bool drawn = K <= S.tcap;
  if (drawn) {
    for (uint32_t gq = gt; gq < Q; gq += kT) {
      uint32_t lo = 0, hi = Mt;  // largest r with quad offset <= gq
      while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((S.m_off[mid] >> 16) <= gq) lo = mid;
        else hi = mid;
      }
      const uint32_t r = lo;
      const uint32_t T = S.m_T[r], N = S.m_N[r];
      const uint32_t quad = (T >> 2) + (gq - (S.m_off[r] >> 16));
      const uint32_t id = static_cast<uint32_t>(rbase + r);
      const uint4 w0 = philox10(make_uint4(quad, id, (kTagTail << 16) | lam, 0u), a.key);
      const uint32_t koff = S.m_off[r] & 0xFFFFu;
#pragma unroll
      for (uint32_t v = 0; v < 4u; ++v) {
        const uint32_t i = 4u * quad + v;
        if (i >= T && i < N)
          S.mv[koff + (i - T)] = static_cast<uint16_t>(
              draw_with_word0(a.key, kTagTail, lam, id, i, i + 1u, pick_word(w0, v)));
      }
    }
  }
  Gp::sync();

  // ---- random insertion of positions T..N-1 (Algorithm 3's second loop), resolved in parallel:
  // the element at tail position i lands on m_i at step i and moves on to T + s at every later
  // step s whose draw hits its position; the element a first hit displaces from m < T follows
  // the same rule from position i. Final positions are found for every tail step at once, then
  // all moved values are read (into the dead input buffer V) before any is written back.
  const bool parallel = drawn && (2ull * K * sizeof(E) + 4ull * K <= 1ull * vcap * sizeof(E));
  if (parallel) {
    uint32_t *const fin = reinterpret_cast<uint32_t *>(V + 2u * K);  // d1 | d2 << 16 per step
    auto merge_of_step = [&](uint32_t g) {
      uint32_t lo = 0, hi = Mt;  // largest r with tail offset <= g
      while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((S.m_off[mid] & 0xFFFFu) <= g) lo = mid;
        else hi = mid;
      }
      return lo;
    };
    for (uint32_t g = gt; g < K; g += kT) {
      const uint32_t r = merge_of_step(g);
      const uint32_t koff = S.m_off[r] & 0xFFFFu;
      const uint32_t T = S.m_T[r];
      const uint32_t k_r = S.m_N[r] - T;
      const uint16_t *mr = S.mv + koff;  // mr[st] = draw of position T + st
      const uint32_t st = g - koff;
      const uint32_t m = mr[st];
      // follow an element from position pos after step `from - 1` (eight draws loaded at a
      // time, then compared in order)
      auto follow = [&](uint32_t pos, uint32_t from) {
        uint32_t s2 = from;
        for (; s2 + 8u <= k_r; s2 += 8u) {
          uint32_t d[8];
#pragma unroll
          for (uint32_t k = 0; k < 8u; ++k) d[k] = mr[s2 + k];
#pragma unroll
          for (uint32_t k = 0; k < 8u; ++k)
            if (d[k] == pos) pos = T + s2 + k;
        }
        for (; s2 < k_r; ++s2)
          if (mr[s2] == pos) pos = T + s2;
        return pos;
      };
      const uint32_t d1 = follow(m, st + 1u);
      uint32_t d2 = 0xFFFFu;
      if (m < T) {
        uint32_t hits = 0;
        uint32_t s2 = 0;
        for (; s2 + 8u <= st; s2 += 8u) {
#pragma unroll
          for (uint32_t k = 0; k < 8u; ++k) hits += (mr[s2 + k] == m);
        }
        for (; s2 < st; ++s2) hits += (mr[s2] == m);
        if (hits == 0) d2 = follow(T + st, st + 1u);
      }
      fin[g] = d1 | (d2 << 16);
    }
    Gp::sync();
    for (uint32_t g = gt; g < K; g += kT) {
      const uint32_t r = merge_of_step(g);
      const uint32_t koff = S.m_off[r] & 0xFFFFu;
      const uint32_t C = S.m_s[r];
      const uint32_t i = S.m_T[r] + (g - koff);
      V[g] = Y[C + i];
      if ((fin[g] >> 16) != 0xFFFFu) V[K + g] = Y[C + S.mv[g]];
    }
    Gp::sync();
    for (uint32_t g = gt; g < K; g += kT) {
      const uint32_t r = merge_of_step(g);
      const uint32_t koff = S.m_off[r] & 0xFFFFu;
      const uint32_t C = S.m_s[r];
      const uint32_t i = S.m_T[r] + (g - koff);
      const uint32_t f = fin[g];
      const uint32_t d1 = f & 0xFFFFu, d2 = f >> 16;
      if (d1 != i) Y[C + d1] = V[g];
      if (d2 != 0xFFFFu) Y[C + d2] = V[K + g];
    }
  } else {
    // sequential fallback (more tail steps than the scratch holds): one thread per merge
    // applies the swaps in order, eight at a time whenever those eight provably commute
    constexpr uint32_t kBatch = sizeof(E) >= 16 ? 4u : 8u;
    for (uint32_t r = gt; r < Mt; r += kT) {
      const uint32_t T = S.m_T[r], N = S.m_N[r], s = S.m_s[r];
      E *C = Y + s;
      uint32_t i = T;
      if (drawn) {
        const uint16_t *mk = S.mv + (S.m_off[r] & 0xFFFFu);  // mk[i - T] = draw of position i
        while (i < N) {
          if (i + kBatch <= N) {
            // swaps (i+k, m_k) for k < kBatch commute when every m_k lies before the window and
            // all m_k differ: then they touch 2*kBatch distinct positions
            uint32_t m[kBatch];
            bool ok = true;
#pragma unroll
            for (uint32_t k = 0; k < kBatch; ++k) {
              m[k] = mk[i - T + k];
              ok &= m[k] < i;
            }
#pragma unroll
            for (uint32_t k = 0; k < kBatch; ++k)
#pragma unroll
              for (uint32_t l = k + 1; l < kBatch; ++l) ok &= m[k] != m[l];
            if (ok) {
              E lo[kBatch], hi[kBatch];
#pragma unroll
              for (uint32_t k = 0; k < kBatch; ++k) {
                lo[k] = C[i + k];
                hi[k] = C[m[k]];
              }
#pragma unroll
              for (uint32_t k = 0; k < kBatch; ++k) {
                C[i + k] = hi[k];
                C[m[k]] = lo[k];
              }
              i += kBatch;
              continue;
            }
          }
          swap_smem(C, i, static_cast<uint32_t>(mk[i - T]));
          ++i;
        }
      } else {
        const uint32_t id = static_cast<uint32_t>(rbase + r);
        for (; i < N; ++i) swap_smem(C, i, draw_uniform(a.key, kTagTail, lam, id, i, i + 1u));
      }
    }
  }
  Gp::sync();
}

}  // namespace
}  // namespace msk
