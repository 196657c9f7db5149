// ms_merge.cuh -- device building blocks shared by the base-block, local-level and batch
// kernels: rejection draws from a given Philox word, warp / CTA groups, and one merge level of
// Algorithm 3 (arXiv 1508.03167) executed by a group over a region held in (or read from)
// memory, with the stable interleave of Algorithm 2 and its random-insertion tail.
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

template <typename E>
__device__ __forceinline__ void swap_smem(E *a, uint32_t i, uint32_t j) {
  const E t = a[i];
  a[i] = a[j];
  a[j] = t;
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

// One merge level of Algorithm 3 over the group's region: 2^(gl-lam) merged runs of 2^lam base
// blocks become 2^(gl-lam-1) runs. lb = global index of the region's first base block; the
// tile-relative positions are relative to g0 (global position of the tile's first element).
// X is read as base blocks at stride P (padded) on level 0 of the warp phase, contiguous
// otherwise (X may also be global memory); Y is written contiguously.
template <int G, typename E>
__device__ __forceinline__ void merge_level(const LeafArgs &a, const GroupSmem &S, uint64_t lb,
                                            uint64_t leaf0, uint64_t g0, uint32_t lam,
                                            uint32_t gl, const E *X, uint32_t xcap, bool padded,
                                            E *Y) {
  using Gp = Group<G>;
  constexpr uint32_t kT = Gp::kThreads;
  // consecutive positions per lane in the gather, kLpw lanes per coin word
  constexpr uint32_t kPos = sizeof(E) >= 16 ? 4u : 8u;
  constexpr uint32_t kLpw = 32u / kPos;
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

  // ---- stable interleave and leftover copy: kLpw lanes per coin word, kPos positions per lane;
  // all loads of a lane are issued before its stores
  for (uint32_t u = gt / kLpw; u < U; u += kT / kLpw) {
    const uint32_t r = merge_of(u);
    const uint32_t j = u - r * Wm;
    const uint32_t N = S.m_N[r];
    const uint32_t sub = (gt % kLpw) * kPos;
    const uint32_t t0 = 32u * j + sub;
    if (t0 >= N) continue;
    const uint32_t word = S.cw[u];
    const uint32_t Zu = S.zp[u];
    const uint32_t aa = S.m_a[r], bb = S.m_b[r], T = S.m_T[r], lbase = S.m_lb[r];
    const uint32_t dst = S.m_s[r] + t0;
    const uint32_t cnt = min(kPos, N - t0);
    uint32_t z = Zu + __popc(~word & low_mask(sub));  // Z + zbase at position t0
    E v[kPos];
#pragma unroll
    for (uint32_t k = 0; k < kPos; ++k) {
      if (k < cnt) {
        const uint32_t t = t0 + k;
        const uint32_t bit = (word >> (sub + k)) & 1u;
        const uint32_t src = (t < T) ? (bit ? bb + t - z : aa + z) : lbase + t;
        z += bit ^ 1u;
        v[k] = X[min(src, xcap - 1u)];  // clamp keeps the read inside the buffer
      }
    }
#pragma unroll
    for (uint32_t k = 0; k < kPos; ++k)
      if (k < cnt) Y[dst + k] = v[k];
  }

  // ---- tail draws, one Philox block per four consecutive positions
  const uint32_t Q = total >> 16;
  const uint32_t K = total & 0xFFFFu;
  const bool precomputed = K <= S.tcap;
  if (precomputed) {
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

  // ---- random insertion of positions T..N-1, in order (Algorithm 2's second loop)
  constexpr uint32_t kBatch = sizeof(E) >= 16 ? 4u : 8u;
  for (uint32_t r = gt; r < Mt; r += kT) {
    const uint32_t T = S.m_T[r], N = S.m_N[r], s = S.m_s[r];
    E *C = Y + s;
    uint32_t i = T;
    if (precomputed) {
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
  Gp::sync();
}

}  // namespace
}  // namespace msk
