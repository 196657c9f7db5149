// ms_level.cu -- one merge level of Algorithm 2 (arXiv 1508.03167) streamed through HBM.
//
// Every merge r of level l joins two shuffled halves [s, mid) and [mid, e). The merge is split
// into data-oblivious planning and one streaming pass:
//   count    zero coins per 4096-step chunk of every merge (Philox only, no array traffic);
//   scan     per merge: exclusive prefix of the chunk counts and the break step T, where a coin
//            first asks for an exhausted half (Algorithm 3's first loop);
//   kscan    prefix of the tail lengths N - T over the level's merges, and the first merge of
//            every 1024 tail steps (so a tail step finds its merge in a few probes);
//   insert   tail draws m_i (i = T..N-1, uniform in {0..i}) into a hash table keyed by
//            (merge, target position);
//   resolve  replays the random insertions (Algorithm 3's second loop) on indices only: every
//            displaced element's trajectory gives one (destination, source) patch;
//   gather   the streaming pass: out[s+t] = coin t ? B[t - Z_t] : A[Z_t] for t < T, the
//            remainder of the non-exhausted half for t >= T. For 4- and 8-byte elements each
//            4096-step chunk first copies its two source runs into shared memory (16-byte
//            asynchronous copies), then places eight outputs a thread; 16-byte records are
//            read straight from both halves (coalesced);
//   patch    two small kernels apply the patches (read all sources, then write).
// If a level's tails exceed the planned capacity, a sequential per-merge tail (in place on the
// output) runs instead of insert/resolve/patch; the result is the same.
#include "mergeshuffle.h"
#include "ms_common.cuh"
#include "ms_device.cuh"
#include "ms_plan.h"

namespace msk {
namespace {

constexpr int kThreads = 256;
constexpr unsigned long long kEmptyKey = ~0ull;

struct LevelArgs {
  const void *in;
  void *out;
  uint64_t n;
  uint2 key;
  uint32_t c;
  uint32_t level;
  uint32_t M;
  uint32_t J;
  uint32_t kcap;
  uint32_t hbits;
  uint32_t flags;
  uint32_t *zc;
  uint4 *minfo;  // per merge: {T, Z_T, tail offset, tail length}
  uint32_t *ctrl;  // [0] tail steps of the level, [1] 1 = sequential-tail fallback
  uint32_t *mv;
  unsigned long long *hkeys;
  uint32_t *hvals;
  uint32_t *pdst;
  uint32_t *psrc;
  void *ptmp;
  uint32_t *ostart;        // first merge of every 1024 tail steps (kscan), then a sentinel
  uint8_t *zb;             // optional: zero coins per 128-step block (count_kernel)
  const uint32_t *gate;    // optional: the kernel runs only if (*gate != 0) == gate_on
  uint32_t gate_on;
  void *out_alt;           // optional: tails and patches act on out_alt when *alt_sel != 0
  const uint32_t *alt_sel;
  uint2 *laps;             // literal merge: per merge, lcap entries (lap start, zeros before it)
  uint32_t lcap;
  uint2 *ctab;             // literal merge: per coin word (128 a chunk), the word and the zeros
                           // of the chunk's earlier words (count_kernel)
};

__device__ __forceinline__ bool gated_off(const LevelArgs &a) {
  return a.gate != nullptr && ((*a.gate != 0u) != (a.gate_on != 0u));
}
template <typename E>
__device__ __forceinline__ E *target_of(const LevelArgs &a) {
  return static_cast<E *>((a.alt_sel != nullptr && *a.alt_sel != 0u) ? a.out_alt : a.out);
}

struct MergeBounds {
  uint64_t s, mid, e;
};

__device__ __forceinline__ MergeBounds merge_bounds(const LevelArgs &a, uint32_t r) {
  const uint64_t L0 = static_cast<uint64_t>(r) << (a.level + 1u);
  MergeBounds b;
  b.s = boundary(a.n, a.c, L0);
  b.mid = boundary(a.n, a.c, L0 + (1ull << a.level));
  b.e = boundary(a.n, a.c, L0 + (2ull << a.level));
  return b;
}

// zeros among the coins of steps [128*blk, 128*blk+128) that are below N
__device__ __forceinline__ uint32_t block_zero_count(const uint4 &c, uint32_t blk, uint32_t N) {
  const uint64_t base = 128ull * blk;
  if (base >= N) return 0u;
  const uint32_t valid = static_cast<uint32_t>((N - base < 128ull ? N - base : 128ull));
  uint32_t z = 0;
  z += __popc(~c.x & low_mask(min(valid, 32u)));
  z += __popc(~c.y & low_mask(valid > 32u ? min(valid - 32u, 32u) : 0u));
  z += __popc(~c.z & low_mask(valid > 64u ? min(valid - 64u, 32u) : 0u));
  z += __popc(~c.w & low_mask(valid > 96u ? valid - 96u : 0u));
  return z;
}

// chunks of kChunk steps in N steps (N may be close to 2^32: no rounding sum)
__device__ __forceinline__ uint32_t chunks_of(uint32_t N) {
  return N / kChunk + ((N % kChunk) ? 1u : 0u);
}

// ---------------------------------------------------------------------------- count ---------
__global__ void __launch_bounds__(kThreads) count_kernel(LevelArgs a) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nchunks = static_cast<uint64_t>(a.M) * a.J;
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (kThreads / 32);
  for (uint64_t cid = (static_cast<uint64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
       cid < nchunks; cid += warps) {
    const uint32_t r = static_cast<uint32_t>(cid / a.J);
    const uint32_t j = static_cast<uint32_t>(cid - static_cast<uint64_t>(r) * a.J);
    const MergeBounds mb = merge_bounds(a, r);
    const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
    const uint32_t blk = j * (kChunk / 128u) + lane;
    uint32_t z = 0;
    uint4 c = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
    if (128ull * blk < N) {
      c = coin_block(a.key, a.level, r, blk);
      z = block_zero_count(c, blk, N);
    }
    if (a.zb) a.zb[cid * 32u + lane] = static_cast<uint8_t>(z);  // z <= 128
    if (a.ctab) {
      // the block's words with the zeros of the chunk's earlier words (whole words: a query at
      // step x < N counts only words below x)
      const uint32_t w4[4] = {c.x, c.y, c.z, c.w};
      uint32_t zw4[4], zs = 0;
#pragma unroll
      for (uint32_t k = 0; k < 4u; ++k) {
        zw4[k] = static_cast<uint32_t>(__popc(~w4[k]));
        zs += zw4[k];
      }
      uint32_t ex = warp_inclusive_scan(zs) - zs;
      uint2 *const t = a.ctab + cid * 128u + 4u * lane;
#pragma unroll
      for (uint32_t k = 0; k < 4u; ++k) {
        t[k] = make_uint2(w4[k], ex);
        ex += zw4[k];
      }
    }
    z = warp_sum(z);
    if (lane == 0) a.zc[cid] = z;
  }
}

// ---------------------------------------------------------------------------- scan + T ------
// Position (merge-relative step) of the rank-th zero (want_one = 0) or one (want_one = 1) inside
// chunk j; executed by one full warp.
__device__ uint32_t locate_in_chunk(const LevelArgs &a, uint32_t r, uint32_t j, uint32_t N,
                                    uint32_t rank, bool want_one) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t blk = j * (kChunk / 128u) + lane;
  uint4 c = make_uint4(0, 0, 0, 0);
  uint32_t cnt = 0;
  if (128ull * blk < N) {
    c = coin_block(a.key, a.level, r, blk);
    const uint32_t z = block_zero_count(c, blk, N);
    const uint32_t valid = static_cast<uint32_t>((N - 128ull * blk < 128ull ? N - 128ull * blk : 128ull));
    cnt = want_one ? valid - z : z;
  }
  const uint32_t incl = warp_inclusive_scan(cnt);
  const uint32_t excl = incl - cnt;
  uint32_t found = kNone;
  if (cnt > 0 && excl <= rank && rank < incl) {
    uint32_t k = rank - excl;
    const uint32_t words[4] = {c.x, c.y, c.z, c.w};
    const uint32_t valid = static_cast<uint32_t>((N - 128ull * blk < 128ull ? N - 128ull * blk : 128ull));
    for (uint32_t wi = 0; wi < 4u; ++wi) {
      const uint32_t vbits = valid > 32u * wi ? min(valid - 32u * wi, 32u) : 0u;
      const uint32_t m = (want_one ? words[wi] : ~words[wi]) & low_mask(vbits);
      const uint32_t pc = __popc(m);
      if (k < pc) {
        found = 128u * blk + 32u * wi + select_set_bit(m, k);
        break;
      }
      k -= pc;
    }
  }
  // exactly one lane found it
  const unsigned ball = __ballot_sync(kFullMask, found != kNone);
  return __shfl_sync(kFullMask, found, __ffs(static_cast<int>(ball)) - 1);
}

__global__ void __launch_bounds__(kThreads) scan_kernel(LevelArgs a) {
  __shared__ uint32_t scratch[33];
  __shared__ uint32_t s_zchunk, s_zrank, s_ochunk, s_orank, s_tz, s_to;
  constexpr uint32_t kPer = 8;
  for (uint32_t r = blockIdx.x; r < a.M; r += gridDim.x) {
    const MergeBounds mb = merge_bounds(a, r);
    const uint32_t n1 = static_cast<uint32_t>(mb.mid - mb.s);
    const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
    const uint32_t n2 = N - n1;
    const uint32_t J = chunks_of(N);  // chunks of this merge (<= a.J)
    uint32_t *zc = a.zc + static_cast<uint64_t>(r) * a.J;
    if (threadIdx.x == 0) {
      s_zchunk = kNone;
      s_ochunk = kNone;
    }
    __syncthreads();
    uint32_t carry = 0;
    for (uint32_t base = 0; base < J; base += kThreads * kPer) {
      const uint32_t j0 = base + threadIdx.x * kPer;
      uint32_t v[kPer];
      uint32_t local = 0;
#pragma unroll
      for (uint32_t k = 0; k < kPer; ++k) {
        v[k] = (j0 + k < J) ? zc[j0 + k] : 0u;
        local += v[k];
      }
      uint32_t total;
      uint32_t excl = carry + block_exclusive_scan(local, scratch, &total);
#pragma unroll
      for (uint32_t k = 0; k < kPer; ++k) {
        const uint32_t j = j0 + k;
        if (j < J) {
          zc[j] = excl;  // zeros before chunk j
          const uint32_t len = min(kChunk, N - j * kChunk);
          const uint32_t ones = len - v[k];
          const uint32_t Ob = j * kChunk - excl;
          if (excl <= n1 && n1 < excl + v[k]) {
            s_zchunk = j;
            s_zrank = n1 - excl;
          }
          if (Ob <= n2 && n2 < Ob + ones) {
            s_ochunk = j;
            s_orank = n2 - Ob;
          }
        }
        excl += v[k];
      }
      carry += total;
    }
    __syncthreads();
    const uint32_t warp = threadIdx.x >> 5;
    if (warp == 0) {
      const uint32_t t = (s_zchunk == kNone) ? kNone
                                             : locate_in_chunk(a, r, s_zchunk, N, s_zrank, false);
      if ((threadIdx.x & 31u) == 0) s_tz = t;
    } else if (warp == 1) {
      const uint32_t t = (s_ochunk == kNone) ? kNone
                                             : locate_in_chunk(a, r, s_ochunk, N, s_orank, true);
      if ((threadIdx.x & 31u) == 0) s_to = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t T = N, ZT = n1;
      if (s_tz != kNone && s_tz < T) {
        T = s_tz;
        ZT = n1;
      }
      if (s_to != kNone && s_to < T) {
        T = s_to;
        ZT = T - n2;
      }
      a.minfo[r] = make_uint4(T, ZT, 0u, N - T);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------- kscan ---------
__global__ void __launch_bounds__(1024) kscan_kernel(LevelArgs a) {
  __shared__ uint32_t scratch[33];
  uint32_t carry = 0;
  for (uint32_t base = 0; base < a.M; base += 1024u) {
    const uint32_t r = base + threadIdx.x;
    const uint32_t k = r < a.M ? a.minfo[r].w : 0u;
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(k, scratch, &total);
    if (r < a.M) {
      const uint32_t koff = carry + excl;
      a.minfo[r].z = koff;
      // merge r owns the tail steps [koff, koff + k): record it for every 1024-step block that
      // starts inside (within the capacity; beyond it the level runs its tails in order)
      for (uint32_t b = (koff + 1023u) >> 10; 1024ull * b < koff + k && 1024ull * b < a.kcap; ++b)
        a.ostart[b] = r;
    }
    carry += total;
  }
  if (threadIdx.x == 0) {
    a.ctrl[0] = carry;
    a.ctrl[1] = (carry > a.kcap || (a.flags & 1u)) ? 1u : 0u;
    if (carry <= a.kcap) a.ostart[(carry + 1023u) >> 10] = a.M - 1u;  // sentinel
  }
}

// ---------------------------------------------------------------------------- tails ---------
__device__ __forceinline__ uint32_t hash_slot(unsigned long long key, uint32_t hbits) {
  return static_cast<uint32_t>((key * 0x9E3779B97F4A7C15ull) >> (64u - hbits));
}

__device__ __forceinline__ unsigned long long tail_key(uint32_t r, uint32_t pos) {
  return (static_cast<unsigned long long>(r) << 32) | pos;
}

// merge owning tail step g: the largest r whose tail offset is <= g (offsets are
// non-decreasing; merges with an empty tail share their successor's offset and are skipped)
__device__ __forceinline__ uint32_t owner_merge(const LevelArgs &a, uint32_t g) {
  // the owner lies between the owners of the 1024-step block starts around g (kscan's table)
  uint32_t lo = min(a.ostart[g >> 10], a.M - 1u);
  uint32_t hi = min(a.ostart[(g >> 10) + 1u] + 1u, a.M);
  if (hi <= lo) hi = a.M;
  // invariant: offset[lo] <= g, and offset[hi] > g or hi == M
  while (hi - lo > 1u) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a.minfo[mid].z <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads) tail_insert_kernel(LevelArgs a) {
  if (a.ctrl[1]) return;
  const uint32_t K = a.ctrl[0];
  const uint32_t hmask = (1u << a.hbits) - 1u;
  for (uint32_t g = blockIdx.x * kThreads + threadIdx.x; g < K; g += gridDim.x * kThreads) {
    const uint32_t r = owner_merge(a, g);
    const uint4 mi = a.minfo[r];
    const uint32_t i = mi.x + (g - mi.z);
    uint32_t m;
    if (a.flags & MS_FLAG_FDR) {
      uint32_t nb;
      m = draw_fdr(a.key, kTagTail, a.level, r, i, i + 1u, &nb);
    } else {
      m = draw_uniform(a.key, kTagTail, a.level, r, i, i + 1u);
    }
    a.mv[g] = m;
    const unsigned long long key = tail_key(r, m);
    uint32_t h = hash_slot(key, a.hbits);
    for (uint32_t probe = 0; probe <= hmask; ++probe) {
      const unsigned long long old = atomicCAS(&a.hkeys[h], kEmptyKey, key);
      if (old == kEmptyKey) {
        a.hvals[h] = i;
        break;
      }
      h = (h + 1u) & hmask;
    }
  }
}

// smallest tail step > after that targets (r, pos); kNone if there is none
__device__ __forceinline__ uint32_t next_writer(const LevelArgs &a, uint32_t r, uint32_t pos,
                                                uint32_t after) {
  const uint32_t hmask = (1u << a.hbits) - 1u;
  const unsigned long long key = tail_key(r, pos);
  uint32_t best = kNone;
  uint32_t h = hash_slot(key, a.hbits);
  for (uint32_t probe = 0; probe <= hmask; ++probe) {
    const unsigned long long k = a.hkeys[h];
    if (k == kEmptyKey) break;
    if (k == key) {
      const uint32_t v = a.hvals[h];
      if (v > after && v < best) best = v;
    }
    h = (h + 1u) & hmask;
  }
  return best;
}

__device__ __forceinline__ bool has_earlier_writer(const LevelArgs &a, uint32_t r, uint32_t pos,
                                                   uint32_t before) {
  const uint32_t hmask = (1u << a.hbits) - 1u;
  const unsigned long long key = tail_key(r, pos);
  uint32_t h = hash_slot(key, a.hbits);
  for (uint32_t probe = 0; probe <= hmask; ++probe) {
    const unsigned long long k = a.hkeys[h];
    if (k == kEmptyKey) return false;
    if (k == key && a.hvals[h] < before) return true;
    h = (h + 1u) & hmask;
  }
  return false;
}

// follow an element from position pos at time `time` through all later insertions
__device__ __forceinline__ uint32_t final_position(const LevelArgs &a, uint32_t r, uint32_t pos,
                                                   uint32_t time) {
  for (;;) {
    const uint32_t nx = next_writer(a, r, pos, time);
    if (nx == kNone) return pos;
    pos = nx;
    time = nx;
  }
}

__global__ void __launch_bounds__(kThreads) tail_resolve_kernel(LevelArgs a) {
  if (a.ctrl[1]) return;
  const uint32_t K = a.ctrl[0];
  for (uint32_t g = blockIdx.x * kThreads + threadIdx.x; g < K; g += gridDim.x * kThreads) {
    const uint32_t r = owner_merge(a, g);
    const uint4 mi = a.minfo[r];
    const uint32_t T = mi.x;
    const uint32_t i = T + (g - mi.z);
    const uint32_t m = a.mv[g];
    const uint32_t s = static_cast<uint32_t>(merge_bounds(a, r).s);
    // the element that sat at position i before the insertions lands at m at time i
    const uint32_t f = final_position(a, r, m, i);
    a.pdst[g] = (f != i) ? s + f : kNone;
    a.psrc[g] = s + i;
    // the element that sat at m < T moves at the first insertion that targets m
    uint32_t dst2 = kNone;
    if (m < T && !has_earlier_writer(a, r, m, i)) dst2 = s + final_position(a, r, i, i);
    a.pdst[a.kcap + g] = dst2;
    a.psrc[a.kcap + g] = s + m;
  }
}

template <typename E>
__global__ void __launch_bounds__(kThreads) patch_read_kernel(LevelArgs a) {
  if (a.ctrl[1]) return;
  const uint32_t K = a.ctrl[0];
  const E *out = target_of<E>(a);
  E *tmp = static_cast<E *>(a.ptmp);
  for (uint32_t g = blockIdx.x * kThreads + threadIdx.x; g < 2u * K; g += gridDim.x * kThreads) {
    const uint32_t p = g < K ? g : a.kcap + (g - K);
    if (a.pdst[p] != kNone) tmp[p] = out[a.psrc[p] < a.n ? a.psrc[p] : 0u];
  }
}

template <typename E>
__global__ void __launch_bounds__(kThreads) patch_write_kernel(LevelArgs a) {
  if (a.ctrl[1]) return;
  const uint32_t K = a.ctrl[0];
  E *out = target_of<E>(a);
  const E *tmp = static_cast<const E *>(a.ptmp);
  for (uint32_t g = blockIdx.x * kThreads + threadIdx.x; g < 2u * K; g += gridDim.x * kThreads) {
    const uint32_t p = g < K ? g : a.kcap + (g - K);
    const uint32_t d = a.pdst[p];
    if (d != kNone && d < a.n) out[d] = tmp[p];
  }
}

// fallback: Algorithm 3's second loop as printed, one thread per merge, in place
template <typename E>
__global__ void __launch_bounds__(kThreads) tail_sequential_kernel(LevelArgs a) {
  if (!a.ctrl[1]) return;
  E *out = target_of<E>(a);
  for (uint32_t r = blockIdx.x * kThreads + threadIdx.x; r < a.M; r += gridDim.x * kThreads) {
    const uint4 mi = a.minfo[r];
    const MergeBounds mb = merge_bounds(a, r);
    const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
    E *c = out + mb.s;
    DrawMemo memo;
    for (uint32_t i = mi.x; i < N; ++i) {
      uint32_t m, nb;
      if (a.flags & MS_FLAG_FDR) m = draw_fdr(a.key, kTagTail, a.level, r, i, i + 1u, &nb);
      else m = draw_uniform(a.key, kTagTail, a.level, r, i, i + 1u, memo);
      const E t = c[i];
      c[i] = c[m];
      c[m] = t;
    }
  }
}

// ---------------------------------------------------------------------------- gather --------
template <typename E>
__global__ void __launch_bounds__(kThreads) gather_kernel(LevelArgs a) {
  __shared__ uint32_t cw[kChunk / 32u];
  __shared__ uint32_t zw[kChunk / 32u];
  __shared__ uint32_t scratch[33];
  if (gated_off(a)) return;
  const E *__restrict__ in = static_cast<const E *>(a.in);
  E *__restrict__ out = static_cast<E *>(a.out);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  const uint64_t nchunks = static_cast<uint64_t>(a.M) * a.J;
  for (uint64_t cid = blockIdx.x; cid < nchunks; cid += gridDim.x) {
    const uint32_t r = static_cast<uint32_t>(cid / a.J);
    const uint32_t j = static_cast<uint32_t>(cid - static_cast<uint64_t>(r) * a.J);
    const MergeBounds mb = merge_bounds(a, r);
    const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
    const uint32_t t0 = j * kChunk;
    if (t0 >= N) continue;  // uniform across the CTA
    const uint32_t t1 = t0 + min(kChunk, N - t0);  // (t0 < N; no 32-bit overflow)
    const uint4 mi = a.minfo[r];
    const uint32_t T = mi.x;
    const uint32_t n1 = static_cast<uint32_t>(mb.mid - mb.s);
    const uint32_t Z0 = a.zc[cid];
    const bool first_exhausted = (mi.y == n1);
    if (threadIdx.x < kChunk / 128u) {
      const uint32_t blk = j * (kChunk / 128u) + threadIdx.x;
      const uint4 c = coin_block(a.key, a.level, r, blk);
      cw[4u * threadIdx.x + 0u] = c.x;
      cw[4u * threadIdx.x + 1u] = c.y;
      cw[4u * threadIdx.x + 2u] = c.z;
      cw[4u * threadIdx.x + 3u] = c.w;
    }
    __syncthreads();
    // zeros per 32-step word, exclusive prefix inside the chunk (threads 0..127 own one word)
    {
      uint32_t z = 0;
      if (threadIdx.x < kChunk / 32u) {
        const uint32_t tw = t0 + 32u * threadIdx.x;
        const uint32_t valid = tw >= N ? 0u : min(32u, N - tw);
        z = __popc(~cw[threadIdx.x] & low_mask(valid));
      }
      uint32_t total;
      const uint32_t excl = block_exclusive_scan(z, scratch, &total);
      if (threadIdx.x < kChunk / 32u) zw[threadIdx.x] = excl;
    }
    __syncthreads();
    const E *A = in + mb.s;  // the second half starts at A + n1
    E *C = out + mb.s;
    // Warp w owns coin words w, w+8, ...; lane L places step 32u + L of word u, so each store
    // instruction writes 32 consecutive elements. All loads of a batch are issued before any
    // store, keeping kBatch independent loads in flight per thread.
    constexpr uint32_t kWarps = kThreads / 32;
    constexpr uint32_t kWordsPerWarp = kChunk / 32u / kWarps;
    constexpr uint32_t kBatch = sizeof(E) >= 16 ? 8u : 16u;
#pragma unroll
    for (uint32_t b0 = 0; b0 < kWordsPerWarp; b0 += kBatch) {
      E v[kBatch];
#pragma unroll
      for (uint32_t k = 0; k < kBatch; ++k) {
        const uint32_t u = warp + (b0 + k) * kWarps;
        const uint32_t t = t0 + 32u * u + lane;
        if (t < t1) {
          // source index inside the merge; the clamp keeps every load inside [s, e) even if
          // the plan were inconsistent (parity tests would then fail instead of a load faulting)
          uint32_t src;
          if (t < T) {
            const uint32_t word = cw[u];
            const uint32_t Z = Z0 + zw[u] + __popc(~word & low_mask(lane));
            src = ((word >> lane) & 1u) ? n1 + (t - Z) : Z;
          } else if (first_exhausted) {
            src = t;
          } else {
            src = t - (N - n1);
          }
          v[k] = A[min(src, N - 1u)];
        }
      }
#pragma unroll
      for (uint32_t k = 0; k < kBatch; ++k) {
        const uint32_t t = t0 + 32u * (warp + (b0 + k) * kWarps) + lane;
        if (t < t1) C[t] = v[k];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ staged gather (w <= 8) --
// The same data pass for 4- and 8-byte elements, one CTA per 4096-step chunk. The chunk's
// outputs read one contiguous run of each half: its zeros from the first half and its ones from
// the second, and after the break step the rest of the half that did not run out. The runs'
// bounds follow from the chunk's zero prefix and the merge's break step alone, so both runs are
// copied into shared memory with 16-byte asynchronous copies while the chunk's coins are
// generated. Each thread then places eight consecutive outputs, walking one index per run
// (past the break step the coin is replaced by the half that did not run out), and stores them
// as 16-byte vectors aligned to the output.
constexpr uint32_t kStageGroup = 8;  // outputs per thread group
constexpr uint32_t kStageThreads = 128;  // (16 CTAs an SM: more chunks in flight than 256)

// copies n elements from global src to shared dst (dst at src's 16-byte phase)
template <typename E>
__device__ __forceinline__ void stage_run(E *dst, const E *src, uint32_t n) {
  constexpr uint32_t kV = 16u / sizeof(E);
  const uint32_t ph = static_cast<uint32_t>((reinterpret_cast<uintptr_t>(src) & 15u) / sizeof(E));
  const uint32_t head = min(n, (kV - ph) % kV);
  const uint32_t body = (n - head) / kV;
  const uint32_t tail0 = head + body * kV;
  const uint32_t tid = threadIdx.x;
  if (tid < head) cp_async_elem(dst + tid, src + tid);
  for (uint32_t c = tid; c < body; c += kStageThreads)
    cp_async_elem(reinterpret_cast<uint4 *>(dst + head) + c,
                  reinterpret_cast<const uint4 *>(src + head) + c);
  if (tid < n - tail0) cp_async_elem(dst + tail0 + tid, src + tail0 + tid);
}

template <typename E>
__global__ void __launch_bounds__(kStageThreads) gather_staged_kernel(LevelArgs a) {
  constexpr uint32_t kV = 16u / sizeof(E);      // elements per 16 bytes
  // both runs with their 16-byte phases (at most kChunk + 3 kV - 2 entries), plus one group of
  // slack so that a clamped walk of eight steps stays inside
  constexpr uint32_t kBuf = kChunk + 4u * kV + kStageGroup;
  __shared__ __align__(16) E sbuf[kBuf];
  __shared__ uint32_t cw[kChunk / 32u + 1u];
  __shared__ uint32_t zw[kChunk / 32u];
  if (gated_off(a)) return;
  const E *__restrict__ in = static_cast<const E *>(a.in);
  E *__restrict__ out = static_cast<E *>(a.out);
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint64_t nchunks = static_cast<uint64_t>(a.M) * a.J;
  for (uint64_t cid = blockIdx.x; cid < nchunks; cid += gridDim.x) {
    const uint32_t r = static_cast<uint32_t>(cid / a.J);
    const uint32_t j = static_cast<uint32_t>(cid - static_cast<uint64_t>(r) * a.J);
    const MergeBounds mb = merge_bounds(a, r);
    const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
    const uint32_t t0 = j * kChunk;
    if (t0 >= N) continue;  // uniform across the CTA
    const uint32_t t1 = t0 + min(kChunk, N - t0);  // (t0 < N; no 32-bit overflow)
    const uint32_t len = t1 - t0;
    const uint4 mi = a.minfo[r];
    const uint32_t T = mi.x;
    const uint32_t n1 = static_cast<uint32_t>(mb.mid - mb.s);
    const uint32_t n2 = N - n1;
    const bool a_out = (mi.y == n1);  // the first half ran out at T (or T = N)
    // chunk-relative break step, zeros before it, and the two runs (half-relative start, size)
    uint32_t Tc, zT, za, na, ob, nb;
    if (t0 >= T) {
      Tc = 0;
      zT = 0;
      za = a_out ? 0u : t0 - n2;
      ob = a_out ? t0 - n1 : 0u;
      na = a_out ? 0u : len;
      nb = a_out ? len : 0u;
    } else {
      const uint32_t Z0 = a.zc[cid];
      Tc = min(t1, T) - t0;
      const uint32_t Jr = chunks_of(N);
      zT = (t1 <= T) ? ((j + 1u < Jr) ? a.zc[cid + 1] - Z0 : n1 - Z0) : mi.y - Z0;
      za = Z0;
      ob = t0 - Z0;
      na = zT + (a_out ? 0u : len - Tc);
      nb = (Tc - zT) + (a_out ? len - Tc : 0u);
    }
    // (the runs stay inside their halves even for an inconsistent plan)
    za = min(za, n1);
    na = min(na, n1 - za);
    ob = min(ob, n2);
    nb = min(nb, n2 - ob);
    const E *const srcA = in + mb.s + za;
    const E *const srcB = in + mb.mid + ob;
    const uint32_t offA = static_cast<uint32_t>((reinterpret_cast<uintptr_t>(srcA) & 15u) / sizeof(E));
    const uint32_t offB = ((offA + na + kV - 1u) / kV) * kV +
                          static_cast<uint32_t>((reinterpret_cast<uintptr_t>(srcB) & 15u) / sizeof(E));
    stage_run(sbuf + offA, srcA, min(na, kBuf - offA));
    stage_run(sbuf + offB, srcB, min(nb, kBuf - min(offB, kBuf)));
    cp_async_commit();
    // coins of steps [t0, t0 + Tc) and the zeros before each of their words (warp 0)
    if (tid < 32u) {
      const uint32_t nwords = (Tc + 31u) >> 5;
      if (4u * lane < nwords) {
        const uint4 c = coin_block(a.key, a.level, r, j * (kChunk / 128u) + lane);
        cw[4u * lane + 0u] = c.x;
        cw[4u * lane + 1u] = c.y;
        cw[4u * lane + 2u] = c.z;
        cw[4u * lane + 3u] = c.w;
      }
      __syncwarp();
      uint32_t z4[4], zs = 0;
#pragma unroll
      for (uint32_t k = 0; k < 4u; ++k) {
        z4[k] = (4u * lane + k < nwords) ? static_cast<uint32_t>(__popc(~cw[4u * lane + k])) : 0u;
        zs += z4[k];
      }
      uint32_t ex = warp_inclusive_scan(zs) - zs;
#pragma unroll
      for (uint32_t k = 0; k < 4u; ++k) {
        zw[4u * lane + k] = ex;
        ex += z4[k];
      }
    }
    cp_async_wait<0>();
    __syncthreads();
    // groups of eight outputs aligned to 16 bytes of the output (group 0: the head before the
    // first aligned one)
    E *const C = out + mb.s + t0;
    const uint32_t cph = static_cast<uint32_t>((reinterpret_cast<uintptr_t>(C) & 15u) / sizeof(E));
    const uint32_t hd = min(len, (kV - cph) % kV);
    const uint32_t ngroups = 1u + (len - hd + kStageGroup - 1u) / kStageGroup;
    const uint32_t abit = a_out ? 1u : 0u;
    for (uint32_t gi = tid; gi < ngroups; gi += kStageThreads) {
      const uint32_t p0 = gi == 0u ? 0u : hd + kStageGroup * (gi - 1u);
      const uint32_t cnt = gi == 0u ? hd : min(kStageGroup, len - p0);
      if (cnt == 0u) continue;
      uint32_t pa, pb, bits;
      if (p0 < Tc) {
        const uint32_t u = p0 >> 5, sh = p0 & 31u;
        const uint32_t w0 = cw[u];
        pa = zw[u] + static_cast<uint32_t>(__popc(~w0 & low_mask(sh)));
        pb = p0 - pa;
        bits = __funnelshift_r(w0, cw[u + 1u], sh);  // coins of p0 .. p0+31
      } else {
        pa = zT + (p0 - Tc) * (1u - abit);
        pb = (Tc - zT) + (p0 - Tc) * abit;
        bits = 0u;
      }
      // (the walk stays inside the buffer even for an inconsistent plan)
      pa = min(offA + pa, kBuf - kStageGroup);
      pb = min(offB + pb, kBuf - kStageGroup);
      E v[kStageGroup];
      if (p0 + kStageGroup <= Tc) {
#pragma unroll
        for (uint32_t i = 0; i < kStageGroup; ++i) {
          const uint32_t bit = (bits >> i) & 1u;
          v[i] = sbuf[bit ? pb : pa];
          pa += bit ^ 1u;
          pb += bit;
        }
      } else {
#pragma unroll
        for (uint32_t i = 0; i < kStageGroup; ++i) {
          const uint32_t bit = (p0 + i < Tc) ? ((bits >> i) & 1u) : abit;
          v[i] = sbuf[bit ? pb : pa];
          pa += bit ^ 1u;
          pb += bit;
        }
      }
      if (gi != 0u && cnt == kStageGroup) {
        uint4 *const dst = reinterpret_cast<uint4 *>(C + p0);
#pragma unroll
        for (uint32_t q = 0; q < kStageGroup / kV; ++q) {
          uint4 o;
          if constexpr (sizeof(E) == 4) {
            o = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else {
            o = make_uint4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
          }
          dst[q] = o;
        }
      } else {
#pragma unroll
        for (uint32_t i = 0; i < kStageGroup; ++i)
          if (i < cnt) C[p0 + i] = v[i];
      }
    }
    __syncthreads();  // the staging buffer is reused by the next chunk
  }
}

// zeros among the coins of steps [0, x) of merge r, x <= N (zb and the scanned zc)
__device__ uint32_t zeros_before(const LevelArgs &a, uint32_t r, uint32_t x) {
  uint32_t chunk = x / kChunk;
  if (chunk >= a.J) chunk = a.J - 1u;  // x = N on a chunk boundary: the whole last chunk
  const uint64_t cid = static_cast<uint64_t>(r) * a.J + chunk;
  uint32_t Z = a.zc[cid];
  const uint32_t rel = min(x - chunk * kChunk, kChunk);
  const uint32_t nb = rel >> 7;  // whole 128-step blocks before x (their counts: 32 bytes read
                                 // as two vectors, the first nb bytes summed)
  {
    const uint4 *zb4 = reinterpret_cast<const uint4 *>(a.zb + cid * 32u);
    const uint4 lo = zb4[0], hi = zb4[1];
    const uint32_t w8[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (uint32_t k = 0; k < 8u; ++k) {
      const uint32_t keep = nb >= 4u * k + 4u ? 4u : (nb > 4u * k ? nb - 4u * k : 0u);
      const uint32_t m = keep >= 4u ? 0xFFFFFFFFu : ((1u << (8u * keep)) - 1u);
      Z += __vsadu4(w8[k] & m, 0u);  // sum of the kept bytes
    }
  }
  const uint32_t q = rel & 127u;
  if (q != 0u && nb < 32u) {
    const uint4 c = coin_block(a.key, a.level, r, chunk * 32u + nb);
    const uint32_t w4[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (uint32_t k = 0; k < 4u; ++k) {
      const uint32_t lo = 32u * k;
      if (q > lo) Z += __popc(~w4[k] & low_mask(min(q - lo, 32u)));
    }
  }
  return Z;
}

// ---------------------------------------------------------------------------- fused pairs --
// Two consecutive levels l, l+1 in one data pass. Level l's output (never written) is the
// stable interleave of its halves with the tail moves applied; a tail move is an exception:
// output position q holds the interleave element of merge position F(q) != q. The plan lists,
// for every exception in position order, the input index that element comes from: a bitmap
// marks the exception positions, and the rank of an exception (exceptions at lower positions)
// is its index in the list. Ranks come from a two-level prefix of the bitmap's bit counts
// (per 1024 positions within their tile of 2^17 positions, and per tile), so a data chunk finds
// its range's exceptions as one contiguous slice of the list. The data pass then gathers level
// l+1's interleave straight from level l's input.

struct ExcArgs {
  uint32_t *bits;  // one bit per element of level l's output
  uint32_t *src;   // input index of each tail patch's element (by patch)
  uint32_t *val;   // input index of each exception's element (by rank)
  uint32_t *bpre;  // exceptions before each block of kXBlock positions, within its tile
  uint32_t *tpre;  // exceptions before each tile of kXTileBlocks blocks
  uint64_t n;
};

// Exceptions at positions below q (q < n): the block and tile prefixes plus the bits of q's
// block before it. The block's 32 bitmap words arrive as eight 16-byte loads.
__device__ __forceinline__ uint32_t exception_rank(const ExcArgs &x, uint32_t q) {
  const uint32_t b = q / kXBlock;
  uint32_t rank = x.tpre[b / kXTileBlocks] + x.bpre[b];
  const uint4 *const w4 = reinterpret_cast<const uint4 *>(x.bits + static_cast<uint64_t>(b) * 32u);
  const uint64_t nwords = (x.n + 31u) >> 5;
  const uint32_t wq = (q >> 5) & 31u;  // q's word within the block
  uint4 v[8];
#pragma unroll
  for (uint32_t k = 0; k < 8u; ++k)
    v[k] = (static_cast<uint64_t>(b) * 32u + 4u * k < nwords) ? w4[k] : make_uint4(0, 0, 0, 0);
#pragma unroll
  for (uint32_t k = 0; k < 8u; ++k) {
    const uint32_t w[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
    for (uint32_t e = 0; e < 4u; ++e) {
      const uint32_t wi = 4u * k + e;
      const uint32_t m = wi < wq ? 0xFFFFFFFFu : (wi == wq ? low_mask(q & 31u) : 0u);
      rank += static_cast<uint32_t>(__popc(w[e] & m));
    }
  }
  return rank;
}

// Input index (into level l's input) of the interleave element at merge position p of merge r.
__device__ uint32_t interleave_source(const LevelArgs &a, uint32_t r, uint32_t p) {
  const MergeBounds mb = merge_bounds(a, r);
  const uint32_t n1 = static_cast<uint32_t>(mb.mid - mb.s);
  const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
  const uint4 mi = a.minfo[r];
  const uint32_t s = static_cast<uint32_t>(mb.s);
  if (p >= mi.x) return s + ((mi.y == n1) ? p : p - (N - n1));  // leftover, in order
  const uint32_t blk = p >> 7;
  const uint32_t chunk = p >> 12;  // kChunk = 4096 steps = 32 blocks
  const uint64_t cid = static_cast<uint64_t>(r) * a.J + chunk;
  uint32_t Z = a.zc[cid];  // zeros before the chunk (exclusive prefix after the scan)
  {
    // plus the zero counts of the chunk's blocks before blk: 32 bytes read as two vectors
    const uint4 *zb4 = reinterpret_cast<const uint4 *>(a.zb + cid * 32u);
    const uint32_t nb = blk - chunk * 32u;  // bytes to add, < 32
    const uint4 lo = zb4[0], hi = zb4[1];
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (uint32_t k = 0; k < 8u; ++k) {
      const uint32_t keep = nb >= 4u * k + 4u ? 4u : (nb > 4u * k ? nb - 4u * k : 0u);
      const uint32_t m = keep >= 4u ? 0xFFFFFFFFu : ((1u << (8u * keep)) - 1u);
      Z += __vsadu4(w[k] & m, 0u);  // sum of the kept bytes
    }
  }
  const uint4 c = coin_block(a.key, a.level, r, blk);
  const uint32_t q = p & 127u;
  const uint32_t words[4] = {c.x, c.y, c.z, c.w};
  for (uint32_t wi = 0; wi < (q >> 5); ++wi) Z += __popc(~words[wi]);
  const uint32_t word = words[q >> 5];
  Z += __popc(~word & low_mask(q & 31u));
  return s + (((word >> (q & 31u)) & 1u) ? n1 + p - Z : Z);
}

__global__ void __launch_bounds__(kThreads) exceptions_kernel(LevelArgs a, ExcArgs x) {
  if (a.ctrl[1]) return;  // the unfused fallback runs instead
  const uint32_t K = a.ctrl[0];
  for (uint32_t g = blockIdx.x * kThreads + threadIdx.x; g < 2u * K; g += gridDim.x * kThreads) {
    const uint32_t pi = g < K ? g : a.kcap + (g - K);
    const uint32_t dst = a.pdst[pi];
    if (dst == kNone || dst >= a.n) continue;
    const uint32_t r = owner_merge(a, g < K ? g : g - K);
    const uint32_t s = static_cast<uint32_t>(merge_bounds(a, r).s);
    x.src[g] = interleave_source(a, r, a.psrc[pi] - s);
    atomicOr(&x.bits[dst >> 5], 1u << (dst & 31u));
  }
}

// Rank index, first level: CTA t counts the exceptions of the kXTileBlocks blocks of tile t
// (a warp a block: one bitmap word a lane), then writes each block's prefix within the tile
// and the tile's total.
__global__ void __launch_bounds__(kThreads) xcount_kernel(LevelArgs a, ExcArgs x) {
  static_assert(kXTileBlocks <= kThreads, "one block count a thread");
  __shared__ uint32_t cnt[kXTileBlocks];
  __shared__ uint32_t scratch[33];
  if (a.ctrl[1]) return;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint64_t nwords = (x.n + 31u) >> 5;
  const uint64_t nblocks = (x.n + kXBlock - 1u) / kXBlock;
  const uint64_t b0 = static_cast<uint64_t>(blockIdx.x) * kXTileBlocks;
#pragma unroll 4
  for (uint32_t k = warp; k < kXTileBlocks; k += kThreads / 32u) {
    const uint64_t wi = (b0 + k) * 32u + lane;
    const uint32_t c = warp_sum(wi < nwords ? static_cast<uint32_t>(__popc(x.bits[wi])) : 0u);
    if (lane == 0) cnt[k] = c;
  }
  __syncthreads();
  const uint32_t v = tid < kXTileBlocks ? cnt[tid] : 0u;
  uint32_t total;
  const uint32_t ex = block_exclusive_scan(v, scratch, &total);
  if (tid < kXTileBlocks && b0 + tid < nblocks) x.bpre[b0 + tid] = ex;
  if (tid == 0) x.tpre[blockIdx.x] = total;
}

// Rank index, second level: exclusive prefix of the tile totals, in place (one CTA of 1024
// threads, each a run of consecutive tiles: up to 2^32 positions).
__global__ void __launch_bounds__(1024) xtiles_kernel(LevelArgs a, ExcArgs x) {
  __shared__ uint32_t scratch[33];
  if (a.ctrl[1]) return;
  const uint32_t tid = threadIdx.x;
  const uint64_t ntiles = ((x.n + kXBlock - 1u) / kXBlock + kXTileBlocks - 1u) / kXTileBlocks;
  const uint32_t per = static_cast<uint32_t>((ntiles + 1023u) / 1024u);
  const uint64_t t0 = static_cast<uint64_t>(tid) * per;
  uint32_t sum = 0;
  for (uint32_t i = 0; i < per; ++i)
    if (t0 + i < ntiles) sum += x.tpre[t0 + i];
  uint32_t total;
  uint32_t ex = block_exclusive_scan(sum, scratch, &total);
  for (uint32_t i = 0; i < per; ++i) {
    if (t0 + i < ntiles) {
      const uint32_t v = x.tpre[t0 + i];
      x.tpre[t0 + i] = ex;
      ex += v;
    }
  }
}

// Every exception's input index into the list at its rank.
__global__ void __launch_bounds__(kThreads) xscatter_kernel(LevelArgs a, ExcArgs x) {
  if (a.ctrl[1]) return;
  const uint32_t K = a.ctrl[0];
  for (uint32_t g = blockIdx.x * kThreads + threadIdx.x; g < 2u * K; g += gridDim.x * kThreads) {
    const uint32_t pi = g < K ? g : a.kcap + (g - K);
    const uint32_t dst = a.pdst[pi];
    if (dst == kNone || dst >= a.n) continue;
    x.val[exception_rank(x, dst)] = x.src[g];
  }
}

struct PairArgs {
  const void *in;
  void *out;
  LevelArgs l1, l2;  // the two levels' plans (l1.J, zc, zb, minfo; l2.M, J, zc, minfo)
  ExcArgs x;
  uint4 *xr;  // per chunk of level l+1: the ranges its halves read (pair_ranges_kernel)
};

// Exceptions at positions below q, q <= n.
__device__ __forceinline__ uint32_t exception_rank_end(const ExcArgs &x, uint64_t q) {
  if (q < x.n) return exception_rank(x, static_cast<uint32_t>(q));
  const uint32_t last = static_cast<uint32_t>(x.n - 1u);
  return exception_rank(x, last) + ((x.bits[last >> 5] >> (last & 31u)) & 1u);
}

// What one half h of a level-(l+1) chunk reads of merge 2R+h of level l, in 16 words (four
// uint4 of the chunk's record, half 0 first):
constexpr uint32_t kRgLo = 0;     // range start (merge position) and
constexpr uint32_t kRgCnt = 1;    //   length
constexpr uint32_t kRgTc = 2;     // range-relative break step of level l (0 past it)
constexpr uint32_t kRgZT = 3;     // zeros of level l's coins in [lo, lo + Tc)
constexpr uint32_t kRgAbit = 4;   // 1: level l's first half ran out at its break step
constexpr uint32_t kRgBlo = 5;    // first 128-step block of level l's coins the range uses
constexpr uint32_t kRgRunA = 6;   // input index and length of the first half's run,
constexpr uint32_t kRgNa = 7;
constexpr uint32_t kRgRunB = 8;   //   and of the second half's run
constexpr uint32_t kRgNb = 9;
constexpr uint32_t kRgGlo = 10;   // global position of the range start
constexpr uint32_t kRgZlo = 11;   // zeros before lo
constexpr uint32_t kRgXbase = 12; // rank of the range's first exception and
constexpr uint32_t kRgXcnt = 13;  //   the range's exception count
constexpr uint32_t kRgZblk = 14;  // zeros before block blo
constexpr uint32_t kRgMerge = 15; // 2R + h
constexpr uint32_t kRgWords = 16;

// The ranges of every chunk of level l+1, on the plan stream once both levels are planned: a
// thread per chunk and half. Level l+1's chunk [t0, t1) takes positions [lo0, lo0 + cnt0) of
// merge 2R and [lo1, lo1 + cnt1) of merge 2R+1 (its zero coins before t0 and in the chunk); each
// range is the interleave of one run of each half of its merge (up to level l's break step),
// then that merge's leftover.
__global__ void __launch_bounds__(kThreads) pair_ranges_kernel(PairArgs pa) {
  const LevelArgs &a1 = pa.l1;
  const LevelArgs &a2 = pa.l2;
  if (a1.ctrl[1]) return;  // level l's tails overflowed: the unfused fallback runs instead
  const uint64_t nchunks = static_cast<uint64_t>(a2.M) * a2.J;
  for (uint64_t g = static_cast<uint64_t>(blockIdx.x) * kThreads + threadIdx.x; g < 2u * nchunks;
       g += static_cast<uint64_t>(gridDim.x) * kThreads) {
    const uint64_t cid = g >> 1;
    const uint32_t h = static_cast<uint32_t>(g & 1u);
    const uint32_t R = static_cast<uint32_t>(cid / a2.J);
    const uint32_t j = static_cast<uint32_t>(cid - static_cast<uint64_t>(R) * a2.J);
    uint32_t rg[kRgWords] = {};
    const MergeBounds mb2 = merge_bounds(a2, R);
    const uint32_t N2 = static_cast<uint32_t>(mb2.e - mb2.s);
    const uint32_t t0 = j * kChunk;
    rg[kRgMerge] = 2u * R + h;
    if (t0 < N2) {
      const uint32_t t1 = t0 + min(kChunk, N2 - t0);  // (t0 < N2; no 32-bit overflow)
      const uint32_t len = t1 - t0;
      const uint32_t h1 = static_cast<uint32_t>(mb2.mid - mb2.s);
      const uint32_t h2 = N2 - h1;
      const uint4 mi2 = a2.minfo[R];
      const uint32_t T2 = mi2.x;
      const uint32_t abit2 = (mi2.y == h1) ? 1u : 0u;
      uint32_t Tc2, zT2, lo;
      if (t0 >= T2) {
        Tc2 = 0;
        zT2 = 0;
        lo = h ? (abit2 ? t0 - h1 : 0u) : (abit2 ? 0u : t0 - h2);
      } else {
        const uint32_t Z0 = a2.zc[cid];
        Tc2 = min(t1, T2) - t0;
        const uint32_t Jr = chunks_of(N2);
        zT2 = (t1 <= T2) ? ((j + 1u < Jr) ? a2.zc[cid + 1] - Z0 : h1 - Z0) : mi2.y - Z0;
        lo = h ? t0 - Z0 : Z0;
      }
      const uint32_t cnt =
          h ? min((Tc2 - zT2) + (abit2 ? len - Tc2 : 0u), h2 - min(lo, h2))
            : min(zT2 + (abit2 ? 0u : len - Tc2), h1 - min(lo, h1));
      const uint32_t r1 = 2u * R + h;
      const MergeBounds mb1 = merge_bounds(a1, r1);
      const uint32_t N1 = static_cast<uint32_t>(mb1.e - mb1.s);
      const uint32_t n11 = static_cast<uint32_t>(mb1.mid - mb1.s);
      const uint32_t n12 = N1 - n11;
      const uint4 mi1 = a1.minfo[r1];
      const uint32_t T1 = mi1.x;
      const uint32_t abit1 = (mi1.y == n11) ? 1u : 0u;
      const uint32_t qe = min(lo + cnt, T1);  // [lo, qe): interleave positions
      uint32_t Tc1 = 0, zT1 = 0, Zlo = 0, za, na, ob, nb;
      if (lo >= T1) {
        za = abit1 ? 0u : lo - n12;
        ob = abit1 ? lo - n11 : 0u;
        na = abit1 ? 0u : cnt;
        nb = abit1 ? cnt : 0u;
      } else {
        Zlo = zeros_before(a1, r1, lo);
        const uint32_t Zqe = (qe == T1) ? mi1.y : zeros_before(a1, r1, qe);
        Tc1 = qe - lo;
        zT1 = Zqe - Zlo;
        const uint32_t rest = lo + cnt - qe;
        za = Zlo;
        ob = lo - Zlo;
        na = zT1 + (abit1 ? 0u : rest);
        nb = (Tc1 - zT1) + (abit1 ? rest : 0u);
      }
      // (the runs stay inside their halves even for an inconsistent plan)
      za = min(za, n11);
      na = min(na, n11 - za);
      ob = min(ob, n12);
      nb = min(nb, n12 - ob);
      const uint32_t blo = lo >> 7;
      const uint32_t g_lo = static_cast<uint32_t>(mb1.s) + lo;
      rg[kRgLo] = lo;
      rg[kRgCnt] = cnt;
      rg[kRgTc] = Tc1;
      rg[kRgZT] = zT1;
      rg[kRgAbit] = abit1;
      rg[kRgBlo] = blo;
      rg[kRgRunA] = static_cast<uint32_t>(mb1.s) + za;
      rg[kRgNa] = na;
      rg[kRgRunB] = static_cast<uint32_t>(mb1.mid) + ob;
      rg[kRgNb] = nb;
      rg[kRgGlo] = g_lo;
      rg[kRgZlo] = Zlo;
      rg[kRgZblk] = Tc1 ? zeros_before(a1, r1, 128u * blo) : 0u;
      if (cnt) {
        rg[kRgXbase] = exception_rank(pa.x, g_lo);
        rg[kRgXcnt] = exception_rank_end(pa.x, static_cast<uint64_t>(g_lo) + cnt) - rg[kRgXbase];
      }
    }
    uint4 *const o = pa.xr + g * 4u;
#pragma unroll
    for (uint32_t k = 0; k < 4u; ++k)
      o[k] = make_uint4(rg[4u * k], rg[4u * k + 1u], rg[4u * k + 2u], rg[4u * k + 3u]);
  }
}

// half h of level l+1's merge R is merge 2R+h of level l; its used position range in the chunk
// is [lo, lo+cnt); the coin words of level l covering it start at block blo.
constexpr uint32_t kPairW = 136;  // words per half: <= 4096 positions + block alignment

// The bitmap words of global positions [g_lo, g_lo + cnt) into xb (word 0: word g_lo / 32),
// bits outside the range cleared; thread t of nt loads words t, t + nt, ...
__device__ __forceinline__ void load_range_bits(const ExcArgs &x, uint32_t g_lo, uint32_t cnt,
                                                uint32_t *xb, uint32_t t, uint32_t nt) {
  const uint64_t nwords = (x.n + 31u) >> 5;
  const uint32_t w0 = g_lo >> 5;
  const uint32_t nw =
      cnt ? static_cast<uint32_t>((static_cast<uint64_t>(g_lo) + cnt + 31u) >> 5) - w0 : 0u;
  for (uint32_t wi = t; wi < nw && wi < kPairW; wi += nt) {
    const uint64_t bw = static_cast<uint64_t>(w0) + wi;
    uint32_t v = bw < nwords ? x.bits[bw] : 0u;
    const uint32_t ws = (w0 + wi) << 5;  // first position of the word
    const uint32_t lo_b = g_lo > ws ? g_lo - ws : 0u;
    const uint32_t hi_b = static_cast<uint32_t>(
        min(static_cast<uint64_t>(g_lo) + cnt - ws, static_cast<uint64_t>(32u)));
    xb[wi] = v & low_mask(hi_b) & ~low_mask(lo_b);
  }
}

// Exclusive prefix of the bit counts of the nw range words xb into xwp, by one full warp (five
// words a lane); the exception of rank k in the range then sits in the last word whose prefix is
// at most k.
__device__ __forceinline__ void range_word_prefix(const uint32_t *xb, uint32_t nw, uint32_t *xwp) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t c5[5], cs = 0;
#pragma unroll
  for (uint32_t k = 0; k < 5u; ++k) {
    const uint32_t wi = 5u * lane + k;
    c5[k] = wi < nw && wi < kPairW ? static_cast<uint32_t>(__popc(xb[wi])) : 0u;
    cs += c5[k];
  }
  uint32_t ex = warp_inclusive_scan(cs) - cs;
#pragma unroll
  for (uint32_t k = 0; k < 5u; ++k) {
    const uint32_t wi = 5u * lane + k;
    if (wi < kPairW) xwp[wi] = ex;
    ex += c5[k];
  }
}

__device__ __forceinline__ uint32_t range_words(uint32_t g_lo, uint32_t cnt) {
  return cnt ? min(static_cast<uint32_t>((static_cast<uint64_t>(g_lo) + cnt + 31u) >> 5) -
                       (g_lo >> 5),
                   kPairW)
             : 0u;
}

// The data pass of a fused pair for 8- and 16-byte elements: a CTA takes 4096 outputs of level
// l+1 and reads every element straight from level l's input (coalesced within each of the four
// runs). Per chunk: level l+1's coins and zero prefix; the record of the two level-l ranges
// (pair_ranges_kernel); level l's coins over each range, the range's exception bits and its
// slice of the exception list; then each output's source through both levels.
template <typename E>
__global__ void __launch_bounds__(kThreads, 5) pair_gather_kernel(PairArgs pa) {
  __shared__ uint32_t cw2[kChunk / 32u];
  __shared__ uint32_t zw2[kChunk / 32u];
  __shared__ uint32_t cw1[2][kPairW];
  __shared__ uint32_t zw1[2][kPairW];
  __shared__ uint32_t xb1[2][kPairW];  // exception bits of each half's range (word-aligned)
  __shared__ uint32_t xwp[2][kPairW];  // exceptions of the range before each word
  __shared__ uint32_t xval[2][kChunk];   // input index of each exception, by position in range
  __shared__ uint32_t scratch[33];
  // per half: the chunk's record (kRgWords), then s1, n11, T1, the leftover shift, N1, nblk
  constexpr uint32_t kS1 = kRgWords, kN11 = kRgWords + 1u, kT1 = kRgWords + 2u,
                     kShift = kRgWords + 3u, kN1 = kRgWords + 4u, kNblk = kRgWords + 5u;
  __shared__ uint32_t hs[2][kRgWords + 6u];
  const LevelArgs &a1 = pa.l1;
  const LevelArgs &a2 = pa.l2;
  if (a1.ctrl[1]) return;  // level l's tails overflowed: the unfused fallback runs instead
  const E *__restrict__ in = static_cast<const E *>(pa.in);
  E *__restrict__ out = static_cast<E *>(pa.out);
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint32_t warp = tid >> 5;
  const uint64_t nchunks = static_cast<uint64_t>(a2.M) * a2.J;
  for (uint64_t cid = blockIdx.x; cid < nchunks; cid += gridDim.x) {
    const uint32_t R = static_cast<uint32_t>(cid / a2.J);
    const uint32_t j = static_cast<uint32_t>(cid - static_cast<uint64_t>(R) * a2.J);
    const MergeBounds mb2 = merge_bounds(a2, R);
    const uint32_t N2 = static_cast<uint32_t>(mb2.e - mb2.s);
    const uint32_t t0 = j * kChunk;
    if (t0 >= N2) continue;  // uniform across the CTA
    const uint32_t t1 = t0 + min(kChunk, N2 - t0);  // (t0 < N2; no 32-bit overflow)
    const uint32_t h1 = static_cast<uint32_t>(mb2.mid - mb2.s);  // level l+1's first half
    const uint32_t h2 = N2 - h1;
    const uint4 mi2 = a2.minfo[R];
    const uint32_t T2 = mi2.x;
    const bool first_exh2 = (mi2.y == h1);
    const uint32_t Z0 = a2.zc[cid];
    const uint32_t tA = min(t1, T2);  // [t0, tA): interleave part of the chunk
    if (warp == 0u) {
      // level l+1's coins of the chunk and the zeros before each word (interleave part)
      const uint4 c = coin_block(a2.key, a2.level, R, j * (kChunk / 128u) + lane);
      const uint32_t c4[4] = {c.x, c.y, c.z, c.w};
      uint32_t z4[4], zs = 0;
#pragma unroll
      for (uint32_t k = 0; k < 4u; ++k) {
        cw2[4u * lane + k] = c4[k];
        const uint32_t tw = t0 + 32u * (4u * lane + k);
        const uint32_t valid = tw >= tA ? 0u : min(32u, tA - tw);
        z4[k] = static_cast<uint32_t>(__popc(~c4[k] & low_mask(valid)));
        zs += z4[k];
      }
      uint32_t ex = warp_inclusive_scan(zs) - zs;
#pragma unroll
      for (uint32_t k = 0; k < 4u; ++k) {
        zw2[4u * lane + k] = ex;
        ex += z4[k];
      }
    } else if (warp == 1u) {
      // the two ranges' records (lane: half lane / 16, word lane % 16) and their merges' shape
      const uint32_t h = lane >> 4, w = lane & 15u;
      hs[h][w] = reinterpret_cast<const uint32_t *>(pa.xr + (2u * cid + h) * 4u)[w];
      if (w == 0u) {
        const uint32_t r1 = 2u * R + h;
        const MergeBounds mb1 = merge_bounds(a1, r1);
        const uint32_t N1 = static_cast<uint32_t>(mb1.e - mb1.s);
        const uint32_t n11 = static_cast<uint32_t>(mb1.mid - mb1.s);
        const uint4 mi1 = a1.minfo[r1];
        hs[h][kS1] = static_cast<uint32_t>(mb1.s);
        hs[h][kN11] = n11;
        hs[h][kT1] = mi1.x;
        hs[h][kShift] = (mi1.y == n11) ? 0u : N1 - n11;  // leftover shift: first half exhausted -> 0
        hs[h][kN1] = N1;
      }
    }
    __syncthreads();
    // level l's coin words over both ranges (threads 0..127: half 0, 128..255: half 1), the
    // ranges' exception bits and their slices of the exception list
    uint32_t xv0, xv1;
    {
      const uint32_t h = tid >> 7;
      const uint32_t k = tid & 127u;
      const uint32_t lo = hs[h][kRgLo], Tc = hs[h][kRgTc], blo = hs[h][kRgBlo];
      const uint32_t nblk = Tc ? min(((lo + Tc + 127u) >> 7) - blo, kPairW / 4u) : 0u;
      if (k == 0u) hs[h][kNblk] = nblk;
      if (k < nblk) {
        const uint4 c = coin_block(a1.key, a1.level, hs[h][kRgMerge], blo + k);
        cw1[h][4u * k + 0u] = c.x;
        cw1[h][4u * k + 1u] = c.y;
        cw1[h][4u * k + 2u] = c.z;
        cw1[h][4u * k + 3u] = c.w;
      }
      load_range_bits(pa.x, hs[h][kRgGlo], hs[h][kRgCnt], xb1[h], k, 128u);
      // the range's first exceptions from the list (ranks k and k + 128), placed once their
      // positions are known
      const uint32_t xc = hs[h][kRgXcnt], xb = hs[h][kRgXbase];
      xv0 = k < xc ? pa.x.val[xb + k] : 0u;
      xv1 = k + 128u < xc ? pa.x.val[xb + k + 128u] : 0u;
    }
    __syncthreads();
    // the exception prefix of each range's words (the second warp of each half), then the zero
    // counts of level l's words and their prefix per half
    if (((tid & 127u) >> 5) == 1u) {
      const uint32_t h = tid >> 7;
      range_word_prefix(xb1[h], range_words(hs[h][kRgGlo], hs[h][kRgCnt]), xwp[h]);
    }
    {
      uint32_t z0 = 0, z1 = 0;  // thread k handles words 2k, 2k+1 of the combined array
      const uint32_t wA = 2u * tid, wB = 2u * tid + 1u;
      auto wz = [&](uint32_t wc) -> uint32_t {
        const uint32_t h = wc >= kPairW ? 1u : 0u;
        const uint32_t wi = wc - h * kPairW;
        if (wi >= 4u * hs[h][kNblk]) return 0u;
        const uint32_t pos = 32u * (4u * hs[h][kRgBlo] + wi);  // merge position of the word
        const uint32_t N1 = hs[h][kN1];
        const uint32_t valid = pos >= N1 ? 0u : min(32u, N1 - pos);
        return __popc(~cw1[h][wi] & low_mask(valid));
      };
      if (wA < 2u * kPairW) z0 = wz(wA);
      if (wB < 2u * kPairW) z1 = wz(wB);
      uint32_t total;
      const uint32_t excl = block_exclusive_scan(z0 + z1, scratch, &total);
      // the prefix restarts at half 1 (word kPairW): its base is the scan value there
      if (wA == kPairW) scratch[32] = excl;  // scratch[32] is free after the scan returned
      __syncthreads();
      const uint32_t base1 = scratch[32];
      if (wA < 2u * kPairW) {
        const uint32_t h = wA >= kPairW ? 1u : 0u;
        zw1[h][wA - h * kPairW] = hs[h][kRgZblk] + excl - (h ? base1 : 0u);
      }
      if (wB < 2u * kPairW) {
        const uint32_t h = wB >= kPairW ? 1u : 0u;
        zw1[h][wB - h * kPairW] = hs[h][kRgZblk] + excl + z0 - (h ? base1 : 0u);
      }
    }
    // every exception of the ranges at its position: rank e sits at the e-th set bit of the
    // range's words (the last word whose prefix is at most e)
    {
      const uint32_t h = tid >> 7;
      const uint32_t k = tid & 127u;
      const uint32_t xc = hs[h][kRgXcnt], xb = hs[h][kRgXbase];
      const uint32_t g_lo = hs[h][kRgGlo];
      const uint32_t nxw = range_words(g_lo, hs[h][kRgCnt]);
      for (uint32_t e = k; e < xc; e += 128u) {
        uint32_t lo = 0, hi = nxw;
        while (hi - lo > 1u) {
          const uint32_t mid = (lo + hi) >> 1;
          if (xwp[h][mid] <= e) lo = mid;
          else hi = mid;
        }
        const uint32_t bit = select_set_bit(xb1[h][lo], e - xwp[h][lo]);
        const uint32_t pos = min(32u * lo + bit - (g_lo & 31u), kChunk - 1u);
        xval[h][pos] = e == k ? xv0 : (e == k + 128u ? xv1 : pa.x.val[xb + e]);
      }
    }
    __syncthreads();
    // per-half constants in registers
    uint32_t hs1[2], hn11[2], hT1[2], hshift[2], hw0[2], hglo[2];
#pragma unroll
    for (uint32_t h = 0; h < 2u; ++h) {
      hs1[h] = hs[h][kS1];
      hn11[h] = hs[h][kN11];
      hT1[h] = hs[h][kT1];
      hshift[h] = hs[h][kShift];
      hw0[h] = 4u * hs[h][kRgBlo];
      hglo[h] = hs[h][kRgGlo];
    }
    // outputs: lane = position in a word of level l+1; warp w owns words w, w+8, ...
    E *C = out + mb2.s;
    constexpr uint32_t kWarps = kThreads / 32;
    constexpr uint32_t kWordsPerWarp = kChunk / 32u / kWarps;
    constexpr uint32_t kBatch = sizeof(E) >= 16 ? 4u : 8u;
#pragma unroll
    for (uint32_t b0 = 0; b0 < kWordsPerWarp; b0 += kBatch) {
      E v[kBatch];
#pragma unroll
      for (uint32_t k = 0; k < kBatch; ++k) {
        const uint32_t u = warp + (b0 + k) * kWarps;
        const uint32_t t = t0 + 32u * u + lane;
        if (t < t1) {
          uint32_t h, p;  // half and merge position in level l's merge 2R + h
          if (t < T2) {
            const uint32_t word = cw2[u];
            const uint32_t Z = Z0 + zw2[u] + __popc(~word & low_mask(lane));
            h = (word >> lane) & 1u;
            p = h ? t - Z : Z;
          } else {
            h = first_exh2 ? 1u : 0u;
            p = first_exh2 ? t - h1 : t - h2;
          }
          const uint32_t s1 = h ? hs1[1] : hs1[0];
          const uint32_t gq = s1 + p;
          const uint32_t glo = h ? hglo[1] : hglo[0];
          const uint32_t bw = (gq >> 5) - (glo >> 5);
          uint32_t xs;
          if ((xb1[h][min(bw, kPairW - 1u)] >> (gq & 31u)) & 1u) {
            // exception: the tail moved another element here
            xs = xval[h][min(gq - glo, kChunk - 1u)];
          } else if (p < (h ? hT1[1] : hT1[0])) {
            const uint32_t wi = min((p >> 5) - (h ? hw0[1] : hw0[0]), kPairW - 1u);
            const uint32_t word = cw1[h][wi];
            const uint32_t Z = zw1[h][wi] + __popc(~word & low_mask(p & 31u));
            xs = s1 + (((word >> (p & 31u)) & 1u) ? (h ? hn11[1] : hn11[0]) + p - Z : Z);
          } else {
            xs = s1 + p - (h ? hshift[1] : hshift[0]);
          }
          v[k] = in[xs < a1.n ? xs : 0u];  // the clamp keeps every load inside the array
        }
      }
#pragma unroll
      for (uint32_t k = 0; k < kBatch; ++k) {
        const uint32_t t = t0 + 32u * (warp + (b0 + k) * kWarps) + lane;
        if (t < t1) C[t] = v[k];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------- literal merge (flag) --------
// Algorithm 3 as printed merges in place: i walks the output, and a 1-coin swaps T[i] with the
// next second-half element T[j], so the front of the first half's unconsumed part moves to its
// back. The second-half elements land exactly where the stable interleave puts them; the first
// half behaves as a queue visited in rounds ("laps"): every step, 0- or 1-coin, visits the next
// remaining first-half element in its original cyclic order, and a 0-coin takes the element it
// visits. Lap 0 visits A[k] at step k; the elements a lap does not take (its 1-coin steps) are
// visited again, in order, in the next lap, which starts where the previous one ends:
//   S_0 = 0, m_0 = n1, S_{j+1} = S_j + m_j, m_{j+1} = ones among coins [S_j, S_{j+1}).
// So first-half element k lands at its first visit step x that has a 0-coin, or, if the loop
// breaks first (the second half ran out at T), at its first visit step x >= T: the leftover part
// [T, N) holds the queue from its front, which is exactly the order of those visits. The gather
// of the stable interleave writes every position first; this pass then overwrites the
// first-half positions with their literal elements. The tails follow unchanged.


// the lap starts S_j and Z(S_j) of every merge, while S_j < T (one thread per merge)
__global__ void __launch_bounds__(kThreads) lap_kernel(LevelArgs a) {
  for (uint32_t r = blockIdx.x * kThreads + threadIdx.x; r < a.M; r += gridDim.x * kThreads) {
    const MergeBounds mb = merge_bounds(a, r);
    const uint32_t n1 = static_cast<uint32_t>(mb.mid - mb.s);
    const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
    const uint32_t T = a.minfo[r].x;
    uint2 *const L = a.laps + static_cast<uint64_t>(r) * a.lcap;
    uint32_t S = 0, Z = 0, m = n1;
    L[0] = make_uint2(0u, 0u);
    for (uint32_t j = 1; j < a.lcap; ++j) {
      if (S >= T || m == 0u) break;
      const uint32_t S2 = min(S + m, N);  // (S_j + m_j <= N: the rest of both halves)
      const uint32_t Z2 = zeros_before(a, r, S2);
      m = (S2 - Z2) - (S - Z);
      S = S2;
      Z = Z2;
      L[j] = make_uint2(S, Z);
    }
  }
}

// every first-half element of every merge to its literal position (one chunk of 4096
// first-half elements per CTA; lap 0's coins come from shared memory)
template <typename E>
__global__ void __launch_bounds__(kThreads) literal_scatter_kernel(LevelArgs a) {
  __shared__ uint32_t cw[kChunk / 32u];
  __shared__ uint32_t zw[kChunk / 32u];
  const E *__restrict__ in = static_cast<const E *>(a.in);
  E *__restrict__ out = static_cast<E *>(a.out);
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint64_t nchunks = static_cast<uint64_t>(a.M) * a.J;
  for (uint64_t cid = blockIdx.x; cid < nchunks; cid += gridDim.x) {
    const uint32_t r = static_cast<uint32_t>(cid / a.J);
    const uint32_t j = static_cast<uint32_t>(cid - static_cast<uint64_t>(r) * a.J);
    const MergeBounds mb = merge_bounds(a, r);
    const uint32_t n1 = static_cast<uint32_t>(mb.mid - mb.s);
    const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
    const uint32_t k0 = j * kChunk;
    if (k0 >= n1) continue;  // uniform across the CTA
    const uint32_t k1 = min(k0 + kChunk, n1);
    const uint32_t T = a.minfo[r].x;
    if (tid < 32u) {
      const uint4 c = coin_block(a.key, a.level, r, j * (kChunk / 128u) + lane);
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
    __syncthreads();
    const uint32_t Zc = a.zc[cid];
    const uint2 *const L = a.laps + static_cast<uint64_t>(r) * a.lcap;
    for (uint32_t k = k0 + tid; k < k1; k += kThreads) {
      uint32_t P;
      // lap 0: visited at step k (coin and zeros before it from shared memory)
      const uint32_t q = k - k0;
      const uint32_t w0 = cw[q >> 5];
      if (k >= T || ((w0 >> (q & 31u)) & 1u) == 0u) {
        P = k;
      } else {
        uint32_t Zx = Zc + zw[q >> 5] + __popc(~w0 & low_mask(q & 31u));
        uint32_t x = k, S = 0, Z = 0, m = n1, lap = 0;
        P = N - 1u;  // (only if the walk below were cut short: an inconsistent plan)
        for (uint32_t h = 0; h <= N; ++h) {
          // x survives lap `lap`: its rank among the lap's survivors, then its next visit
          const uint32_t rk = (x - Zx) - (S - Z);
          uint32_t S2, Z2;
          if (lap + 1u < a.lcap) {
            const uint2 e = L[lap + 1u];
            S2 = e.x;
            Z2 = e.y;
          } else {
            S2 = min(S + m, N);
            Z2 = zeros_before(a, r, S2);
          }
          m = (S2 - Z2) - (S - Z);
          S = S2;
          Z = Z2;
          ++lap;
          x = S + rk;
          if (x >= T) {
            P = x;
            break;
          }
          // the coin word at x and the zeros before x, from the level's word table
          const uint64_t cx = static_cast<uint64_t>(r) * a.J + (x >> 12);
          const uint2 tw = a.ctab[cx * 128u + ((x >> 5) & 127u)];
          if (((tw.x >> (x & 31u)) & 1u) == 0u) {
            P = x;
            break;
          }
          Zx = a.zc[cx] + tw.y + static_cast<uint32_t>(__popc(~tw.x & low_mask(x & 31u)));
        }
      }
      out[mb.s + min(P, N - 1u)] = in[mb.s + k];
    }
    __syncthreads();  // cw / zw are reused by the next chunk
  }
}

// ---------------------------------------------------------- balanced-word merge (flag) -----
// Merges driven by a balanced word (MS_FLAG_BALANCED; the idea of the paper's Section 3). The word
// of merge r is its halves' labels (0 first half, 1 second half) merged by the merge's own coin
// loop and random insertions: label t is coin t for t < T and the label of the half that did not
// run out beyond, then the insertions move labels exactly as they would move elements. So the
// label bytes of a level are written, the usual tail patches (or the sequential fallback) run on
// them, and the data is interleaved stably by the resulting word -- no element is moved by an
// insertion. Label bytes sit at the global position of their merge output.

// the level's labels before the insertions: one chunk of 4096 steps of one merge per CTA
__global__ void __launch_bounds__(kThreads) label_kernel(LevelArgs a, uint8_t *lab) {
  __shared__ uint32_t cw[kChunk / 32u];
  const uint32_t tid = threadIdx.x;
  const uint64_t nchunks = static_cast<uint64_t>(a.M) * a.J;
  for (uint64_t cid = blockIdx.x; cid < nchunks; cid += gridDim.x) {
    const uint32_t r = static_cast<uint32_t>(cid / a.J);
    const uint32_t j = static_cast<uint32_t>(cid - static_cast<uint64_t>(r) * a.J);
    const MergeBounds mb = merge_bounds(a, r);
    const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
    const uint32_t t0 = j * kChunk;
    if (t0 >= N) continue;  // uniform across the CTA
    const uint32_t t1 = t0 + min(kChunk, N - t0);  // (t0 < N; no 32-bit overflow)
    const uint4 mi = a.minfo[r];
    const uint32_t T = mi.x;
    const uint32_t n1 = static_cast<uint32_t>(mb.mid - mb.s);
    const uint8_t left = (mi.y == n1) ? 1u : 0u;  // the first half ran out: the rest are its other
    if (tid < 32u) {
      const uint4 c = coin_block(a.key, a.level, r, j * (kChunk / 128u) + tid);
      cw[4u * tid + 0u] = c.x;
      cw[4u * tid + 1u] = c.y;
      cw[4u * tid + 2u] = c.z;
      cw[4u * tid + 3u] = c.w;
    }
    __syncthreads();
    uint8_t *const L = lab + mb.s;
    for (uint32_t t = t0 + tid; t < t1; t += kThreads) {
      const uint32_t q = t - t0;
      L[t] = t < T ? static_cast<uint8_t>((cw[q >> 5] >> (q & 31u)) & 1u) : left;
    }
    __syncthreads();
  }
}

// zeros among each chunk's final labels (one warp per chunk)
__global__ void __launch_bounds__(kThreads) label_count_kernel(LevelArgs a, const uint8_t *lab,
                                                               uint32_t *zl) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nchunks = static_cast<uint64_t>(a.M) * a.J;
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (kThreads / 32);
  for (uint64_t cid = (static_cast<uint64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
       cid < nchunks; cid += warps) {
    const uint32_t r = static_cast<uint32_t>(cid / a.J);
    const uint32_t j = static_cast<uint32_t>(cid - static_cast<uint64_t>(r) * a.J);
    const MergeBounds mb = merge_bounds(a, r);
    const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
    const uint32_t t0 = j * kChunk;
    const uint32_t len = t0 < N ? min(kChunk, N - t0) : 0u;
    uint32_t z = 0;
    for (uint32_t k = lane; k < len; k += 32u) z += lab[mb.s + t0 + k] == 0u ? 1u : 0u;
    z = warp_sum(z);
    if (lane == 0) zl[cid] = z;
  }
}

// exclusive prefix of the chunk zero counts along each merge's row (one warp per merge)
__global__ void __launch_bounds__(kThreads) label_scan_kernel(LevelArgs a, uint32_t *zl) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (kThreads / 32);
  for (uint64_t r = (static_cast<uint64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5; r < a.M;
       r += warps) {
    uint32_t carry = 0;
    for (uint32_t j0 = 0; j0 < a.J; j0 += 32u) {
      const uint32_t j = j0 + lane;
      const uint32_t v = j < a.J ? zl[r * a.J + j] : 0u;
      const uint32_t incl = warp_inclusive_scan(v);
      if (j < a.J) zl[r * a.J + j] = carry + incl - v;
      carry += __shfl_sync(kFullMask, incl, 31);
    }
  }
}

// the data interleaved stably by the final words: a chunk's two source runs (its zeros from the
// first half, its ones from the second) staged in shared memory, then one output a thread
template <typename E>
__global__ void __launch_bounds__(kStageThreads) word_gather_kernel(LevelArgs a, const uint8_t *lab,
                                                                    const uint32_t *zl) {
  constexpr uint32_t kV = 16u / sizeof(E) > 0 ? 16u / sizeof(E) : 1u;
  constexpr uint32_t kBuf = kChunk + 4u * kV + 8u;
  extern __shared__ __align__(16) unsigned char wg_raw[];
  E *const sbuf = reinterpret_cast<E *>(wg_raw);
  __shared__ uint32_t cw[kChunk / 32u];
  __shared__ uint32_t zw[kChunk / 32u];
  __shared__ uint32_t scratch[33];
  const E *__restrict__ in = static_cast<const E *>(a.in);
  E *__restrict__ out = static_cast<E *>(a.out);
  const uint32_t tid = threadIdx.x;
  const uint64_t nchunks = static_cast<uint64_t>(a.M) * a.J;
  for (uint64_t cid = blockIdx.x; cid < nchunks; cid += gridDim.x) {
    const uint32_t r = static_cast<uint32_t>(cid / a.J);
    const uint32_t j = static_cast<uint32_t>(cid - static_cast<uint64_t>(r) * a.J);
    const MergeBounds mb = merge_bounds(a, r);
    const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
    const uint32_t t0 = j * kChunk;
    if (t0 >= N) continue;  // uniform across the CTA
    const uint32_t len = min(kChunk, N - t0);
    const uint32_t n1 = static_cast<uint32_t>(mb.mid - mb.s);
    const uint32_t n2 = N - n1;
    // the chunk's words: bit = label (1: second half). Thread k builds word k from its 32 label
    // bytes (eight 4-byte loads when the row is 4-byte aligned, all issued before use)
    {
      const uint8_t *const Lr = lab + mb.s + t0;
      const uint32_t t = 32u * tid;
      uint32_t m = 0;
      if ((reinterpret_cast<uintptr_t>(Lr) & 3u) == 0u && t + 32u <= len) {
        uint32_t v[8];
#pragma unroll
        for (uint32_t u = 0; u < 8u; ++u) v[u] = reinterpret_cast<const uint32_t *>(Lr + t)[u];
#pragma unroll
        for (uint32_t u = 0; u < 8u; ++u) {
          // label bytes are 0 or 1: gather bit 0 of each of the four bytes
          const uint32_t x = v[u];
          const uint32_t b4 = (x & 1u) | ((x >> 7) & 2u) | ((x >> 14) & 4u) | ((x >> 21) & 8u);
          m |= b4 << (4u * u);
        }
      } else {
        for (uint32_t i = 0; i < 32u; ++i)
          if (t + i < len && Lr[t + i] != 0u) m |= 1u << i;
      }
      cw[tid] = m;
    }
    __syncthreads();
    uint32_t zc = 0;
    {
      // zeros before each word (one word a thread: kStageThreads = kChunk / 32), and the total
      static_assert(kStageThreads == kChunk / 32u, "one label word per thread");
      const uint32_t valid = 32u * tid >= len ? 0u : min(32u, len - 32u * tid);
      const uint32_t zk = static_cast<uint32_t>(__popc(~cw[tid] & low_mask(valid)));
      zw[tid] = block_exclusive_scan(zk, scratch, &zc);
    }
    const uint32_t Z0 = zl[cid];  // zeros before the chunk
    // the runs: first half [Z0, Z0 + zc), second half [t0 - Z0, t0 - Z0 + len - zc)
    const uint32_t za = min(Z0, n1), na = min(zc, n1 - za);
    const uint32_t ob = min(t0 - Z0, n2), nb = min(len - zc, n2 - ob);
    const E *const srcA = in + mb.s + za;
    const E *const srcB = in + mb.mid + ob;
    const uint32_t offA = static_cast<uint32_t>((reinterpret_cast<uintptr_t>(srcA) & 15u) / sizeof(E));
    const uint32_t offB = ((offA + na + kV - 1u) / kV) * kV +
                          static_cast<uint32_t>((reinterpret_cast<uintptr_t>(srcB) & 15u) / sizeof(E));
    stage_run(sbuf + offA, srcA, min(na, kBuf - offA));
    stage_run(sbuf + offB, srcB, min(nb, kBuf - min(offB, kBuf)));
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    E *const C = out + mb.s + t0;
    for (uint32_t t = tid; t < len; t += kStageThreads) {
      const uint32_t word = cw[t >> 5];
      const uint32_t Z = zw[t >> 5] + static_cast<uint32_t>(__popc(~word & low_mask(t & 31u)));
      const uint32_t src = ((word >> (t & 31u)) & 1u) ? offB + (t - Z) : offA + Z;
      C[t] = sbuf[min(src, kBuf - 1u)];
    }
    __syncthreads();  // the buffers are reused by the next chunk
  }
}

// ---------------------------------------------------------- staged fused pair (w = 4) ----
// Two levels l, l+1 in one pass for 4-byte elements. A CTA takes 4096 outputs of level l+1;
// they read one range of each of its halves (merges 2R and 2R+1 of level l), and each range is
// the interleave of one run of each half of its level-l merge (then that merge's leftover),
// with level l's tail moves as exceptions. The chunk's record (pair_ranges_kernel) names the
// four input runs, which are copied to shared memory with 16-byte asynchronous copies while
// the coins are generated; the two level-l ranges are built there (walking the runs with level
// l's coins, then overwriting the exception positions from the exception list); the level l+1
// outputs are placed from them as in the staged single gather.
__global__ void __launch_bounds__(kStageThreads, 6) pair_staged_kernel(PairArgs pa) {
  using E = uint32_t;
  constexpr uint32_t kV = 4;
  constexpr uint32_t kRunBuf = kChunk + 8u * kV + kStageGroup;  // four runs with their phases
  constexpr uint32_t kValBuf = kChunk + 2u * kStageGroup;       // two ranges, group-aligned
  __shared__ __align__(16) E sruns[kRunBuf];
  __shared__ __align__(16) E svals[kValBuf];
  __shared__ uint32_t cw2[kChunk / 32u + 1u];
  __shared__ uint32_t zw2[kChunk / 32u];
  __shared__ uint32_t cw1[2][kPairW + 1u];
  __shared__ uint32_t zw1[2][kPairW];
  __shared__ uint32_t xb1[2][kPairW];
  __shared__ uint32_t xwp[2][kPairW];
  __shared__ uint32_t hs[2][kRgWords];  // the chunk's record: its two level-l ranges
  const LevelArgs &a1 = pa.l1;
  const LevelArgs &a2 = pa.l2;
  if (a1.ctrl[1]) return;  // level l's tails overflowed: the unfused fallback runs instead
  const E *__restrict__ in = static_cast<const E *>(pa.in);
  E *__restrict__ out = static_cast<E *>(pa.out);
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint32_t warp = tid >> 5;
  const uint64_t nchunks = static_cast<uint64_t>(a2.M) * a2.J;
  for (uint64_t cid = blockIdx.x; cid < nchunks; cid += gridDim.x) {
    const uint32_t R = static_cast<uint32_t>(cid / a2.J);
    const uint32_t j = static_cast<uint32_t>(cid - static_cast<uint64_t>(R) * a2.J);
    const MergeBounds mb2 = merge_bounds(a2, R);
    const uint32_t N2 = static_cast<uint32_t>(mb2.e - mb2.s);
    const uint32_t t0 = j * kChunk;
    if (t0 >= N2) continue;  // uniform across the CTA
    const uint32_t t1 = t0 + min(kChunk, N2 - t0);  // (t0 < N2; no 32-bit overflow)
    const uint32_t len = t1 - t0;
    const uint32_t h1 = static_cast<uint32_t>(mb2.mid - mb2.s);  // level l+1's first half
    const uint32_t h2 = N2 - h1;
    const uint4 mi2 = a2.minfo[R];
    const uint32_t T2 = mi2.x;
    const uint32_t abit2 = (mi2.y == h1) ? 1u : 0u;  // 1: level l+1's first half ran out
    // level l+1: chunk-relative break step Tc2 and the zeros before it zT2
    uint32_t Tc2 = 0, zT2 = 0;
    if (t0 < T2) {
      const uint32_t Z0 = a2.zc[cid];
      Tc2 = min(t1, T2) - t0;
      const uint32_t Jr = chunks_of(N2);
      zT2 = (t1 <= T2) ? ((j + 1u < Jr) ? a2.zc[cid + 1] - Z0 : h1 - Z0) : mi2.y - Z0;
    }
    (void)h2;
    // the record of the two level-l ranges (pair_ranges_kernel), then their four input runs
    // staged at once, each at its own 16-byte phase; the coins follow while the copies run
    if (warp == 1u) hs[lane >> 4][lane & 15u] =
        reinterpret_cast<const uint32_t *>(pa.xr + (2u * cid + (lane >> 4)) * 4u)[lane & 15u];
    __syncthreads();
    const uint32_t cnt0 = hs[0][kRgCnt], cnt1 = hs[1][kRgCnt];
    auto phase_of = [](const E *p) {
      return static_cast<uint32_t>((reinterpret_cast<uintptr_t>(p) & 15u) / sizeof(E));
    };
    auto up = [](uint32_t x) { return ((x + kV - 1u) / kV) * kV; };
    const E *const sa0 = in + hs[0][kRgRunA];
    const E *const sb0 = in + hs[0][kRgRunB];
    const E *const sa1 = in + hs[1][kRgRunA];
    const E *const sb1 = in + hs[1][kRgRunB];
    const uint32_t offA0 = phase_of(sa0);
    const uint32_t offB0 = up(offA0 + hs[0][kRgNa]) + phase_of(sb0);
    const uint32_t offA1 = up(offB0 + hs[0][kRgNb]) + phase_of(sa1);
    const uint32_t offB1 = up(offA1 + hs[1][kRgNa]) + phase_of(sb1);
    stage_run(sruns + offA0, sa0, min(hs[0][kRgNa], kRunBuf - min(offA0, kRunBuf)));
    stage_run(sruns + offB0, sb0, min(hs[0][kRgNb], kRunBuf - min(offB0, kRunBuf)));
    stage_run(sruns + offA1, sa1, min(hs[1][kRgNa], kRunBuf - min(offA1, kRunBuf)));
    stage_run(sruns + offB1, sb1, min(hs[1][kRgNb], kRunBuf - min(offB1, kRunBuf)));
    cp_async_commit();
    if (warp == 2u) {
      // coins of level l+1 for steps [t0, t0 + Tc2) and the zeros before each word
      const uint32_t nwords = (Tc2 + 31u) >> 5;
      if (4u * lane < nwords) {
        const uint4 c = coin_block(a2.key, a2.level, R, j * (kChunk / 128u) + lane);
        cw2[4u * lane + 0u] = c.x;
        cw2[4u * lane + 1u] = c.y;
        cw2[4u * lane + 2u] = c.z;
        cw2[4u * lane + 3u] = c.w;
      }
      __syncwarp();
      uint32_t z4[4], zs = 0;
#pragma unroll
      for (uint32_t k = 0; k < 4u; ++k) {
        z4[k] = (4u * lane + k < nwords) ? static_cast<uint32_t>(__popc(~cw2[4u * lane + k])) : 0u;
        zs += z4[k];
      }
      uint32_t ex = warp_inclusive_scan(zs) - zs;
#pragma unroll
      for (uint32_t k = 0; k < 4u; ++k) {
        zw2[4u * lane + k] = ex;
        ex += z4[k];
      }
    } else if (warp < 2u) {
      // level l, half h = warp: the coin words over its range, the zeros before each word, the
      // range's exception bits and their prefix
      const uint32_t h = warp;
      const uint32_t lo = hs[h][kRgLo], Tc1 = hs[h][kRgTc], blo = hs[h][kRgBlo];
      const uint32_t nblk = Tc1 ? min(((lo + Tc1 + 127u) >> 7) - blo, kPairW / 4u) : 0u;
      for (uint32_t k = lane; k < nblk; k += 32u) {
        const uint4 c = coin_block(a1.key, a1.level, hs[h][kRgMerge], blo + k);
        cw1[h][4u * k + 0u] = c.x;
        cw1[h][4u * k + 1u] = c.y;
        cw1[h][4u * k + 2u] = c.z;
        cw1[h][4u * k + 3u] = c.w;
      }
      load_range_bits(pa.x, hs[h][kRgGlo], hs[h][kRgCnt], xb1[h], lane, 32u);
      __syncwarp();
      // zeros before each word (merge-relative): lane takes words 5*lane .. 5*lane+4
      {
        const uint32_t nw = 4u * nblk;
        uint32_t z5[5], zs = 0;
#pragma unroll
        for (uint32_t k = 0; k < 5u; ++k) {
          const uint32_t wi = 5u * lane + k;
          z5[k] = wi < nw ? static_cast<uint32_t>(__popc(~cw1[h][wi])) : 0u;
          zs += z5[k];
        }
        uint32_t ex = hs[h][kRgZblk] + warp_inclusive_scan(zs) - zs;
#pragma unroll
        for (uint32_t k = 0; k < 5u; ++k) {
          const uint32_t wi = 5u * lane + k;
          if (wi < kPairW) zw1[h][wi] = ex;
          ex += z5[k];
        }
      }
      range_word_prefix(xb1[h], range_words(hs[h][kRgGlo], hs[h][kRgCnt]), xwp[h]);
    }
    cp_async_wait<0>();
    __syncthreads();
    // level l: the two ranges into svals (half 0 at 0, half 1 at voff1), eight positions a thread
    const uint32_t voff1 = (cnt0 + kStageGroup - 1u) & ~(kStageGroup - 1u);
    {
      const uint32_t ng0 = (cnt0 + kStageGroup - 1u) / kStageGroup;
      const uint32_t ng = ng0 + (cnt1 + kStageGroup - 1u) / kStageGroup;
      for (uint32_t g = tid; g < ng; g += kStageThreads) {
        const uint32_t h = g < ng0 ? 0u : 1u;
        const uint32_t p0 = kStageGroup * (h ? g - ng0 : g);
        const uint32_t lo = hs[h][0], Tc1 = hs[h][2], zT1 = hs[h][3], abit1 = hs[h][4];
        uint32_t pa, pb, bits;
        if (p0 < Tc1) {
          const uint32_t q0 = lo + p0;
          const uint32_t u = min((q0 >> 5) - 4u * hs[h][5], kPairW - 1u);
          const uint32_t sh = q0 & 31u;
          const uint32_t w0 = cw1[h][u];
          pa = zw1[h][u] + static_cast<uint32_t>(__popc(~w0 & low_mask(sh))) - hs[h][11];
          pb = p0 - pa;
          bits = __funnelshift_r(w0, cw1[h][u + 1u], sh);
        } else {
          pa = zT1 + (p0 - Tc1) * (1u - abit1);
          pb = (Tc1 - zT1) + (p0 - Tc1) * abit1;
          bits = 0u;
        }
        pa = min((h ? offA1 : offA0) + pa, kRunBuf - kStageGroup);
        pb = min((h ? offB1 : offB0) + pb, kRunBuf - kStageGroup);
        uint32_t v[kStageGroup];
#pragma unroll
        for (uint32_t i = 0; i < kStageGroup; ++i) {
          const uint32_t bit = (p0 + i < Tc1) ? ((bits >> i) & 1u) : abit1;
          v[i] = sruns[bit ? pb : pa];
          pa += bit ^ 1u;
          pb += bit;
        }
        uint4 *const dst = reinterpret_cast<uint4 *>(svals + (h ? voff1 : 0u) + p0);
        dst[0] = make_uint4(v[0], v[1], v[2], v[3]);
        dst[1] = make_uint4(v[4], v[5], v[6], v[7]);
      }
    }
    __syncthreads();
    // level l's tail moves: exception e of a range (its rank in the range) sits at the e-th set
    // bit of the range's words; its element comes from the list. Four exceptions a thread at a
    // time, their loads in flight together.
    {
      const uint32_t c0 = hs[0][13], ctot = c0 + hs[1][13];
      for (uint32_t e0 = 4u * tid; e0 < ctot; e0 += 4u * kStageThreads) {
        uint32_t xs[4], dst[4];
#pragma unroll
        for (uint32_t u = 0; u < 4u; ++u) {
          const uint32_t e = e0 + u;
          dst[u] = kNone;
          if (e < ctot) {
            const uint32_t h = e < c0 ? 0u : 1u;
            const uint32_t k = h ? e - c0 : e;
            // the word holding it: the last word whose prefix is <= k
            const uint32_t nxw = range_words(hs[h][10], hs[h][1]);
            uint32_t lo = 0, hi = nxw;
            while (hi - lo > 1u) {
              const uint32_t mid = (lo + hi) >> 1;
              if (xwp[h][mid] <= k) lo = mid;
              else hi = mid;
            }
            const uint32_t b = select_set_bit(xb1[h][lo], k - xwp[h][lo]);
            dst[u] = (h ? voff1 : 0u) + min(32u * lo + b - (hs[h][10] & 31u), kChunk - 1u);
            xs[u] = pa.x.val[hs[h][12] + k];
          }
        }
#pragma unroll
        for (uint32_t u = 0; u < 4u; ++u)
          if (dst[u] != kNone) xs[u] = in[xs[u] < a1.n ? xs[u] : 0u];
#pragma unroll
        for (uint32_t u = 0; u < 4u; ++u)
          if (dst[u] != kNone) svals[min(dst[u], kValBuf - 1u)] = xs[u];
      }
    }
    __syncthreads();
    // level l+1: outputs placed from the two ranges, in groups of eight aligned to 16 bytes of
    // the output (group 0: the head before the first aligned one)
    E *const C = out + mb2.s + t0;
    const uint32_t cph = static_cast<uint32_t>((reinterpret_cast<uintptr_t>(C) & 15u) / sizeof(E));
    const uint32_t hd = min(len, (kV - cph) % kV);
    const uint32_t ngroups = 1u + (len - hd + kStageGroup - 1u) / kStageGroup;
    for (uint32_t gi = tid; gi < ngroups; gi += kStageThreads) {
      const uint32_t p0 = gi == 0u ? 0u : hd + kStageGroup * (gi - 1u);
      const uint32_t cnt = gi == 0u ? hd : min(kStageGroup, len - p0);
      if (cnt == 0u) continue;
      uint32_t pa2, pb2, bits;
      if (p0 < Tc2) {
        const uint32_t u = p0 >> 5, sh = p0 & 31u;
        const uint32_t w0 = cw2[u];
        pa2 = zw2[u] + static_cast<uint32_t>(__popc(~w0 & low_mask(sh)));
        pb2 = p0 - pa2;
        bits = __funnelshift_r(w0, cw2[u + 1u], sh);
      } else {
        pa2 = zT2 + (p0 - Tc2) * (1u - abit2);
        pb2 = (Tc2 - zT2) + (p0 - Tc2) * abit2;
        bits = 0u;
      }
      pa2 = min(pa2, kValBuf - kStageGroup);
      pb2 = min(voff1 + pb2, kValBuf - kStageGroup);
      E v[kStageGroup];
#pragma unroll
      for (uint32_t i = 0; i < kStageGroup; ++i) {
        const uint32_t bit = (p0 + i < Tc2) ? ((bits >> i) & 1u) : abit2;
        v[i] = svals[bit ? pb2 : pa2];
        pa2 += bit ^ 1u;
        pb2 += bit;
      }
      if (gi != 0u && cnt == kStageGroup) {
        uint4 *const dst = reinterpret_cast<uint4 *>(C + p0);
        dst[0] = make_uint4(v[0], v[1], v[2], v[3]);
        dst[1] = make_uint4(v[4], v[5], v[6], v[7]);
      } else {
#pragma unroll
        for (uint32_t i = 0; i < kStageGroup; ++i)
          if (i < cnt) C[p0 + i] = v[i];
      }
    }
    __syncthreads();  // the buffers are reused by the next chunk
  }
}

template <typename E>
__global__ void __launch_bounds__(kThreads) copy_kernel(LevelArgs a) {
  if (gated_off(a)) return;
  const E *in = static_cast<const E *>(a.in);
  E *out = static_cast<E *>(a.out);
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * kThreads + threadIdx.x; i < a.n;
       i += static_cast<uint64_t>(gridDim.x) * kThreads)
    out[i] = in[i];
}

unsigned grid_for(uint64_t items, uint64_t per_block, uint64_t cap) {
  uint64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return static_cast<unsigned>(g);
}

LevelArgs level_args(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                     const Buffers &b, uint64_t seed) {
  LevelArgs a;
  a.in = in;
  a.out = out;
  a.n = p.n;
  a.key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  a.c = p.c;
  a.level = lv.level;
  a.M = lv.M;
  a.J = lv.J;
  a.kcap = lv.kcap;
  a.hbits = lv.hbits;
  a.flags = p.flags;
  a.zc = b.zc;
  a.minfo = b.minfo;
  a.ctrl = b.ctrl;
  a.mv = b.mv;
  a.hkeys = b.hkeys;
  a.hvals = b.hvals;
  a.pdst = b.pdst;
  a.psrc = b.psrc;
  a.ptmp = b.ptmp;
  a.ostart = b.ostart;
  a.zb = nullptr;
  a.gate = nullptr;
  a.gate_on = 0;
  a.out_alt = nullptr;
  a.alt_sel = nullptr;
  a.laps = b.laps;
  a.lcap = lv.lcap;
  a.ctab = nullptr;
  if (p.flags & MS_FLAG_LITERAL) {  // the literal merge's rank queries read them
    a.zb = b.zb;
    a.ctab = b.ctab;
  }
  return a;
}

constexpr unsigned kResident = 152u * 8u;

ExcArgs exc_args(const Plan &p, const Buffers &b) {
  ExcArgs x;
  x.bits = b.xbits;
  x.src = b.xsrc;
  x.val = b.xval;
  x.bpre = b.xbpre;
  x.tpre = b.xtpre;
  x.n = p.n;
  return x;
}

template <typename F>
void timed(Prof *pf, int kind, cudaStream_t s, F &&launch) {
  if (pf) pf->begin(kind, s);
  launch();
  if (pf) pf->end(s);
}

template <typename E>
cudaError_t launch_data_t(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                          const Buffers &b, uint64_t seed, cudaStream_t s) {
  const LevelArgs a = level_args(p, lv, in, out, b, seed);
  const uint64_t nchunks = static_cast<uint64_t>(lv.M) * lv.J;
  if (p.flags & MS_FLAG_BALANCED) {
    // the labels, their insertions (on the label bytes), their chunk prefix, then the data
    LevelArgs la = level_args(p, lv, nullptr, b.labels, b, seed);
    label_kernel<<<grid_for(nchunks, 1, 1u << 20), kThreads, 0, s>>>(la, b.labels);
    tail_sequential_kernel<uint8_t><<<grid_for(lv.M, kThreads, 1u << 16), kThreads, 0, s>>>(la);
    patch_read_kernel<uint8_t><<<kResident, kThreads, 0, s>>>(la);
    patch_write_kernel<uint8_t><<<kResident, kThreads, 0, s>>>(la);
    label_count_kernel<<<grid_for(nchunks, kThreads / 32, 1u << 20), kThreads, 0, s>>>(
        la, b.labels, b.zlab);
    label_scan_kernel<<<grid_for(lv.M, kThreads / 32, 1u << 16), kThreads, 0, s>>>(la, b.zlab);
    constexpr uint32_t kV = 16u / sizeof(E);
    const size_t smem = (kChunk + 4u * kV + 8u) * sizeof(E);
    auto wk = word_gather_kernel<E>;
    cudaError_t e = allow_dynamic_smem(wk, smem);
    if (e != cudaSuccess) return e;
    timed(p.prof, kKindGather, s, [&] {
      wk<<<grid_for(nchunks, 1, 1u << 20), kStageThreads, smem, s>>>(a, b.labels, b.zlab);
    });
    return cudaGetLastError();
  }
  timed(p.prof, kKindGather, s, [&] {
    if constexpr (sizeof(E) <= 8)
      gather_staged_kernel<E><<<grid_for(nchunks, 1, 1u << 20), kStageThreads, 0, s>>>(a);
    else
      gather_kernel<E><<<grid_for(nchunks, 1, 1u << 20), kThreads, 0, s>>>(a);
  });
  if (p.flags & MS_FLAG_LITERAL) {
    timed(p.prof, kKindGather, s, [&] {
      literal_scatter_kernel<E><<<grid_for(nchunks, 1, 1u << 20), kThreads, 0, s>>>(a);
    });
  }
  timed(p.prof, kKindTailSeq, s, [&] {
    tail_sequential_kernel<E><<<grid_for(lv.M, kThreads, 1u << 16), kThreads, 0, s>>>(a);
  });
  timed(p.prof, kKindPatchRead, s,
        [&] { patch_read_kernel<E><<<kResident, kThreads, 0, s>>>(a); });
  timed(p.prof, kKindPatchWrite, s,
        [&] { patch_write_kernel<E><<<kResident, kThreads, 0, s>>>(a); });
  return cudaGetLastError();
}

}  // namespace

namespace {

cudaError_t plan_kernels(const Plan &p, const LevelArgs &a, const LevelPlan &lv, const Buffers &b,
                         cudaStream_t s) {
  const uint64_t nchunks = static_cast<uint64_t>(lv.M) * lv.J;
  timed(p.prof, kKindCount, s, [&] {
    count_kernel<<<grid_for(nchunks, kThreads / 32, 1u << 20), kThreads, 0, s>>>(a);
  });
  timed(p.prof, kKindScan, s,
        [&] { scan_kernel<<<grid_for(lv.M, 1, 1u << 20), kThreads, 0, s>>>(a); });
  timed(p.prof, kKindKscan, s, [&] { kscan_kernel<<<1, 1024, 0, s>>>(a); });
  if (p.flags & MS_FLAG_LITERAL)
    lap_kernel<<<grid_for(lv.M, kThreads, 1u << 16), kThreads, 0, s>>>(a);
  cudaError_t err = cudaSuccess;
  timed(p.prof, kKindHashClear, s, [&] {
    err = cudaMemsetAsync(b.hkeys, 0xFF, sizeof(unsigned long long) << lv.hbits, s);
  });
  if (err != cudaSuccess) return err;
  timed(p.prof, kKindInsert, s, [&] { tail_insert_kernel<<<kResident, kThreads, 0, s>>>(a); });
  timed(p.prof, kKindResolve, s, [&] { tail_resolve_kernel<<<kResident, kThreads, 0, s>>>(a); });
  return cudaGetLastError();
}

template <typename E>
cudaError_t pair_data_t(const Plan &p, const LevelPlan &lv1, const LevelPlan &lv2, const void *in,
                        void *out, const Buffers &b1, const Buffers &b2, uint64_t seed,
                        cudaStream_t s) {
  void *X = const_cast<void *>(in);  // dead after the pair: the fallback's scratch
  const uint32_t *ovf = b1.ctrl + 1;  // level l's tails overflowed its capacity
  PairArgs pa;
  pa.in = in;
  pa.out = out;
  pa.l1 = level_args(p, lv1, in, out, b1, seed);
  pa.l1.zb = b1.zb;
  pa.l2 = level_args(p, lv2, out, out, b2, seed);
  pa.x = exc_args(p, b1);
  pa.xr = b1.xrange;
  const uint64_t nchunks2 = static_cast<uint64_t>(lv2.M) * lv2.J;
  timed(p.prof, kKindPairGather, s, [&] {
    if constexpr (sizeof(E) == 4)
      pair_staged_kernel<<<grid_for(nchunks2, 1, 1u << 20), kStageThreads, 0, s>>>(pa);
    else
      pair_gather_kernel<E><<<grid_for(nchunks2, 1, 1u << 20), kThreads, 0, s>>>(pa);
  });
  // unfused fallback (each kernel returns at once unless level l overflowed): level l from X
  // into out with its tail in order, level l+1 from out back into X
  LevelArgs f1 = level_args(p, lv1, in, out, b1, seed);
  f1.gate = ovf;
  f1.gate_on = 1;
  // (the fallback's gathers loop over their chunks on a resident grid: when gated off, as almost
  // always, each costs one launch of a resident grid rather than one CTA a chunk)
  const uint64_t nchunks1 = static_cast<uint64_t>(lv1.M) * lv1.J;
  gather_kernel<E><<<grid_for(nchunks1, 1, kResident), kThreads, 0, s>>>(f1);
  tail_sequential_kernel<E><<<grid_for(lv1.M, kThreads, 1u << 16), kThreads, 0, s>>>(f1);
  LevelArgs f2 = level_args(p, lv2, out, X, b2, seed);
  f2.gate = ovf;
  f2.gate_on = 1;
  gather_kernel<E><<<grid_for(nchunks2, 1, kResident), kThreads, 0, s>>>(f2);
  // level l+1's tail, on out (fused) or on X (fallback)
  LevelArgs t2 = level_args(p, lv2, nullptr, out, b2, seed);
  t2.out_alt = X;
  t2.alt_sel = ovf;
  timed(p.prof, kKindTailSeq, s, [&] {
    tail_sequential_kernel<E><<<grid_for(lv2.M, kThreads, 1u << 16), kThreads, 0, s>>>(t2);
  });
  timed(p.prof, kKindPatchRead, s,
        [&] { patch_read_kernel<E><<<kResident, kThreads, 0, s>>>(t2); });
  timed(p.prof, kKindPatchWrite, s,
        [&] { patch_write_kernel<E><<<kResident, kThreads, 0, s>>>(t2); });
  LevelArgs cp = level_args(p, lv2, X, out, b2, seed);
  cp.gate = ovf;
  cp.gate_on = 1;
  copy_kernel<E><<<kResident, kThreads, 0, s>>>(cp);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_level_plan(const Plan &p, const LevelPlan &lv, const Buffers &b, uint64_t seed,
                              cudaStream_t s) {
  return plan_kernels(p, level_args(p, lv, nullptr, nullptr, b, seed), lv, b, s);
}

cudaError_t launch_pair_plan(const Plan &p, const LevelPlan &lv1, const LevelPlan &lv2,
                             const Buffers &b1, const Buffers &b2, uint64_t seed, cudaStream_t s) {
  LevelArgs a1 = level_args(p, lv1, nullptr, nullptr, b1, seed);
  a1.zb = b1.zb;
  cudaError_t err = plan_kernels(p, a1, lv1, b1, s);
  if (err != cudaSuccess) return err;
  // the first level's tail moves as exceptions of the pair's data pass: their bitmap and
  // sources, the rank index, then the list in position order
  err = cudaMemsetAsync(b1.xbits, 0, (p.n + 31) / 32 * 4, s);
  if (err != cudaSuccess) return err;
  const ExcArgs x = exc_args(p, b1);
  const uint64_t xtiles = ((p.n + kXBlock - 1) / kXBlock + kXTileBlocks - 1) / kXTileBlocks;
  timed(p.prof, kKindExceptions, s, [&] {
    exceptions_kernel<<<kResident, kThreads, 0, s>>>(a1, x);
    xcount_kernel<<<static_cast<unsigned>(xtiles), kThreads, 0, s>>>(a1, x);
    xtiles_kernel<<<1, 1024, 0, s>>>(a1, x);
    xscatter_kernel<<<kResident, kThreads, 0, s>>>(a1, x);
  });
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  err = plan_kernels(p, level_args(p, lv2, nullptr, nullptr, b2, seed), lv2, b2, s);
  if (err != cudaSuccess) return err;
  // what every chunk of the data pass reads: the records of its two level-l ranges
  PairArgs pa;
  pa.in = nullptr;
  pa.out = nullptr;
  pa.l1 = a1;
  pa.l2 = level_args(p, lv2, nullptr, nullptr, b2, seed);
  pa.x = x;
  pa.xr = b1.xrange;
  const uint64_t nchunks2 = static_cast<uint64_t>(lv2.M) * lv2.J;
  timed(p.prof, kKindExceptions, s, [&] {
    pair_ranges_kernel<<<grid_for(2 * nchunks2, kThreads, kResident), kThreads, 0, s>>>(pa);
  });
  return cudaGetLastError();
}

cudaError_t launch_pair_data(const Plan &p, const LevelPlan &lv1, const LevelPlan &lv2,
                             const void *in, void *out, const Buffers &b1, const Buffers &b2,
                             uint64_t seed, cudaStream_t s) {
  switch (p.w) {
    case 4: return pair_data_t<uint32_t>(p, lv1, lv2, in, out, b1, b2, seed, s);
    case 8: return pair_data_t<uint2>(p, lv1, lv2, in, out, b1, b2, seed, s);
    case 16: return pair_data_t<uint4>(p, lv1, lv2, in, out, b1, b2, seed, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_level_breaks(const Plan &p, const LevelPlan &lv, const Buffers &b,
                                uint64_t seed, cudaStream_t s) {
  const LevelArgs a = level_args(p, lv, nullptr, nullptr, b, seed);
  const uint64_t nchunks = static_cast<uint64_t>(lv.M) * lv.J;
  count_kernel<<<grid_for(nchunks, kThreads / 32, 1u << 20), kThreads, 0, s>>>(a);
  scan_kernel<<<grid_for(lv.M, 1, 1u << 20), kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_level_data(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                              const Buffers &b, uint64_t seed, cudaStream_t s) {
  switch (p.w) {
    case 4: return launch_data_t<uint32_t>(p, lv, in, out, b, seed, s);
    case 8: return launch_data_t<uint2>(p, lv, in, out, b, seed, s);
    case 16: return launch_data_t<uint4>(p, lv, in, out, b, seed, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace msk
