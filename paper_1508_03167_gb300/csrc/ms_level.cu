// ms_level.cu -- one merge level of Algorithm 2 (arXiv 1508.03167) streamed through HBM.
//
// Every merge r of level l joins two shuffled halves [s, mid) and [mid, e). The merge is split
// into data-oblivious planning and one streaming pass:
//   count    zero coins per 4096-step chunk of every merge (Philox only, no array traffic);
//   scan     per merge: exclusive prefix of the chunk counts and the break step T, where a coin
//            first asks for an exhausted half (Algorithm 3's first loop);
//   kscan    prefix of the tail lengths N - T over the level's merges;
//   insert   tail draws m_i (i = T..N-1, uniform in {0..i}) into a hash table keyed by
//            (merge, target position);
//   resolve  replays the random insertions (Algorithm 3's second loop) on indices only: every
//            displaced element's trajectory gives one (destination, source) patch;
//   gather   the streaming pass: out[s+t] = coin t ? B[t - Z_t] : A[Z_t] for t < T, the
//            remainder of the non-exhausted half for t >= T (coalesced reads of both halves);
//   patch    two small kernels apply the patches (read all sources, then write).
// If a level's tails exceed the planned capacity, a sequential per-merge tail (in place on the
// output) runs instead of insert/resolve/patch; the result is the same.
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
};

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
    if (128ull * blk < N) z = block_zero_count(coin_block(a.key, a.level, r, blk), blk, N);
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
    const uint32_t J = (N + kChunk - 1u) / kChunk;  // chunks of this merge (<= a.J)
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
    if (r < a.M) a.minfo[r].z = carry + excl;
    carry += total;
  }
  if (threadIdx.x == 0) {
    a.ctrl[0] = carry;
    a.ctrl[1] = (carry > a.kcap || (a.flags & 1u)) ? 1u : 0u;
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
  uint32_t lo = 0, hi = a.M;  // invariant: offset[lo] <= g, and offset[hi] > g or hi == M
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
    const uint32_t m = draw_uniform(a.key, kTagTail, a.level, r, i, i + 1u);
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
  const E *out = static_cast<const E *>(a.out);
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
  E *out = static_cast<E *>(a.out);
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
  E *out = static_cast<E *>(a.out);
  for (uint32_t r = blockIdx.x * kThreads + threadIdx.x; r < a.M; r += gridDim.x * kThreads) {
    const uint4 mi = a.minfo[r];
    const MergeBounds mb = merge_bounds(a, r);
    const uint32_t N = static_cast<uint32_t>(mb.e - mb.s);
    E *c = out + mb.s;
    DrawMemo memo;
    for (uint32_t i = mi.x; i < N; ++i) {
      const uint32_t m = draw_uniform(a.key, kTagTail, a.level, r, i, i + 1u, memo);
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
    const uint32_t t1 = min(t0 + kChunk, N);
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
  return a;
}

constexpr unsigned kResident = 152u * 8u;

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
  timed(p.prof, kKindGather, s, [&] {
    gather_kernel<E><<<grid_for(nchunks, 1, 1u << 20), kThreads, 0, s>>>(a);
  });
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

cudaError_t launch_level_plan(const Plan &p, const LevelPlan &lv, const Buffers &b, uint64_t seed,
                              cudaStream_t s) {
  const LevelArgs a = level_args(p, lv, nullptr, nullptr, b, seed);
  const uint64_t nchunks = static_cast<uint64_t>(lv.M) * lv.J;
  timed(p.prof, kKindCount, s, [&] {
    count_kernel<<<grid_for(nchunks, kThreads / 32, 1u << 20), kThreads, 0, s>>>(a);
  });
  timed(p.prof, kKindScan, s,
        [&] { scan_kernel<<<grid_for(lv.M, 1, 1u << 20), kThreads, 0, s>>>(a); });
  timed(p.prof, kKindKscan, s, [&] { kscan_kernel<<<1, 1024, 0, s>>>(a); });
  cudaError_t err = cudaSuccess;
  timed(p.prof, kKindHashClear, s, [&] {
    err = cudaMemsetAsync(b.hkeys, 0xFF, sizeof(unsigned long long) << lv.hbits, s);
  });
  if (err != cudaSuccess) return err;
  timed(p.prof, kKindInsert, s, [&] { tail_insert_kernel<<<kResident, kThreads, 0, s>>>(a); });
  timed(p.prof, kKindResolve, s, [&] { tail_resolve_kernel<<<kResident, kThreads, 0, s>>>(a); });
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
