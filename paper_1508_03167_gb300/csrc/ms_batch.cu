// ms_batch.cu -- batched MergeShuffle (arXiv 1508.03167) for many independent instances.
//
// One persistent launch: every CTA repeatedly takes the next instance from an atomic queue
// (instances are queued largest first) and runs the whole of Algorithm 2 on it alone, so no CTA
// ever waits for another:
//   * Fisher-Yates on the base blocks (Algorithm 1), one thread per block, blocks staged in
//     shared memory at an odd stride;
//   * every merge level whose merges fit the shared-memory span buffer: groups of up to 16
//     merges staged and merged in shared memory (the merge routine shared with the other
//     kernels), tails included;
//   * larger merges: zero counts of the coins per 4096-step chunk, their prefix and the break
//     step, then a chunk-by-chunk streaming gather from one buffer to the other, then the merge
//     tail (Algorithm 3's random insertions) replayed on indices through a hash table in the
//     CTA's own scratch and applied as patches.
// Instances too large for one CTA are run by the single-instance path (same result).
#include "ms_merge.cuh"

namespace msk {
namespace {

constexpr int kEngThreads = 256;
constexpr uint32_t kEngWarps = kEngThreads / 32;

struct BatchInst {
  uint64_t data;   // caller's array (device pointer)
  uint64_t tmp;    // ping-pong partner in the workspace (device pointer)
  uint64_t n;
  uint64_t seed;
  uint32_t flags;  // bit 0: run by the single-instance path, skipped by the engine
  uint32_t pad;
};

struct EngineArgs {
  const BatchInst *inst;  // queue order
  uint32_t k;
  uint32_t perm;          // 1: fill each instance with the permutation of 0..n-1
  uint32_t *queue;        // next queue index (reset before the launch)
  uint32_t B;
  uint32_t span_bytes;    // shared-memory budget of a staged span / base-block group
  unsigned char *scratch; // per-CTA tail scratch
  size_t scratch_per_cta;
  uint32_t kcap;          // tail steps handled by the parallel replay
  uint32_t hbits;         // hash slots 2^hbits
};

constexpr uint32_t kEmpty = 0xFFFFFFFFu;

template <typename E>
__device__ __forceinline__ E make_elem(uint32_t v);
template <>
__device__ __forceinline__ uint32_t make_elem<uint32_t>(uint32_t v) { return v; }
template <>
__device__ __forceinline__ uint2 make_elem<uint2>(uint32_t v) { return make_uint2(v, 0u); }
template <>
__device__ __forceinline__ uint4 make_elem<uint4>(uint32_t v) { return make_uint4(v, 0u, 0u, 0u); }

// bytes of a staged span of 2^m merges on level lvl (stage + coin words + prefixes + draws)
template <typename E>
__device__ __forceinline__ uint64_t span_bytes_needed(const LeafArgs &a, uint32_t lvl,
                                                      uint32_t m) {
  const uint32_t gl = m + lvl + 1u;
  const uint64_t span_max = ((a.n << gl) + a.q - 1u) >> a.c;
  const uint64_t Nmax = ((a.n << (lvl + 1u)) + a.q - 1u) >> a.c;
  const uint64_t units = ((1ull << m) * ((Nmax + 31u) >> 5) + 3u) & ~3ull;
  const uint64_t tcap = (span_max / 4u + 16u) & ~1ull;
  return span_max * sizeof(E) + 16u + units * 8u + tcap * 2u + 64u;
}

// per-CTA scratch layout (global memory): hash keys, hash values, draws, destinations
struct TailScratch {
  uint32_t *hkeys, *hvals, *mv, *d1, *d2;
};

__device__ __forceinline__ uint32_t eng_hash(uint32_t key, uint32_t hbits) {
  return (key * 0x9E3779B1u) >> (32u - hbits);
}

// smallest tail step > after whose draw targets position pos (kEmpty if none)
__device__ __forceinline__ uint32_t eng_next(const TailScratch &t, uint32_t hbits, uint32_t pos,
                                             uint32_t after) {
  const uint32_t mask = (1u << hbits) - 1u;
  uint32_t best = kEmpty;
  uint32_t h = eng_hash(pos, hbits);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const uint32_t k = t.hkeys[h];
    if (k == kEmpty) break;
    if (k == pos) {
      const uint32_t v = t.hvals[h];
      if (v > after && v < best) best = v;
    }
    h = (h + 1u) & mask;
  }
  return best;
}

__device__ __forceinline__ bool eng_earlier(const TailScratch &t, uint32_t hbits, uint32_t pos,
                                            uint32_t before) {
  const uint32_t mask = (1u << hbits) - 1u;
  uint32_t h = eng_hash(pos, hbits);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const uint32_t k = t.hkeys[h];
    if (k == kEmpty) return false;
    if (k == pos && t.hvals[h] < before) return true;
    h = (h + 1u) & mask;
  }
  return false;
}

// A large merge of one instance, streamed from src to dst by the whole CTA.
template <typename E>
__device__ void cta_big_merge(const LeafArgs &a, const EngineArgs &g, const TailScratch &ts,
                              uint32_t lvl, uint32_t r, E *src, E *dst, uint32_t *sm) {
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint64_t L0 = static_cast<uint64_t>(r) << (lvl + 1u);
  const uint64_t s = boundary(a.n, a.c, L0);
  const uint64_t mid = boundary(a.n, a.c, L0 + (1ull << lvl));
  const uint64_t e = boundary(a.n, a.c, L0 + (2ull << lvl));
  const uint32_t n1 = static_cast<uint32_t>(mid - s);
  const uint32_t N = static_cast<uint32_t>(e - s);
  const uint32_t n2 = N - n1;
  const uint32_t J = (N + kChunk - 1u) / kChunk;
  // shared memory: chunk prefix [J], coin words [128], word prefix [128], scan scratch [33],
  // control words [8]
  uint32_t *cpre = sm;
  uint32_t *cw = cpre + J;
  uint32_t *zw = cw + kChunk / 32u;
  uint32_t *scr = zw + kChunk / 32u;
  uint32_t *ctl = scr + 33;

  // ---- zero coins per chunk
  for (uint32_t jc = warp; jc < J; jc += kEngWarps) {
    const uint32_t blk = jc * (kChunk / 128u) + lane;
    uint32_t z = 0;
    if (128ull * blk < N) {
      const uint4 cb = coin_block(a.key, lvl, r, blk);
      const uint32_t valid = (N - 128u * blk < 128u) ? N - 128u * blk : 128u;
      z += __popc(~cb.x & low_mask(min(valid, 32u)));
      z += __popc(~cb.y & low_mask(valid > 32u ? min(valid - 32u, 32u) : 0u));
      z += __popc(~cb.z & low_mask(valid > 64u ? min(valid - 64u, 32u) : 0u));
      z += __popc(~cb.w & low_mask(valid > 96u ? valid - 96u : 0u));
    }
    z = warp_sum(z);
    if (lane == 0) cpre[jc] = z;
  }
  if (tid == 0) {
    ctl[0] = kEmpty;  // chunk holding the (n1+1)-th zero
    ctl[2] = kEmpty;  // chunk holding the (n2+1)-th one
  }
  __syncthreads();
  // ---- exclusive prefix over chunks; locate the break chunks
  {
    uint32_t carry = 0;
    for (uint32_t base = 0; base < J; base += kEngThreads) {
      const uint32_t jc = base + tid;
      const uint32_t v = jc < J ? cpre[jc] : 0u;
      uint32_t total;
      const uint32_t excl = carry + block_exclusive_scan(v, scr, &total);
      if (jc < J) {
        cpre[jc] = excl;
        const uint32_t len = min(kChunk, N - jc * kChunk);
        const uint32_t Ob = jc * kChunk - excl;
        if (excl <= n1 && n1 < excl + v) {
          ctl[0] = jc;
          ctl[1] = n1 - excl;
        }
        if (Ob <= n2 && n2 < Ob + (len - v)) {
          ctl[2] = jc;
          ctl[3] = n2 - Ob;
        }
      }
      carry += total;
    }
  }
  __syncthreads();
  // ---- break step T (warp 0: zero break, warp 1: one break)
  if (warp < 2u) {
    const uint32_t chunk = ctl[2u * warp];
    uint32_t found = kEmpty;
    if (chunk != kEmpty) {
      const uint32_t rank = ctl[2u * warp + 1u];
      const bool want_one = warp == 1u;
      const uint32_t blk = chunk * (kChunk / 128u) + lane;
      uint4 cb = make_uint4(0, 0, 0, 0);
      uint32_t cnt = 0, valid = 0;
      if (128ull * blk < N) {
        cb = coin_block(a.key, lvl, r, blk);
        valid = (N - 128u * blk < 128u) ? N - 128u * blk : 128u;
        uint32_t z = 0;
        z += __popc(~cb.x & low_mask(min(valid, 32u)));
        z += __popc(~cb.y & low_mask(valid > 32u ? min(valid - 32u, 32u) : 0u));
        z += __popc(~cb.z & low_mask(valid > 64u ? min(valid - 64u, 32u) : 0u));
        z += __popc(~cb.w & low_mask(valid > 96u ? valid - 96u : 0u));
        cnt = want_one ? valid - z : z;
      }
      const uint32_t incl = warp_inclusive_scan(cnt);
      const uint32_t excl = incl - cnt;
      if (cnt > 0 && excl <= rank && rank < incl) {
        uint32_t kk = rank - excl;
        const uint32_t words[4] = {cb.x, cb.y, cb.z, cb.w};
        for (uint32_t wi = 0; wi < 4u; ++wi) {
          const uint32_t vb = valid > 32u * wi ? min(valid - 32u * wi, 32u) : 0u;
          const uint32_t m = (want_one ? words[wi] : ~words[wi]) & low_mask(vb);
          const uint32_t pc = __popc(m);
          if (kk < pc) {
            found = 128u * blk + 32u * wi + select_set_bit(m, kk);
            break;
          }
          kk -= pc;
        }
      }
      const unsigned ball = __ballot_sync(kFullMask, found != kEmpty);
      found = ball ? __shfl_sync(kFullMask, found, __ffs(static_cast<int>(ball)) - 1) : kEmpty;
    }
    if (lane == 0) ctl[4u + warp] = found;
  }
  __syncthreads();
  uint32_t T = N, ZT = n1;
  {
    const uint32_t tz = ctl[4], to = ctl[5];
    if (tz != kEmpty && tz < T) {
      T = tz;
      ZT = n1;
    }
    if (to != kEmpty && to < T) {
      T = to;
      ZT = T - n2;
    }
  }
  const bool first_exhausted = (ZT == n1);

  // ---- streaming gather, chunk by chunk
  const E *A = src + s;
  E *C = dst + s;
  constexpr uint32_t kBatch = sizeof(E) >= 16 ? 8u : 16u;
  constexpr uint32_t kWordsPerWarp = kChunk / 32u / kEngWarps;
  for (uint32_t jc = 0; jc < J; ++jc) {
    const uint32_t t0 = jc * kChunk;
    const uint32_t t1 = min(t0 + kChunk, N);
    if (tid < kChunk / 128u) {
      const uint4 cb = coin_block(a.key, lvl, r, jc * (kChunk / 128u) + tid);
      cw[4u * tid + 0u] = cb.x;
      cw[4u * tid + 1u] = cb.y;
      cw[4u * tid + 2u] = cb.z;
      cw[4u * tid + 3u] = cb.w;
    }
    __syncthreads();
    {
      uint32_t z = 0;
      if (tid < kChunk / 32u) {
        const uint32_t tw = t0 + 32u * tid;
        const uint32_t valid = tw >= N ? 0u : min(32u, N - tw);
        z = __popc(~cw[tid] & low_mask(valid));
      }
      uint32_t total;
      const uint32_t excl = block_exclusive_scan(z, scr, &total);
      if (tid < kChunk / 32u) zw[tid] = excl;
    }
    __syncthreads();
    const uint32_t Z0 = cpre[jc];
#pragma unroll
    for (uint32_t b0 = 0; b0 < kWordsPerWarp; b0 += kBatch) {
      E v[kBatch];
#pragma unroll
      for (uint32_t kk = 0; kk < kBatch; ++kk) {
        const uint32_t u = warp + (b0 + kk) * kEngWarps;
        const uint32_t t = t0 + 32u * u + lane;
        if (t < t1) {
          uint32_t sidx;
          if (t < T) {
            const uint32_t word = cw[u];
            const uint32_t Z = Z0 + zw[u] + __popc(~word & low_mask(lane));
            sidx = ((word >> lane) & 1u) ? n1 + (t - Z) : Z;
          } else if (first_exhausted) {
            sidx = t;
          } else {
            sidx = t - n2;
          }
          v[kk] = A[min(sidx, N - 1u)];
        }
      }
#pragma unroll
      for (uint32_t kk = 0; kk < kBatch; ++kk) {
        const uint32_t t = t0 + 32u * (warp + (b0 + kk) * kEngWarps) + lane;
        if (t < t1) C[t] = v[kk];
      }
    }
    __syncthreads();
  }

  // ---- merge tail: positions T..N-1, replayed on indices
  const uint32_t K = N - T;
  if (K == 0) return;
  const uint32_t id = r;
  if (K > g.kcap) {  // never expected for the instance sizes this engine takes: serial fallback
    if (tid == 0) {
      DrawMemo memo;
      for (uint32_t i = T; i < N; ++i) {
        const uint32_t m = draw_uniform(a.key, kTagTail, lvl, id, i, i + 1u, memo);
        const E t = C[i];
        C[i] = C[m];
        C[m] = t;
      }
    }
    __syncthreads();
    return;
  }
  const uint32_t hbits = g.hbits;
  const uint32_t hslots = 1u << hbits;
  for (uint32_t h = tid; h < hslots; h += kEngThreads) ts.hkeys[h] = kEmpty;
  __syncthreads();
  for (uint32_t st = tid; st < K; st += kEngThreads) {
    const uint32_t i = T + st;
    const uint32_t m = draw_uniform(a.key, kTagTail, lvl, id, i, i + 1u);
    ts.mv[st] = m;
    uint32_t h = eng_hash(m, hbits);
    for (uint32_t probe = 0; probe < hslots; ++probe) {
      if (atomicCAS(&ts.hkeys[h], kEmpty, m) == kEmpty) {
        ts.hvals[h] = i;
        break;
      }
      h = (h + 1u) & (hslots - 1u);
    }
  }
  __syncthreads();
  // trajectories: the element at position i = T+st lands at m at time i, then moves to every
  // later step that targets its position; the element first displaced from m < T follows the
  // same rule from position i
  for (uint32_t st = tid; st < K; st += kEngThreads) {
    const uint32_t i = T + st;
    const uint32_t m = ts.mv[st];
    uint32_t pos = m, time = i;
    for (;;) {
      const uint32_t nx = eng_next(ts, hbits, pos, time);
      if (nx == kEmpty) break;
      pos = nx;
      time = nx;
    }
    ts.d1[st] = pos;
    uint32_t d2 = kEmpty;
    if (m < T && !eng_earlier(ts, hbits, m, i)) {
      pos = i;
      time = i;
      for (;;) {
        const uint32_t nx = eng_next(ts, hbits, pos, time);
        if (nx == kEmpty) break;
        pos = nx;
        time = nx;
      }
      d2 = pos;
    }
    ts.d2[st] = d2;
  }
  __syncthreads();
  // The values move through this merge's source range, which the level no longer needs:
  // slot st holds the element of tail position T+st, slot K+m the element first displaced
  // from prefix position m < T (K + m < K + T = N). All reads finish before any write.
  E *vals = src + s;
  for (uint32_t st = tid; st < K; st += kEngThreads) {
    vals[st] = C[T + st];
    if (ts.d2[st] != kEmpty) vals[K + ts.mv[st]] = C[ts.mv[st]];
  }
  __syncthreads();
  for (uint32_t st = tid; st < K; st += kEngThreads) {
    const uint32_t d1 = ts.d1[st];
    if (d1 != T + st) C[d1] = vals[st];
    const uint32_t d2 = ts.d2[st];
    if (d2 != kEmpty) C[d2] = vals[K + ts.mv[st]];
  }
  __syncthreads();
}

template <typename E>
__global__ void __launch_bounds__(kEngThreads, 2) engine_kernel(EngineArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t scan_scratch[33];
  __shared__ uint32_t merges[8][kGroupMerges];
  __shared__ uint32_t s_idx;
  TailScratch ts;
  {
    unsigned char *base = g.scratch + g.scratch_per_cta * blockIdx.x;
    const size_t slots = static_cast<size_t>(1u) << g.hbits;
    ts.hkeys = reinterpret_cast<uint32_t *>(base);
    ts.hvals = ts.hkeys + slots;
    ts.mv = ts.hvals + slots;
    ts.d1 = ts.mv + g.kcap;
    ts.d2 = ts.d1 + g.kcap;
  }
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  for (;;) {
    if (tid == 0) s_idx = atomicAdd(g.queue, 1u);
    __syncthreads();
    const uint32_t idx = s_idx;
    __syncthreads();
    if (idx >= g.k) break;
    const BatchInst I = g.inst[idx];
    if ((I.flags & 1u) || I.n <= 1) continue;

    LeafArgs a;
    a.n = I.n;
    a.key = make_uint2(static_cast<uint32_t>(I.seed), static_cast<uint32_t>(I.seed >> 32));
    uint32_t c = 0;
    while ((a.n >> c) > g.B) ++c;
    a.c = c;
    a.q = 1ull << c;
    a.d = 0;
    a.dw = 0;
    const uint32_t leaf_max = static_cast<uint32_t>((a.n + a.q - 1) >> c);
    a.stride = leaf_max | 1u;
    E *data = reinterpret_cast<E *>(I.data);
    E *tmp = reinterpret_cast<E *>(I.tmp);

    // ---- Algorithm 1 on every base block: groups of up to 256 blocks in shared memory
    E *fy_dst = (c % 2u == 0u) ? data : tmp;  // after c merge levels the result is in data
    {
      E *blocks = reinterpret_cast<E *>(smem_raw);
      uint32_t per = g.span_bytes / (a.stride * static_cast<uint32_t>(sizeof(E)));
      per = max(1u, min(per, static_cast<uint32_t>(kEngThreads)));
      for (uint64_t lb = 0; lb < a.q; lb += per) {
        const uint32_t cnt = static_cast<uint32_t>(a.q - lb < per ? a.q - lb : per);
        for (uint32_t k = warp; k < cnt; k += kEngWarps) {
          const uint64_t bs = boundary(a.n, c, lb + k);
          const uint32_t L = static_cast<uint32_t>(boundary(a.n, c, lb + k + 1) - bs);
          if (g.perm) {
            for (uint32_t i = lane; i < L; i += 32u)
              blocks[k * a.stride + i] = make_elem<E>(static_cast<uint32_t>(bs + i));
          } else {
            for (uint32_t i = lane; i < L; i += 32u) blocks[k * a.stride + i] = data[bs + i];
          }
        }
        __syncthreads();
        if (tid < cnt) {
          const uint64_t leaf = lb + tid;
          const uint32_t L = static_cast<uint32_t>(boundary(a.n, c, leaf + 1) -
                                                   boundary(a.n, c, leaf));
          fisher_yates_block(blocks + tid * a.stride, L, static_cast<uint32_t>(leaf), a.key);
        }
        __syncthreads();
        for (uint32_t k = warp; k < cnt; k += kEngWarps) {
          const uint64_t bs = boundary(a.n, c, lb + k);
          const uint32_t L = static_cast<uint32_t>(boundary(a.n, c, lb + k + 1) - bs);
          for (uint32_t i = lane; i < L; i += 32u) fy_dst[bs + i] = blocks[k * a.stride + i];
        }
        __syncthreads();
      }
    }

    // ---- merge levels
    E *cur = fy_dst;
    E *other = (cur == data) ? tmp : data;
    for (uint32_t lvl = 0; lvl < c; ++lvl) {
      const uint64_t Nmax = ((a.n << (lvl + 1u)) + a.q - 1u) >> c;
      const uint64_t M = a.q >> (lvl + 1u);
      if (span_bytes_needed<E>(a, lvl, 0u) <= g.span_bytes) {
        // staged spans of up to 16 merges
        uint32_t m = 0;
        while (m < kLocalMaxMergesLog && (M >> (m + 1u)) >= 1u &&
               span_bytes_needed<E>(a, lvl, m + 1u) <= g.span_bytes)
          ++m;
        const uint32_t gl = m + lvl + 1u;
        const uint64_t span_max = ((a.n << gl) + a.q - 1u) >> c;
        const uint32_t Mt = 1u << m;
        const uint32_t Wm = static_cast<uint32_t>((Nmax + 31u) >> 5);
        a.tile_max = static_cast<uint32_t>(span_max);
        a.ucap_c = (Mt * Wm + 3u) & ~3u;  // the prefixes start 16-byte aligned too
        a.tcap_c = static_cast<uint32_t>((span_max / 4u + 16u) & ~1ull);
        GroupSmem S;
        E *stage = reinterpret_cast<E *>(smem_raw);
        S.cw = reinterpret_cast<uint32_t *>(align16(stage + span_max));
        S.zp = S.cw + a.ucap_c;
        S.mv = reinterpret_cast<uint16_t *>(S.zp + a.ucap_c);
        S.ucap = a.ucap_c;
        S.tcap = a.tcap_c;
        S.m_a = merges[0]; S.m_b = merges[1]; S.m_s = merges[2]; S.m_n1 = merges[3];
        S.m_N = merges[4]; S.m_T = merges[5]; S.m_off = merges[6]; S.m_lb = merges[7];
        S.scratch = scan_scratch;
        const uint64_t spans = a.q >> gl;
        for (uint64_t sp = 0; sp < spans; ++sp) {
          const uint64_t lb = sp << gl;
          const uint64_t g0 = boundary(a.n, c, lb);
          const uint32_t len = static_cast<uint32_t>(boundary(a.n, c, lb + (1ull << gl)) - g0);
          // X is global here: the tails run in shared memory, in order (no patch scratch)
          merge_level<kEngWarps, E>(a, S, lb, lb, g0, lvl, gl, cur + g0, len, false, stage,
                                    nullptr, 0u);
          for (uint32_t i = tid; i < len; i += kEngThreads) other[g0 + i] = stage[i];
          __syncthreads();
        }
      } else {
        uint32_t *sm = reinterpret_cast<uint32_t *>(smem_raw);
        for (uint64_t r = 0; r < M; ++r) {
          cta_big_merge<E>(a, g, ts, lvl, static_cast<uint32_t>(r), cur, other, sm);
          __syncthreads();
        }
      }
      E *t = cur;
      cur = other;
      other = t;
    }
    __syncthreads();
  }
}

}  // namespace

// Host side of the engine launch (the tables are already in the workspace).
cudaError_t launch_engine(uint32_t w, bool perm, const void *inst, uint32_t k, uint32_t *queue,
                          uint32_t B, void *scratch, size_t scratch_per_cta, uint32_t kcap,
                          uint32_t hbits, uint32_t grid, size_t smem, cudaStream_t s, Prof *prof) {
  EngineArgs g;
  g.inst = static_cast<const BatchInst *>(inst);
  g.k = k;
  g.perm = perm ? 1u : 0u;
  g.queue = queue;
  g.B = B;
  g.span_bytes = static_cast<uint32_t>(smem);
  g.scratch = static_cast<unsigned char *>(scratch);
  g.scratch_per_cta = scratch_per_cta;
  g.kcap = kcap;
  g.hbits = hbits;
  cudaError_t err = cudaMemsetAsync(queue, 0, sizeof(uint32_t), s);
  if (err != cudaSuccess) return err;
  auto launch = [&](auto kern) -> cudaError_t {
    cudaError_t e = allow_dynamic_smem(kern, smem);
    if (e != cudaSuccess) return e;
    if (prof) prof->begin(kKindEngine, s);
    kern<<<grid, kEngThreads, smem, s>>>(g);
    if (prof) prof->end(s);
    return cudaGetLastError();
  };
  switch (w) {
    case 4: return launch(engine_kernel<uint32_t>);
    case 8: return launch(engine_kernel<uint2>);
    case 16: return launch(engine_kernel<uint4>);
    default: return cudaErrorInvalidValue;
  }
}

size_t engine_inst_bytes() { return sizeof(BatchInst); }

}  // namespace msk
