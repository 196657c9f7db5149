// ms_wlevel.cu -- one HBM merge level of small merges, one warp per span of merges.
//
// Each warp takes 2^m consecutive merges of level l (Algorithm 2 of arXiv 1508.03167) and
// finishes them alone, with warp barriers only, straight from one global buffer to the other:
//   coins, zero prefix and break step T of every merge in shared memory (Algorithm 3's first
//   loop); the stable interleave written directly to the output with one lane per position, so
//   every store instruction covers 32 consecutive elements and every load instruction two short
//   runs of the halves; then the merge tails (Algorithm 3's second loop) resolved in parallel:
//   every draw is computed, every displaced element's final position is found by following the
//   later insertions that target it, and the moves are applied as patches (all values read
//   first, through the merge's input range, which the level no longer needs, then written).
// No staging buffer: a warp needs a few KiB of shared memory, so many warps share an SM.
#include "ms_merge.cuh"

namespace msk {
namespace {

constexpr uint32_t kWlWarps = 4;
constexpr uint32_t kWlMerges = 16;
constexpr uint32_t kNoPos = 0xFFFFFFFFu;
constexpr uint16_t kNoPos16 = 0xFFFFu;  // merges here have fewer than 2^16 positions

struct WlArgs {
  void *in;  // read as the level's input, reused as patch scratch afterwards
  void *out;
  uint64_t n, q;
  uint2 key;
  uint32_t c;
  uint32_t lam, m;   // level and log2(merges per span)
  uint32_t ucap;     // coin words per span
  uint32_t tcap;     // tail steps per span resolved in parallel
  uint32_t warp_bytes;
};

// smallest tail step index s' in [from, k) with mv[s'] == pos, or kNoPos
__device__ __forceinline__ uint32_t wl_next(const uint16_t *mv, uint32_t from, uint32_t k,
                                            uint32_t pos) {
  for (uint32_t s = from; s < k; ++s)
    if (mv[s] == pos) return s;
  return kNoPos;
}

template <typename E>
__global__ void __launch_bounds__(kWlWarps * 32, 8) warp_stream_level_kernel(WlArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t mrg[kWlWarps][8][kWlMerges];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  uint32_t *const cw = reinterpret_cast<uint32_t *>(smem_raw + warp * a.warp_bytes);
  uint32_t *const zp = cw + a.ucap;
  uint16_t *const mv = reinterpret_cast<uint16_t *>(zp + a.ucap);  // tail draws
  uint16_t *const d1 = mv + a.tcap;  // final position of each tail element
  uint16_t *const d2 = d1 + a.tcap;  // final position of the prefix element it displaced
  uint32_t *const m_s = mrg[warp][0];
  uint32_t *const m_n1 = mrg[warp][1];
  uint32_t *const m_N = mrg[warp][2];
  uint32_t *const m_T = mrg[warp][3];
  uint32_t *const m_aa = mrg[warp][4];
  uint32_t *const m_bb = mrg[warp][5];
  uint32_t *const m_lb = mrg[warp][6];
  uint32_t *const m_off = mrg[warp][7];

  E *const in = static_cast<E *>(a.in);
  E *const out = static_cast<E *>(a.out);
  const uint32_t lam = a.lam;
  const uint32_t gl = a.m + lam + 1u;
  const uint32_t Mt = 1u << a.m;
  const uint64_t spans = a.q >> gl;
  const uint32_t Nmax = static_cast<uint32_t>(((a.n << (lam + 1u)) + a.q - 1u) >> a.c);
  const uint32_t Wm = (Nmax + 31u) >> 5;
  const uint32_t BPM = (Nmax + 127u) >> 7;
  const uint32_t U = Mt * Wm;
  const uint32_t wm_magic = Wm > 1u ? static_cast<uint32_t>(0x100000000ull / Wm) + 1u : 0u;
  auto merge_of = [&](uint32_t u) { return Wm > 1u ? __umulhi(u, wm_magic) : u; };

  for (uint64_t sp = static_cast<uint64_t>(blockIdx.x) * kWlWarps + warp; sp < spans;
       sp += static_cast<uint64_t>(gridDim.x) * kWlWarps) {
    const uint64_t lb = sp << gl;
    const uint64_t g0 = boundary(a.n, a.c, lb);
    E *const X = in + g0;
    E *const Y = out + g0;
    const uint64_t rbase = lb >> (lam + 1u);

    // ---- geometry (span-relative positions)
    if (lane < Mt) {
      const uint64_t L0 = lb + (static_cast<uint64_t>(lane) << (lam + 1u));
      const uint64_t s = boundary(a.n, a.c, L0);
      const uint64_t mid = boundary(a.n, a.c, L0 + (1ull << lam));
      const uint64_t e = boundary(a.n, a.c, L0 + (2ull << lam));
      m_s[lane] = static_cast<uint32_t>(s - g0);
      m_n1[lane] = static_cast<uint32_t>(mid - s);
      m_N[lane] = static_cast<uint32_t>(e - s);
      m_T[lane] = static_cast<uint32_t>(e - s);
    }
    // ---- coins
    for (uint32_t idx = lane; idx < Mt * BPM; idx += 32u) {
      const uint32_t r = idx / BPM;
      const uint32_t jb = idx - r * BPM;
      const uint4 blk = coin_block(a.key, lam, static_cast<uint32_t>(rbase + r), jb);
      const uint32_t base = r * Wm + 4u * jb;
      if (4u * jb + 0u < Wm) cw[base + 0u] = blk.x;
      if (4u * jb + 1u < Wm) cw[base + 1u] = blk.y;
      if (4u * jb + 2u < Wm) cw[base + 2u] = blk.z;
      if (4u * jb + 3u < Wm) cw[base + 3u] = blk.w;
    }
    __syncwarp();
    // ---- zero counts and their exclusive prefix over the span's words
    {
      const uint32_t per = (U + 31u) >> 5;
      const uint32_t u0 = min(lane * per, U);
      const uint32_t u1 = min(u0 + per, U);
      uint32_t local = 0;
      for (uint32_t u = u0; u < u1; ++u) {
        const uint32_t r = merge_of(u);
        const uint32_t j = u - r * Wm;
        const uint32_t N = m_N[r];
        const uint32_t valid = (32u * j >= N) ? 0u : min(32u, N - 32u * j);
        const uint32_t z = __popc(~cw[u] & low_mask(valid));
        zp[u] = z;
        local += z;
      }
      const uint32_t incl = warp_inclusive_scan(local);
      uint32_t excl = incl - local;
      for (uint32_t u = u0; u < u1; ++u) {
        const uint32_t z = zp[u];
        zp[u] = excl;
        excl += z;
      }
    }
    __syncwarp();
    // ---- break step T of every merge
    for (uint32_t u = lane; u < U; u += 32u) {
      const uint32_t r = merge_of(u);
      const uint32_t j = u - r * Wm;
      const uint32_t N = m_N[r];
      if (32u * j >= N) continue;
      const uint32_t valid = min(32u, N - 32u * j);
      const uint32_t vm = low_mask(valid);
      const uint32_t word = cw[u];
      const uint32_t Zs = zp[u] - zp[r * Wm];
      const uint32_t Os = 32u * j - Zs;
      const uint32_t zeros = __popc(~word & vm);
      const uint32_t ones = valid - zeros;
      const uint32_t n1 = m_n1[r];
      const uint32_t n2 = N - n1;
      if (Zs <= n1 && n1 < Zs + zeros)
        atomicMin(&m_T[r], 32u * j + select_set_bit(~word & vm, n1 - Zs));
      if (Os <= n2 && n2 < Os + ones)
        atomicMin(&m_T[r], 32u * j + select_set_bit(word & vm, n2 - Os));
    }
    __syncwarp();
    // ---- per merge: rebased sources, leftover base, tail length and its prefix
    uint32_t k = 0;
    if (lane < Mt) {
      const uint32_t r = lane;
      const uint32_t T = m_T[r], N = m_N[r], n1 = m_n1[r], s = m_s[r];
      const uint32_t zbase = zp[r * Wm];
      uint32_t lbase = s;  // first half exhausted: the second half's rest is X[s + t]
      if (T < N) {
        const uint32_t bitT = (cw[r * Wm + (T >> 5)] >> (T & 31u)) & 1u;
        if (bitT) lbase = s - (N - n1);  // second half exhausted: X[s + t - n2]
      }
      m_lb[r] = lbase;
      m_aa[r] = s - zbase;       // X[s + Z], Z = zp[u] - zbase + zeros below the lane
      m_bb[r] = s + n1 + zbase;  // X[s + n1 + t - Z]
      k = N - T;
    }
    const uint32_t kincl = warp_inclusive_scan(k);
    if (lane < Mt) m_off[lane] = kincl - k;
    const uint32_t K = __shfl_sync(kFullMask, kincl, 31);
    __syncwarp();  // the per-merge values above are read by every lane below

    // ---- stable interleave and leftover copy, global to global: lane = position in a word,
    // merge by merge (its bases in registers), eight words per batch, loads before stores
    for (uint32_t r = 0; r < Mt; ++r) {
      const uint32_t N = m_N[r], T = m_T[r], s = m_s[r];
      const uint32_t aa = m_aa[r], bb = m_bb[r], lbase = m_lb[r];
      const uint32_t Wr = (N + 31u) >> 5;
      const uint32_t *cwr = cw + r * Wm;
      const uint32_t *zpr = zp + r * Wm;
      const uint32_t last = s + N - 1u;
      for (uint32_t j0 = 0; j0 < Wr; j0 += 8u) {
        E v[8];
#pragma unroll
        for (uint32_t kk = 0; kk < 8u; ++kk) {
          const uint32_t j = j0 + kk;
          const uint32_t t = 32u * j + lane;
          if (j < Wr && t < N) {
            uint32_t src;
            if (t < T) {
              const uint32_t word = cwr[j];
              const uint32_t Z = zpr[j] + __popc(~word & low_mask(lane));
              src = ((word >> lane) & 1u) ? bb + t - Z : aa + Z;
            } else {
              src = lbase + t;
            }
            v[kk] = X[min(src, last)];  // clamp keeps the read inside the merge
          }
        }
#pragma unroll
        for (uint32_t kk = 0; kk < 8u; ++kk) {
          const uint32_t j = j0 + kk;
          const uint32_t t = 32u * j + lane;
          if (j < Wr && t < N) Y[s + t] = v[kk];
        }
      }
    }
    __syncwarp();

    // ---- merge tails (Algorithm 3's second loop)
    if (K <= a.tcap) {
      // draws: tail step st of merge r is position i = T_r + st, uniform in {0..i}
      for (uint32_t g = lane; g < K; g += 32u) {
        uint32_t r = 0;
        while (r + 1u < Mt && m_off[r + 1u] <= g) ++r;
        const uint32_t i = m_T[r] + (g - m_off[r]);
        mv[g] = static_cast<uint16_t>(
            draw_uniform(a.key, kTagTail, lam, static_cast<uint32_t>(rbase + r), i, i + 1u));
      }
      __syncwarp();
      // trajectories: the element at tail position i lands at m at time i and moves to every
      // later step that targets its position; the element first displaced from m < T follows
      // the same rule from position i
      for (uint32_t g = lane; g < K; g += 32u) {
        uint32_t r = 0;
        while (r + 1u < Mt && m_off[r + 1u] <= g) ++r;
        const uint32_t T = m_T[r];
        const uint32_t k_r = m_N[r] - T;
        const uint16_t *mr = mv + m_off[r];  // mr[st] = draw of position T + st
        const uint32_t st = g - m_off[r];
        const uint32_t m = mr[st];
        uint32_t pos = m, from = st + 1u;
        for (;;) {
          const uint32_t nx = wl_next(mr, from, k_r, pos);
          if (nx == kNoPos) break;
          pos = T + nx;
          from = nx + 1u;
        }
        d1[g] = static_cast<uint16_t>(pos);
        uint32_t p2 = kNoPos16;
        if (m < T) {
          bool first = true;
          for (uint32_t s2 = 0; s2 < st; ++s2) first &= (mr[s2] != m);
          if (first) {
            pos = T + st;
            from = st + 1u;
            for (;;) {
              const uint32_t nx = wl_next(mr, from, k_r, pos);
              if (nx == kNoPos) break;
              pos = T + nx;
              from = nx + 1u;
            }
            p2 = pos;
          }
        }
        d2[g] = static_cast<uint16_t>(p2);
      }
      __syncwarp();
      // patches: values pass through the merge's input range (slot st: tail element, slot
      // k_r + m: prefix element m < T; k_r + T = N), all read before any write
      for (uint32_t g = lane; g < K; g += 32u) {
        uint32_t r = 0;
        while (r + 1u < Mt && m_off[r + 1u] <= g) ++r;
        const uint32_t T = m_T[r], s = m_s[r];
        const uint32_t k_r = m_N[r] - T;
        const uint32_t st = g - m_off[r];
        E *vals = X + s;
        vals[st] = Y[s + T + st];
        if (d2[g] != kNoPos16) vals[k_r + mv[g]] = Y[s + mv[g]];
      }
      __syncwarp();
      for (uint32_t g = lane; g < K; g += 32u) {
        uint32_t r = 0;
        while (r + 1u < Mt && m_off[r + 1u] <= g) ++r;
        const uint32_t T = m_T[r], s = m_s[r];
        const uint32_t k_r = m_N[r] - T;
        const uint32_t st = g - m_off[r];
        const E *vals = X + s;
        if (d1[g] != T + st) Y[s + d1[g]] = vals[st];
        if (d2[g] != kNoPos16) Y[s + d2[g]] = vals[k_r + mv[g]];
      }
      __syncwarp();
    } else if (lane < Mt) {
      // more tail steps than the parallel replay holds: Algorithm 3's loop as printed
      const uint32_t r = lane;
      const uint32_t T = m_T[r], N = m_N[r];
      E *C = Y + m_s[r];
      DrawMemo memo;
      for (uint32_t i = T; i < N; ++i) {
        const uint32_t m = draw_uniform(a.key, kTagTail, lam, static_cast<uint32_t>(rbase + r),
                                        i, i + 1u, memo);
        const E t = C[i];
        C[i] = C[m];
        C[m] = t;
      }
    }
    __syncwarp();
  }
}

template <typename E>
cudaError_t launch_t(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                     uint64_t seed, cudaStream_t s) {
  WlArgs a;
  a.in = const_cast<void *>(in);
  a.out = out;
  a.n = p.n;
  a.q = p.q;
  a.key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  a.c = p.c;
  a.lam = lv.level;
  a.m = lv.mlog;
  a.ucap = lv.ucap;
  a.tcap = lv.tcap;
  a.warp_bytes = lv.warp_bytes;
  auto kern = warp_stream_level_kernel<E>;
  const size_t smem = static_cast<size_t>(lv.warp_bytes) * kWlWarps;
  cudaError_t err = allow_dynamic_smem(kern, smem);
  if (err != cudaSuccess) return err;
  const uint64_t spans = p.q >> (lv.mlog + lv.level + 1u);
  const uint64_t blocks = (spans + kWlWarps - 1) / kWlWarps;
  const uint64_t grid = blocks < 1048576ull ? blocks : 1048576ull;
  if (p.prof) p.prof->begin(kKindLocal, s);
  kern<<<static_cast<unsigned>(grid), kWlWarps * 32, smem, s>>>(a);
  if (p.prof) p.prof->end(s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_warp_level(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                              uint64_t seed, cudaStream_t s) {
  switch (p.w) {
    case 4: return launch_t<uint32_t>(p, lv, in, out, seed, s);
    case 8: return launch_t<uint2>(p, lv, in, out, seed, s);
    case 16: return launch_t<uint4>(p, lv, in, out, seed, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace msk
