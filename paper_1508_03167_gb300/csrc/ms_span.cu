// ms_span.cu -- one HBM merge level of small merges, streamed span by span through shared
// memory (merges of at most one span: 32 KiB of elements).
//
// A persistent CTA takes spans of 2^m consecutive merges of level l (Algorithm 2 of
// arXiv 1508.03167). For every span:
//   * the input span is copied into shared memory asynchronously (cp.async), one span ahead:
//     while span k is merged, span k+1 is already in flight;
//   * what does not depend on the data runs while the copy lands: coin words, zero prefixes,
//     break steps (Algorithm 3's first loop) and the tail draws;
//   * the stable interleave is gathered into a shared-memory output span, one lane per output
//     position (conflict-free stores; the loads are two runs, one per half);
//   * the tails (Algorithm 3's second loop) run in order in shared memory, one thread per
//     merge, eight swaps at a time whenever those eight provably commute;
//   * the output span is stored coalesced.
#include "ms_merge.cuh"

namespace msk {
namespace {


struct SpanArgs {
  const void *in;
  void *out;
  uint64_t n, q, spans;
  uint2 key;
  uint32_t c, lam, m;  // level, log2(merges per span)
  uint32_t S;          // elements per span buffer (>= every span of the level)
  uint32_t ucap;       // coin words per span (a multiple of four)
  uint32_t tcap;       // tail draws per span made ahead of the data (else made in the loop)
  uint32_t flags;      // MS_FLAG_TAIL_SEQUENTIAL (0x1): draws made in the loop
};

__host__ __device__ __forceinline__ size_t r16(size_t x) { return (x + 15) & ~size_t(15); }

// kThreads = 128 or 256; the register budget (64 a thread) lets 1024 / kThreads CTAs share an SM
template <typename E, int kThreads>
__global__ void __launch_bounds__(kThreads, 1024 / kThreads) span_level_kernel(SpanArgs a) {
  constexpr uint32_t kSpanThreads = kThreads;
  constexpr uint32_t kSpanWarps = kThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t mg[8][kSpanMaxMerges];
  __shared__ uint32_t scratch[33];
  constexpr uint32_t kV = 16u / sizeof(E);  // elements per 16 bytes
  const size_t bufb = r16((static_cast<size_t>(a.S) + kV) * sizeof(E));
  E *const buf0 = reinterpret_cast<E *>(smem_raw);
  E *const buf1 = reinterpret_cast<E *>(smem_raw + bufb);
  E *const Ys = reinterpret_cast<E *>(smem_raw + 2 * bufb);  // merged output span
  uint32_t *const cw = reinterpret_cast<uint32_t *>(smem_raw + 3 * bufb);
  uint32_t *const zp = cw + a.ucap;
  uint16_t *const mv = reinterpret_cast<uint16_t *>(zp + a.ucap);
  uint32_t *const m_s = mg[0];
  uint32_t *const m_n1 = mg[1];
  uint32_t *const m_N = mg[2];
  uint32_t *const m_T = mg[3];
  uint32_t *const m_a = mg[4];
  uint32_t *const m_b = mg[5];
  uint32_t *const m_lb = mg[6];
  uint32_t *const m_off = mg[7];

  const E *const in = static_cast<const E *>(a.in);
  E *const out = static_cast<E *>(a.out);
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint32_t warp = tid >> 5;
  const uint32_t lam = a.lam;
  const uint32_t gl = a.m + lam + 1u;
  const uint32_t Mt = 1u << a.m;
  const uint32_t Nmax = static_cast<uint32_t>(((a.n << (lam + 1u)) + a.q - 1u) >> a.c);
  const uint32_t Wm = (Nmax + 31u) >> 5;
  const uint32_t BPM = (Nmax + 127u) >> 7;
  const uint32_t U = Mt * Wm;
  const uint32_t wm_magic = Wm > 1u ? static_cast<uint32_t>(0x100000000ull / Wm) + 1u : 0u;
  auto merge_of = [&](uint32_t u) { return Wm > 1u ? __umulhi(u, wm_magic) : u; };
  const uint32_t lt = low_mask(lane);

  auto span_range = [&](uint64_t sp, uint64_t &g0, uint32_t &len) {
    const uint64_t lb = sp << gl;
    g0 = boundary(a.n, a.c, lb);
    len = static_cast<uint32_t>(boundary(a.n, a.c, lb + (1ull << gl)) - g0);
  };
  // elements from p to the next 16-byte boundary, and the buffer offset that gives a span
  // starting at global element g the same 16-byte phase in shared memory
  auto phase = [&](const E *base, uint64_t g) {
    return static_cast<uint32_t>((reinterpret_cast<uintptr_t>(base + g) & 15u) / sizeof(E));
  };
  // copy span sp (if any) into buf at its phase; one commit group per call, possibly empty
  auto prefetch = [&](uint64_t sp, E *buf) {
    if (sp < a.spans) {
      uint64_t g0;
      uint32_t len;
      span_range(sp, g0, len);
      const uint32_t ph = phase(in, g0);
      E *dst = buf + ph;
      const E *src = in + g0;
      // head: elements before the first 16-byte boundary, tail: after the last one
      const uint32_t head = min(len, (kV - ph) % kV);
      const uint32_t body = (len - head) / kV;
      const uint32_t tail0 = head + body * kV;
      if (tid < head) cp_async_elem(dst + tid, src + tid);
      for (uint32_t c = tid; c < body; c += kSpanThreads)
        cp_async_elem(reinterpret_cast<uint4 *>(dst + head) + c,
                      reinterpret_cast<const uint4 *>(src + head) + c);
      if (tid < len - tail0) cp_async_elem(dst + tail0 + tid, src + tail0 + tid);
    }
    cp_async_commit();
  };

  uint64_t sp = blockIdx.x;
  prefetch(sp, buf0);
  for (uint32_t it = 0; sp < a.spans; ++it, sp += gridDim.x) {
    prefetch(sp + gridDim.x, (it & 1u) ? buf0 : buf1);
    uint64_t g0;
    uint32_t len;
    span_range(sp, g0, len);
    const E *X = ((it & 1u) ? buf1 : buf0) + phase(in, g0);
    const uint32_t oph = phase(out, g0);
    E *const Yo = Ys + oph;  // the merged span, at the output's 16-byte phase
    const uint64_t lb = sp << gl;
    const uint64_t rbase = lb >> (lam + 1u);

    // ---- geometry, coin words
    if (tid < Mt) {
      const uint64_t L0 = lb + (static_cast<uint64_t>(tid) << (lam + 1u));
      const uint64_t s = boundary(a.n, a.c, L0);
      const uint64_t mid = boundary(a.n, a.c, L0 + (1ull << lam));
      const uint64_t e = boundary(a.n, a.c, L0 + (2ull << lam));
      m_s[tid] = static_cast<uint32_t>(s - g0);
      m_n1[tid] = static_cast<uint32_t>(mid - s);
      m_N[tid] = static_cast<uint32_t>(e - s);
      m_T[tid] = static_cast<uint32_t>(e - s);
    }
    for (uint32_t idx = tid; idx < Mt * BPM; idx += kSpanThreads) {
      const uint32_t r = idx / BPM;
      const uint32_t jb = idx - r * BPM;
      const uint4 blk = coin_block(a.key, lam, static_cast<uint32_t>(rbase + r), jb);
      const uint32_t base = r * Wm + 4u * jb;
      if (4u * jb + 0u < Wm) cw[base + 0u] = blk.x;
      if (4u * jb + 1u < Wm) cw[base + 1u] = blk.y;
      if (4u * jb + 2u < Wm) cw[base + 2u] = blk.z;
      if (4u * jb + 3u < Wm) cw[base + 3u] = blk.w;
    }
    __syncthreads();

    // ---- zero counts per coin word and their exclusive prefix over the span
    {
      const uint32_t per = (U + kSpanThreads - 1u) / kSpanThreads;
      const uint32_t u0 = min(tid * per, U);
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
      uint32_t total;
      uint32_t excl = block_exclusive_scan(local, scratch, &total);
      for (uint32_t u = u0; u < u1; ++u) {
        const uint32_t z = zp[u];
        zp[u] = excl;
        excl += z;
      }
    }
    __syncthreads();

    // ---- break step T: the (n1+1)-th zero or the (n2+1)-th one, whichever comes first
    for (uint32_t u = tid; u < U; u += kSpanThreads) {
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
    __syncthreads();

    // ---- per merge: rebased sources, leftover base, tail length and its prefix
    uint32_t packed = 0;
    if (tid < Mt) {
      const uint32_t r = tid;
      const uint32_t T = m_T[r], N = m_N[r], n1 = m_n1[r], s = m_s[r];
      const uint32_t zbase = zp[r * Wm];
      // position t >= T takes the rest of the half that did not run out, in order; the coin
      // at T names the half that ran out (0: the first half, so t reads X[s + t])
      uint32_t lbase = s;
      if (T < N && ((cw[r * Wm + (T >> 5)] >> (T & 31u)) & 1u)) lbase = s - (N - n1);
      m_lb[r] = lbase;
      m_a[r] = s - zbase;       // X[s + Z], Z = zp - zbase + zeros below t in its word
      m_b[r] = s + n1 + zbase;  // X[s + n1 + t - Z]
      const uint32_t k = N - T;
      const uint32_t quads = k ? ((N - 1u) >> 2) - (T >> 2) + 1u : 0u;
      packed = (quads << 16) | k;
    }
    uint32_t total;
    {
      const uint32_t excl = block_exclusive_scan(packed, scratch, &total);
      if (tid < Mt) m_off[tid] = excl;
    }
    __syncthreads();
    const uint32_t Q = total >> 16;
    const uint32_t K = total & 0xFFFFu;
    const bool drawn = K <= a.tcap && !(a.flags & 1u);

    // ---- tail draws, one Philox block per four consecutive positions
    if (drawn) {
      for (uint32_t gq = tid; gq < Q; gq += kSpanThreads) {
        uint32_t lo = 0, hi = Mt;  // largest r with quad offset <= gq
        while (hi - lo > 1u) {
          const uint32_t mid = (lo + hi) >> 1;
          if ((m_off[mid] >> 16) <= gq) lo = mid;
          else hi = mid;
        }
        const uint32_t r = lo;
        const uint32_t T = m_T[r], N = m_N[r];
        const uint32_t quad = (T >> 2) + (gq - (m_off[r] >> 16));
        const uint32_t id = static_cast<uint32_t>(rbase + r);
        const uint4 w0 = philox10(make_uint4(quad, id, (kTagTail << 16) | lam, 0u), a.key);
        const uint32_t koff = m_off[r] & 0xFFFFu;
#pragma unroll
        for (uint32_t v = 0; v < 4u; ++v) {
          const uint32_t i = 4u * quad + v;
          if (i >= T && i < N)
            mv[koff + (i - T)] = static_cast<uint16_t>(
                draw_with_word0(a.key, kTagTail, lam, id, i, i + 1u, pick_word(w0, v)));
        }
      }
    }
    __syncthreads();

    // ---- this span's data (the newest commit group is the next span's prefetch)
    cp_async_wait<1>();
    __syncthreads();

    // ---- stable interleave and leftover copy into the output span
    {
      constexpr uint32_t kWords = sizeof(E) >= 16 ? 2u : 4u;
      for (uint32_t u0 = warp * kWords; u0 < U; u0 += kSpanWarps * kWords) {
        uint32_t cwv[kWords], zpv[kWords];
        if (u0 + kWords <= U) {
          if constexpr (kWords == 4) {
            const uint4 c4 = *reinterpret_cast<const uint4 *>(cw + u0);
            const uint4 z4 = *reinterpret_cast<const uint4 *>(zp + u0);
            cwv[0] = c4.x; cwv[1] = c4.y; cwv[2] = c4.z; cwv[3] = c4.w;
            zpv[0] = z4.x; zpv[1] = z4.y; zpv[2] = z4.z; zpv[3] = z4.w;
          } else {
            const uint2 c2 = *reinterpret_cast<const uint2 *>(cw + u0);
            const uint2 z2 = *reinterpret_cast<const uint2 *>(zp + u0);
            cwv[0] = c2.x; cwv[1] = c2.y;
            zpv[0] = z2.x; zpv[1] = z2.y;
          }
        } else {
#pragma unroll
          for (uint32_t k = 0; k < kWords; ++k) {
            cwv[k] = u0 + k < U ? cw[u0 + k] : 0u;
            zpv[k] = u0 + k < U ? zp[u0 + k] : 0u;
          }
        }
        const uint32_t r0 = merge_of(u0);
        const bool one_merge = merge_of(min(u0 + kWords - 1u, U - 1u)) == r0;
        const uint32_t N0 = m_N[r0], T0 = m_T[r0], A0 = m_a[r0], B0 = m_b[r0], L0 = m_lb[r0],
                       s0 = m_s[r0];
        E v[kWords];
        const uint32_t j0 = u0 - r0 * Wm;
        if (one_merge && u0 + kWords <= U && 32u * (j0 + kWords) <= T0) {
          // every position of the four words precedes the break step: coins decide them all
          const uint32_t t0 = 32u * j0 + lane;
#pragma unroll
          for (uint32_t k = 0; k < kWords; ++k) {
            const uint32_t word = cwv[k];
            const uint32_t t = t0 + 32u * k;
            const uint32_t z = zpv[k] + __popc(~word & lt);
            v[k] = X[min(((word >> lane) & 1u) ? B0 + t - z : A0 + z, a.S - 1u)];
          }
#pragma unroll
          for (uint32_t k = 0; k < kWords; ++k) Yo[s0 + t0 + 32u * k] = v[k];
          continue;
        }
        uint32_t dst[kWords];
#pragma unroll
        for (uint32_t k = 0; k < kWords; ++k) {
          dst[k] = kNone;
          const uint32_t u = u0 + k;
          if (u < U) {
            uint32_t r = r0, N = N0, T = T0, aa = A0, bb = B0, lbase = L0, sb = s0;
            if (!one_merge) {
              r = merge_of(u);
              N = m_N[r]; T = m_T[r]; aa = m_a[r]; bb = m_b[r]; lbase = m_lb[r]; sb = m_s[r];
            }
            const uint32_t t = 32u * (u - r * Wm) + lane;
            if (t < N) {
              const uint32_t word = cwv[k];
              const uint32_t z = zpv[k] + __popc(~word & lt);  // Z + zbase at t
              const uint32_t src =
                  (t < T) ? (((word >> lane) & 1u) ? bb + t - z : aa + z) : lbase + t;
              v[k] = X[min(src, a.S - 1u)];  // clamp keeps the read inside the buffer
              dst[k] = sb + t;
            }
          }
        }
#pragma unroll
        for (uint32_t k = 0; k < kWords; ++k)
          if (dst[k] != kNone) Yo[dst[k]] = v[k];
      }
    }
    __syncthreads();

    // ---- random insertion of positions T..N-1, in order, one thread per merge
    {
      constexpr uint32_t kBatch = sizeof(E) >= 16 ? 4u : 8u;
      for (uint32_t r = tid; r < Mt; r += kSpanThreads) {
        const uint32_t T = m_T[r], N = m_N[r];
        E *C = Yo + m_s[r];
        uint32_t i = T;
        if (drawn) {
          const uint16_t *mk = mv + (m_off[r] & 0xFFFFu);  // mk[i - T] = draw of position i
          while (i < N) {
            if (i + kBatch <= N) {
              // swaps (i+k, m_k) for k < kBatch commute when every m_k lies before the window
              // and all m_k differ: then they touch 2*kBatch distinct positions
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
          // more tail steps than the draw buffer holds: draws made in the loop
          const uint32_t id = static_cast<uint32_t>(rbase + r);
          DrawMemo memo;
          for (; i < N; ++i)
            swap_smem(C, i, draw_uniform(a.key, kTagTail, lam, id, i, i + 1u, memo));
        }
      }
    }
    __syncthreads();

    // ---- store the merged span: element stores up to the first and from the last 16-byte
    // boundary of the output range, 16-byte stores in between
    {
      E *const Y = out + g0;
      const uint32_t head = min(len, (kV - oph) % kV);
      const uint32_t body = (len - head) / kV;
      const uint32_t tail0 = head + body * kV;
      if (tid < head) Y[tid] = Yo[tid];
      const uint4 *vs = reinterpret_cast<const uint4 *>(Yo + head);
      uint4 *vd = reinterpret_cast<uint4 *>(Y + head);
      uint32_t c = tid;
      for (; c + kSpanThreads < body; c += 2u * kSpanThreads) {
        const uint4 x0 = vs[c], x1 = vs[c + kSpanThreads];
        vd[c] = x0;
        vd[c + kSpanThreads] = x1;
      }
      for (; c < body; c += kSpanThreads) vd[c] = vs[c];
      if (tid < len - tail0) Y[tail0 + tid] = Yo[tail0 + tid];
    }
    __syncthreads();  // the span buffers and per-merge values are reused
  }
  cp_async_wait<0>();  // nothing in flight at exit
}

template <typename E, int kThreads>
cudaError_t launch_t(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                     uint64_t seed, cudaStream_t s) {
  SpanArgs a;
  a.in = in;
  a.out = out;
  a.n = p.n;
  a.q = p.q;
  a.spans = p.q >> (lv.mlog + lv.level + 1u);
  a.key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  a.c = p.c;
  a.lam = lv.level;
  a.m = lv.mlog;
  a.S = lv.span_max;
  a.ucap = lv.ucap;
  a.tcap = lv.tcap;
  a.flags = p.flags;
  auto kern = span_level_kernel<E, kThreads>;
  cudaError_t err = allow_dynamic_smem(kern, lv.smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, lv.smem);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorUnknown;
  const uint64_t resident = static_cast<uint64_t>(per_sm > 0 ? per_sm : 1) * sms;
  const uint64_t grid = a.spans < resident ? a.spans : resident;
  if (p.prof) p.prof->begin(kKindLocal, s);
  kern<<<static_cast<unsigned>(grid), kThreads, lv.smem, s>>>(a);
  if (p.prof) p.prof->end(s);
  return cudaGetLastError();
}

}  // namespace

size_t span_smem_bytes(uint32_t S, uint32_t w, uint32_t ucap, uint32_t tcap) {
  return 3 * r16((static_cast<size_t>(S) + 16u / w) * w) + r16(2ull * ucap * 4 + 2ull * tcap);
}

cudaError_t launch_span_level(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                              uint64_t seed, cudaStream_t s) {
  const bool small = lv.span_threads == 128;
  switch (p.w) {
    case 4: return small ? launch_t<uint32_t, 128>(p, lv, in, out, seed, s)
                         : launch_t<uint32_t, 256>(p, lv, in, out, seed, s);
    case 8: return small ? launch_t<uint2, 128>(p, lv, in, out, seed, s)
                         : launch_t<uint2, 256>(p, lv, in, out, seed, s);
    case 16: return small ? launch_t<uint4, 128>(p, lv, in, out, seed, s)
                          : launch_t<uint4, 256>(p, lv, in, out, seed, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace msk
