// ms_leaf.cu -- the base-block kernel: one CTA per tile of 2^d consecutive base blocks.
//
// A tile is loaded into shared memory (or generated as the identity for perm), every base block
// is shuffled by Fisher-Yates (Algorithm 1 of arXiv 1508.03167, descending form), and merge
// levels 0..d-1 of Algorithm 2 run inside shared memory with the stable random merge (Algorithm 3:
// coin interleave until one half is exhausted, leftovers in order, then random insertion).
// The tile is written back once, so this kernel is the first of the 1 + (c - d) HBM passes.
//
// Two phases, both running the same group-generic merge level:
//   warp phase  each warp owns 2^dw consecutive base blocks (one lane per block for Fisher-Yates)
//               and merges them through levels 0..dw-1 on its own, with warp barriers only;
//   CTA phase   the 2^(d-dw) <= 8 warp results are merged through levels dw..d-1 by the whole
//               CTA.
// Base blocks sit at an odd stride in buffer 0, so the lanes of a warp (all at the same
// Fisher-Yates step i) hit 32 different banks; merge level 0 reads that layout and writes
// buffer 1 contiguously; later levels ping-pong between the buffers.
// Every gather takes one lane per output position (conflict-free stores, loads in two runs) and
// issues several words' loads before their stores; every merge tail (the random insertions) has
// its draws and the final positions of the elements it moves computed in parallel, then the
// moved values are read into the level's dead input buffer and written back.
#include <algorithm>

#include "mergeshuffle.h"
#include "ms_merge.cuh"

namespace msk {
namespace {

template <typename E, bool kPerm>
__global__ void __launch_bounds__(kLeafThreads, 2) leaf_kernel(LeafArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t scan_scratch[33];
  __shared__ uint32_t merges[kLeafWarps][8][kGroupMerges];

  E *const buf0 = reinterpret_cast<E *>(smem_raw);
  E *const buf1 = buf0 + a.buf0;
  unsigned char *const aux = align16(buf1 + a.tile_max);

  const E *in = static_cast<const E *>(a.in);
  E *out = static_cast<E *>(a.out);
  const uint64_t tiles = a.q >> a.d;
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint32_t warp = tid >> 5;
  const uint32_t P = a.stride;
  const uint32_t dc = a.d - a.dw;            // CTA-phase levels
  const uint32_t nwt = 1u << dc;             // warp tiles per CTA tile (<= 8)
  const uint32_t wleaves = 1u << a.dw;       // base blocks per warp tile

  // this warp's group views (warp phase) and the CTA's (CTA phase, aliasing warp 0's merges)
  GroupSmem Sw;
  {
    unsigned char *base = aux + warp * a.aux_w;
    Sw.cw = reinterpret_cast<uint32_t *>(base);
    Sw.zp = Sw.cw + a.ucap_w;
    Sw.mv = reinterpret_cast<uint16_t *>(Sw.zp + a.ucap_w);
    Sw.ucap = a.ucap_w;
    Sw.tcap = a.tcap_w;
    Sw.m_a = merges[warp][0]; Sw.m_b = merges[warp][1]; Sw.m_s = merges[warp][2];
    Sw.m_n1 = merges[warp][3]; Sw.m_N = merges[warp][4]; Sw.m_T = merges[warp][5];
    Sw.m_off = merges[warp][6]; Sw.m_lb = merges[warp][7];
    Sw.scratch = scan_scratch;
  }
  GroupSmem Sc;
  {
    Sc.cw = reinterpret_cast<uint32_t *>(aux);
    Sc.zp = Sc.cw + a.ucap_c;
    Sc.mv = reinterpret_cast<uint16_t *>(Sc.zp + a.ucap_c);
    Sc.ucap = a.ucap_c;
    Sc.tcap = a.tcap_c;
    Sc.m_a = merges[0][0]; Sc.m_b = merges[0][1]; Sc.m_s = merges[0][2];
    Sc.m_n1 = merges[0][3]; Sc.m_N = merges[0][4]; Sc.m_T = merges[0][5];
    Sc.m_off = merges[0][6]; Sc.m_lb = merges[0][7];
    Sc.scratch = scan_scratch;
  }

  for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint64_t leaf0 = tile << a.d;
    const uint64_t g0 = boundary(a.n, a.c, leaf0);
    const uint64_t g1 = boundary(a.n, a.c, leaf0 + (1ull << a.d));
    const uint32_t len = static_cast<uint32_t>(g1 - g0);

    // ---------------- load: one warp per base block (perm: the identity is generated) -------
    const uint32_t nleaves = 1u << a.d;
    for (uint32_t k = warp; k < nleaves; k += kLeafWarps) {
      const uint64_t bs = boundary(a.n, a.c, leaf0 + k);
      const uint32_t L = static_cast<uint32_t>(boundary(a.n, a.c, leaf0 + k + 1) - bs);
      E *blk = buf0 + k * P;
      if constexpr (kPerm) {
        for (uint32_t i = lane; i < L; i += 32u) blk[i] = static_cast<E>(bs + i);
      } else {
        for (uint32_t i = lane; i < L; i += 32u) blk[i] = in[bs + i];
      }
    }
    __syncthreads();
    // ---------------- Algorithm 1: one thread per base block (odd stride: distinct banks) ----
    for (uint32_t k = tid; k < nleaves; k += kLeafThreads) {
      const uint64_t leaf = leaf0 + k;
      const uint32_t L = static_cast<uint32_t>(boundary(a.n, a.c, leaf + 1) -
                                               boundary(a.n, a.c, leaf));
      fisher_yates_block(buf0 + k * P, L, static_cast<uint32_t>(leaf), a.key);
    }
    __syncthreads();
    if (warp < nwt) {
      // ---------------- warp phase: base blocks [lb, lb + 2^dw) ----------------
      const uint64_t lb = leaf0 + static_cast<uint64_t>(warp) * wleaves;
      if (a.dw > 0)
        merge_level<1, E>(a, Sw, lb, leaf0, g0, 0u, a.dw, buf0, a.buf0, true, buf1,
                          buf0 + warp * wleaves * P, wleaves * P);
    }
    // buffer 0 switches from the padded layout to the contiguous one
    __syncthreads();
    E *X = (a.dw > 0) ? buf1 : buf0;
    E *Y = (a.dw > 0) ? buf0 : buf1;
    if (warp < nwt) {
      const uint64_t lb = leaf0 + static_cast<uint64_t>(warp) * wleaves;
      // this warp's range of the tile (its tail scratch on every warp level)
      const uint32_t w0 = static_cast<uint32_t>(boundary(a.n, a.c, lb) - g0);
      const uint32_t wn = static_cast<uint32_t>(boundary(a.n, a.c, lb + wleaves) - g0) - w0;
      for (uint32_t lam = 1; lam < a.dw; ++lam) {
        merge_level<1, E>(a, Sw, lb, leaf0, g0, lam, a.dw, X, a.tile_max, false, Y, X + w0, wn);
        E *t = X;
        X = Y;
        Y = t;
      }
    } else if (a.dw > 1) {
      for (uint32_t lam = 1; lam < a.dw; ++lam) {  // keep the buffer roles in step
        E *t = X;
        X = Y;
        Y = t;
      }
    }
    __syncthreads();
    // ---------------- CTA phase: levels dw..d-1 ----------------
    for (uint32_t lam = a.dw; lam < a.d; ++lam) {
      const bool padded = (lam == 0);  // only when the warp phase is empty
      merge_level<kLeafWarps, E>(a, Sc, leaf0, leaf0, g0, lam, a.d, X,
                                 padded ? a.buf0 : a.tile_max, padded, Y, X,
                                 padded ? a.buf0 : a.tile_max);
      E *t = X;
      X = Y;
      Y = t;
    }
    // ---------------- store ----------------
    // d = 0: the tile is one base block at offset 0 of buffer 0
    const E *res = (a.d == 0) ? buf0 : X;
    for (uint32_t i = tid; i < len; i += kLeafThreads) out[g0 + i] = res[i];
    __syncthreads();
  }
}

// Fisher-Yates only (d = 0): one warp per CTA, one lane per base block. The blocks of a CTA sit
// at an odd stride in shared memory, so the lanes (all at the same step) hit distinct banks.
// Loads and stores go block by block with all 32 lanes, so global accesses stay coalesced.
template <typename E, bool kPerm>
__global__ void __launch_bounds__(32) fy_kernel(LeafArgs a, uint32_t per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E *const blocks = reinterpret_cast<E *>(smem_raw);
  const E *in = static_cast<const E *>(a.in);
  E *out = static_cast<E *>(a.out);
  const uint32_t lane = threadIdx.x;
  const uint32_t P = a.stride;
  const uint64_t groups = (a.q + per_cta - 1) / per_cta;
  for (uint64_t gidx = blockIdx.x; gidx < groups; gidx += gridDim.x) {
    const uint64_t lb = gidx * per_cta;
    const uint32_t cnt = static_cast<uint32_t>(a.q - lb < per_cta ? a.q - lb : per_cta);
    if constexpr (kPerm) {
      if (lane < cnt) {
        const uint64_t bs = boundary(a.n, a.c, lb + lane);
        const uint32_t L = static_cast<uint32_t>(boundary(a.n, a.c, lb + lane + 1) - bs);
        E *blk = blocks + lane * P;
        for (uint32_t i = 0; i < L; ++i) blk[i] = static_cast<E>(bs + i);
      }
    } else {
      for (uint32_t k = 0; k < cnt; ++k) {
        const uint64_t bs = boundary(a.n, a.c, lb + k);
        const uint32_t L = static_cast<uint32_t>(boundary(a.n, a.c, lb + k + 1) - bs);
        E *blk = blocks + k * P;
        for (uint32_t i = lane; i < L; i += 32u) blk[i] = in[bs + i];
      }
    }
    __syncwarp();
    if (lane < cnt) {
      const uint64_t leaf = lb + lane;
      const uint32_t L = static_cast<uint32_t>(boundary(a.n, a.c, leaf + 1) -
                                               boundary(a.n, a.c, leaf));
      fisher_yates_block(blocks + lane * P, L, static_cast<uint32_t>(leaf), a.key);
    }
    __syncwarp();
    for (uint32_t k = 0; k < cnt; ++k) {
      const uint64_t bs = boundary(a.n, a.c, lb + k);
      const uint32_t L = static_cast<uint32_t>(boundary(a.n, a.c, lb + k + 1) - bs);
      const E *blk = blocks + k * P;
      for (uint32_t i = lane; i < L; i += 32u) out[bs + i] = blk[i];
    }
    __syncwarp();
  }
}

// Fisher-Yates only, on indices (d = 0, elements of 8 or 16 bytes, base blocks of at most
// kIdxMaxLeaf elements): the lane of each base block shuffles the 32-bit indices 0..L-1 in shared
// memory (the draws and swaps of Algorithm 1, so the block ends up as in[perm]), then the warp
// gathers the block's elements through them: out[b + i] = in[b + idx[i]]. Shared memory per
// block is 4 bytes an element instead of w, so more warps fit an SM. When out and in are the
// same array a block is read whole into registers before any of it is written.
constexpr uint32_t kIdxMaxLeaf = 256;
template <typename E>
__global__ void __launch_bounds__(32) fy_index_kernel(LeafArgs a, uint32_t per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *const idx = reinterpret_cast<uint32_t *>(smem_raw);
  const E *in = static_cast<const E *>(a.in);
  E *out = static_cast<E *>(a.out);
  const bool in_place = static_cast<const void *>(in) == static_cast<const void *>(out);
  const uint32_t lane = threadIdx.x;
  const uint32_t P = a.stride;
  const uint64_t groups = (a.q + per_cta - 1) / per_cta;
  for (uint64_t gidx = blockIdx.x; gidx < groups; gidx += gridDim.x) {
    const uint64_t lb = gidx * per_cta;
    const uint32_t cnt = static_cast<uint32_t>(a.q - lb < per_cta ? a.q - lb : per_cta);
    if (lane < cnt) {
      const uint64_t leaf = lb + lane;
      const uint32_t L = static_cast<uint32_t>(boundary(a.n, a.c, leaf + 1) -
                                               boundary(a.n, a.c, leaf));
      uint32_t *blk = idx + lane * P;
      for (uint32_t i = 0; i < L; ++i) blk[i] = i;
      fisher_yates_block(blk, L, static_cast<uint32_t>(leaf), a.key);
    }
    __syncwarp();
    constexpr uint32_t kPer = kIdxMaxLeaf / 32;
    for (uint32_t k = 0; k < cnt; ++k) {
      const uint64_t bs = boundary(a.n, a.c, lb + k);
      const uint32_t L = static_cast<uint32_t>(boundary(a.n, a.c, lb + k + 1) - bs);
      const uint32_t *blk = idx + k * P;
      E v[kPer];
#pragma unroll
      for (uint32_t j = 0; j < kPer; ++j) {
        const uint32_t i = lane + 32u * j;
        if (i < L) v[j] = in[bs + blk[i]];
      }
      if (in_place) __syncwarp();  // the whole block is read before any of it is written
#pragma unroll
      for (uint32_t j = 0; j < kPer; ++j) {
        const uint32_t i = lane + 32u * j;
        if (i < L) out[bs + i] = v[j];
      }
      __syncwarp();
    }
  }
}

// Algorithm 1 on every base block with uniform draws by the Fast Dice Roller (MS_FLAG_FDR): one
// thread per block copies it to the output (a perm writes its positions) and swaps there, in
// order, i = L-1 .. 1 with j from stream (LEAF, 0, block, i). The output is out of place or the
// input itself; a thread touches only its own block. (Used for an in-place shuffle.)
template <typename E, bool kPerm>
__global__ void __launch_bounds__(128) fy_fdr_kernel(const E *in, E *out, uint64_t n, uint32_t c,
                                                    uint2 key) {
  const uint64_t q = 1ull << c;
  for (uint64_t k = static_cast<uint64_t>(blockIdx.x) * 128u + threadIdx.x; k < q;
       k += static_cast<uint64_t>(gridDim.x) * 128u) {
    const uint64_t s0 = boundary(n, c, k);
    const uint32_t L = static_cast<uint32_t>(boundary(n, c, k + 1) - s0);
    E *const o = out + s0;
    for (uint32_t i = 0; i < L; ++i) {
      if constexpr (kPerm) o[i] = static_cast<E>(s0 + i);
      else if (in != out) o[i] = in[s0 + i];
    }
    for (uint32_t i = L; i-- > 1u;) {
      uint32_t nb;
      const uint32_t j = min(draw_fdr(key, kTagLeaf, 0u, static_cast<uint32_t>(k), i, i + 1u, &nb), i);
      const E t = o[i];
      o[i] = o[j];
      o[j] = t;
    }
  }
}

// Algorithm 1 on every base block out of place, on eight-warp CTAs with 16-bit local indices in
// shared memory (stride P = 2 mod 64 a block), a batch of `lanes` consecutive base blocks at a
// time (block k of the batch on lane k): all eight warps make the draws (warp w: quads w, w + 8,
// ... of every block; one Philox block serves a quad's four first words, and a draw that needs
// more than its first word is queued by its thread and finished after the loop), warp 0 runs
// the swap chains, and a warp per block writes it through the indices. kFdr selects the Fast
// Dice Roller draws (MS_FLAG_FDR), else the rejection draws of the other kernels.
constexpr uint32_t kFdrWarps = 8u;
constexpr uint32_t kFdrThreads = 32u * kFdrWarps;
constexpr uint32_t kFdrFail = 8u;  // queued draws a thread

// The Fast Dice Roller of draw_fdr on word 0 of its stream alone: true with the value if the
// word's bits decide it (the loop then stops exactly where draw_fdr's does).
__device__ __forceinline__ bool fdr_first_word(uint32_t word, uint32_t R, uint32_t &x) {
  uint32_t v = 1u, c = 0u;  // (v < 2R and c < v throughout)
  for (uint32_t u = 0; u < 32u; ++u) {
    v <<= 1;
    c = (c << 1) | ((word >> u) & 1u);
    if (v >= R) {
      if (c < R) {
        x = c;
        return true;
      }
      v -= R;
      c -= R;
    }
  }
  return false;
}

// The whole draw of position pos of block id (from word 0 of its stream on).
template <bool kFdr>
__device__ __forceinline__ uint32_t fy8_draw(uint2 key, uint32_t id, uint32_t pos) {
  if constexpr (kFdr) {
    uint32_t nb;
    return draw_fdr(key, kTagLeaf, 0u, id, pos, pos + 1u, &nb);
  } else {
    return draw_continue(key, kTagLeaf, 0u, id, pos, pos + 1u);
  }
}

template <typename E, bool kPerm, bool kFdr>
__global__ void __launch_bounds__(kFdrThreads) fy8_kernel(const E *in, E *out, uint64_t n,
                                                         uint32_t c, uint2 key, uint32_t P,
                                                         uint32_t lanes) {
  extern __shared__ __align__(16) uint16_t fdr_smem[];
  uint16_t *const Abuf = fdr_smem;
  uint16_t *const Dbuf = fdr_smem + lanes * P;
  uint16_t *const F = Dbuf + lanes * P;
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint32_t warp = tid >> 5;
  const uint64_t q = 1ull << c;
  for (uint64_t k0 = static_cast<uint64_t>(blockIdx.x) * lanes; k0 < q;
       k0 += static_cast<uint64_t>(gridDim.x) * lanes) {
    const uint32_t kb = (q - k0 < lanes) ? static_cast<uint32_t>(q - k0) : lanes;
    // draws
    if (lane < kb) {
      const uint64_t k = k0 + lane;
      const uint32_t id = static_cast<uint32_t>(k);
      const uint32_t L = min(static_cast<uint32_t>(boundary(n, c, k + 1) - boundary(n, c, k)),
                             P - 2u);
      uint16_t *const A = Abuf + lane * P;
      uint16_t *const D = Dbuf + lane * P;
      uint16_t *const Fq = F + tid * kFdrFail;
      const uint32_t nq = L ? ((L - 1u) >> 2) + 1u : 0u;
      uint32_t nf = 0;
#pragma unroll 2
      for (uint32_t qd = warp; qd < nq; qd += kFdrWarps) {
        const uint4 blk = philox10(make_uint4(qd, id, kTagLeaf << 16, 0u), key);
        // (rejection draws: the slice width of the quad's ranges; positions 1..3 of quad 0 take
        // the general draw)
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
              bool ok;
              if constexpr (kFdr) {
                ok = fdr_first_word(word, pos + 1u, x);
              } else {
                ok = qd ? draw_first_word_b(word, pos + 1u, qb, qmask, 2u * qb, 3u * qb, x)
                        : draw_first_word(word, pos + 1u, x);
              }
              if (ok) {
                D[pos] = static_cast<uint16_t>(x);
              } else if (nf < kFdrFail) {
                Fq[nf++] = static_cast<uint16_t>(pos);
              } else {
                D[pos] = static_cast<uint16_t>(fy8_draw<kFdr>(key, id, pos));
              }
            }
          }
        }
      }
      for (uint32_t e = 0; e < nf; ++e) {
        const uint32_t pos = Fq[e];
        D[pos] = static_cast<uint16_t>(fy8_draw<kFdr>(key, id, pos));
      }
    }
    __syncthreads();
    // swaps, i = L-1 .. 1, four steps a group (the draws clamped to the block)
    if (warp == 0u && lane < kb) {
      const uint64_t k = k0 + lane;
      const uint32_t L = min(static_cast<uint32_t>(boundary(n, c, k + 1) - boundary(n, c, k)),
                             P - 2u);
      uint16_t *const A = Abuf + lane * P;
      const uint16_t *const D = Dbuf + lane * P;
      fy_chain16(A, D, L);
    }
    __syncthreads();
    // the blocks through their indices, a warp per block
    constexpr uint32_t kRows = sizeof(E) >= 16u ? 4u : 8u;
    for (uint32_t kk = warp; kk < kb; kk += kFdrWarps) {
      const uint64_t k = k0 + kk;
      const uint64_t s0 = boundary(n, c, k);
      const uint32_t L = min(static_cast<uint32_t>(boundary(n, c, k + 1) - s0), P - 2u);
      const uint16_t *const A = Abuf + kk * P;
      for (uint32_t i0 = 0; i0 < L; i0 += 32u * kRows) {
        E v[kRows];
#pragma unroll
        for (uint32_t u = 0; u < kRows; ++u) {
          const uint32_t i = i0 + 32u * u + lane;
          if (i < L) {
            const uint32_t src = min(static_cast<uint32_t>(A[i]), L - 1u);
            if constexpr (kPerm) v[u] = static_cast<E>(s0 + src);
            else v[u] = in[s0 + src];
          }
        }
#pragma unroll
        for (uint32_t u = 0; u < kRows; ++u) {
          const uint32_t i = i0 + 32u * u + lane;
          if (i < L) out[s0 + i] = v[u];
        }
      }
    }
    __syncthreads();
  }
}

template <typename E, bool kPerm>
cudaError_t launch_leaf_t(const Plan &p, const void *in, void *out, uint64_t seed,
                          cudaStream_t s) {
  const bool fdr = (p.flags & MS_FLAG_FDR) != 0;
  // Algorithm 1 alone (no fused levels), out of place, or with the Fast Dice Roller draws: the
  // eight-warp kernel
  if (fdr || (p.d == 0 && p.fy_per_cta > 0 && (kPerm || in != out))) {
    const uint2 key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    uint32_t P = p.leaf_max + 2u;  // (a base block has at most leaf_max elements)
    while (P % 64u != 2u) ++P;
    constexpr uint32_t kBudget = 132u * 1024u;  // index and draw regions (two of P entries a lane)
    const uint32_t lanes = std::max<uint32_t>(1u, std::min<uint32_t>(32u, kBudget / (4u * P)));
    if (!kPerm && in == out) {
      // (FDR draws) in place: one thread per base block copies nothing and swaps in the array
      const uint64_t grid = std::min<uint64_t>((p.q + 127u) / 128u, 1048576ull);
      if (p.prof) p.prof->begin(kKindLeaf, s);
      fy_fdr_kernel<E, kPerm><<<static_cast<unsigned>(grid), 128, 0, s>>>(
          static_cast<const E *>(in), static_cast<E *>(out), p.n, p.c, key);
      if (p.prof) p.prof->end(s);
      return cudaGetLastError();
    }
    const size_t smem = (2u * static_cast<size_t>(lanes) * P + kFdrThreads * kFdrFail) * 2u;
    auto fk = fdr ? fy8_kernel<E, kPerm, true> : fy8_kernel<E, kPerm, false>;
    cudaError_t e = allow_dynamic_smem(fk, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fk, kFdrThreads, smem) !=
            cudaSuccess)
      return cudaErrorUnknown;
    const uint64_t batches = (p.q + lanes - 1u) / lanes;
    const uint64_t grid = std::min<uint64_t>(batches, static_cast<uint64_t>(std::max(per_sm, 1)) * sms);
    if (p.prof) p.prof->begin(kKindLeaf, s);
    fk<<<static_cast<unsigned>(grid), kFdrThreads, smem, s>>>(
        static_cast<const E *>(in), static_cast<E *>(out), p.n, p.c, key, P, lanes);
    if (p.prof) p.prof->end(s);
    return cudaGetLastError();
  }
  LeafArgs a;
  a.in = in;
  a.out = out;
  a.n = p.n;
  a.q = p.q;
  a.key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  a.c = p.c;
  a.d = p.d;
  a.dw = p.dw;
  a.tile_max = p.tile_max;
  a.stride = p.leaf_stride;
  a.buf0 = p.buf0_elems;
  a.ucap_w = p.ucap_w;
  a.tcap_w = p.tcap_w;
  a.ucap_c = p.ucap_c;
  a.tcap_c = p.tcap_c;
  a.aux_w = p.aux_w;
  if (p.d == 0 && p.fy_per_cta > 0 && !kPerm && sizeof(E) >= 8 && p.leaf_max <= kIdxMaxLeaf) {
    auto fk = fy_index_kernel<E>;
    const uint32_t per = 32;
    const size_t smem = static_cast<size_t>(per) * p.leaf_stride * sizeof(uint32_t);
    cudaError_t e2 = allow_dynamic_smem(fk, smem);
    if (e2 != cudaSuccess) return e2;
    const uint64_t groups = (p.q + per - 1) / per;
    const uint64_t grid = groups < 1048576ull ? groups : 1048576ull;
    if (p.prof) p.prof->begin(kKindLeaf, s);
    fk<<<static_cast<unsigned>(grid), 32, smem, s>>>(a, per);
    if (p.prof) p.prof->end(s);
    return cudaGetLastError();
  }
  if (p.d == 0 && p.fy_per_cta > 0) {
    auto fk = fy_kernel<E, kPerm>;
    const size_t smem = static_cast<size_t>(p.fy_per_cta) * p.leaf_stride * sizeof(E);
    cudaError_t e2 = allow_dynamic_smem(fk, smem);
    if (e2 != cudaSuccess) return e2;
    const uint64_t groups = (p.q + p.fy_per_cta - 1) / p.fy_per_cta;
    const uint64_t grid = groups < 1048576ull ? groups : 1048576ull;
    if (p.prof) p.prof->begin(kKindLeaf, s);
    fk<<<static_cast<unsigned>(grid), 32, smem, s>>>(a, p.fy_per_cta);
    if (p.prof) p.prof->end(s);
    return cudaGetLastError();
  }
  auto kern = leaf_kernel<E, kPerm>;
  cudaError_t err = allow_dynamic_smem(kern, p.leaf_smem);
  if (err != cudaSuccess) return err;
  const uint64_t grid = p.tiles < 1048576ull ? p.tiles : 1048576ull;
  if (p.prof) p.prof->begin(kKindLeaf, s);
  kern<<<static_cast<unsigned>(grid), kLeafThreads, p.leaf_smem, s>>>(a);
  if (p.prof) p.prof->end(s);
  return cudaGetLastError();
}

// One HBM merge level whose merges are small enough to finish inside one CTA: each CTA takes
// 2^m consecutive merges (2^(m+l+1) base blocks), reads both halves of each straight from global
// memory into a shared-memory staging copy of the merged output (same merge routine as the
// tile phase), applies the merge tails there, and stores the span coalesced. No plan kernels,
// hash tables or patches are needed for such levels.
template <typename E>
__global__ void __launch_bounds__(kLeafThreads, 2) local_level_kernel(LeafArgs a, uint32_t lam,
                                                                      uint32_t m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t scan_scratch[33];
  __shared__ uint32_t merges[8][kGroupMerges];
  E *const stage = reinterpret_cast<E *>(smem_raw);
  GroupSmem S;
  S.cw = reinterpret_cast<uint32_t *>(align16(stage + a.tile_max));
  S.zp = S.cw + a.ucap_c;
  S.mv = reinterpret_cast<uint16_t *>(S.zp + a.ucap_c);
  S.ucap = a.ucap_c;
  S.tcap = a.tcap_c;
  S.m_a = merges[0]; S.m_b = merges[1]; S.m_s = merges[2]; S.m_n1 = merges[3];
  S.m_N = merges[4]; S.m_T = merges[5]; S.m_off = merges[6]; S.m_lb = merges[7];
  S.scratch = scan_scratch;
  const E *in = static_cast<const E *>(a.in);
  E *out = static_cast<E *>(a.out);
  const uint32_t gl = m + lam + 1u;  // base blocks per span: 2^gl
  const uint64_t spans = a.q >> gl;
  for (uint64_t sp = blockIdx.x; sp < spans; sp += gridDim.x) {
    const uint64_t lb = sp << gl;
    const uint64_t g0 = boundary(a.n, a.c, lb);
    const uint32_t len = static_cast<uint32_t>(boundary(a.n, a.c, lb + (1ull << gl)) - g0);
    // X is global here: the tails run in shared memory, in order (no patch scratch)
    merge_level<kLeafWarps, E>(a, S, lb, lb, g0, lam, gl, in + g0, len, false, stage, nullptr,
                               0u);
    for (uint32_t i = threadIdx.x; i < len; i += kLeafThreads) out[g0 + i] = stage[i];
    __syncthreads();
  }
}

template <typename E>
cudaError_t launch_local_t(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                           uint64_t seed, cudaStream_t s) {
  LeafArgs a;
  a.in = in;
  a.out = out;
  a.n = p.n;
  a.q = p.q;
  a.key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  a.c = p.c;
  a.d = 0;
  a.dw = 0;
  a.tile_max = lv.span_max;
  a.stride = 1;
  a.buf0 = 0;
  a.ucap_w = 0;
  a.tcap_w = 0;
  a.ucap_c = lv.ucap;
  a.tcap_c = lv.tcap;
  a.aux_w = lv.warp_bytes;
  auto kern = local_level_kernel<E>;
  cudaError_t err = allow_dynamic_smem(kern, lv.smem);
  if (err != cudaSuccess) return err;
  const uint64_t spans = p.q >> (lv.mlog + lv.level + 1u);
  const uint64_t grid = spans < 1048576ull ? spans : 1048576ull;
  if (p.prof) p.prof->begin(kKindLocal, s);
  kern<<<static_cast<unsigned>(grid), kLeafThreads, lv.smem, s>>>(a, lv.level, lv.mlog);
  if (p.prof) p.prof->end(s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_local_level(const Plan &p, const LevelPlan &lv, const void *in, void *out,
                               uint64_t seed, cudaStream_t s) {
  switch (p.w) {
    case 4: return launch_local_t<uint32_t>(p, lv, in, out, seed, s);
    case 8: return launch_local_t<uint2>(p, lv, in, out, seed, s);
    case 16: return launch_local_t<uint4>(p, lv, in, out, seed, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_leaf(const Plan &p, const void *in, void *out, bool perm, uint64_t seed,
                        cudaStream_t s) {
  if (p.tile_mode) return launch_tile(p, in, out, perm, seed, s);
  if (perm) return launch_leaf_t<uint32_t, true>(p, in, out, seed, s);
  switch (p.w) {
    case 4: return launch_leaf_t<uint32_t, false>(p, in, out, seed, s);
    case 8: return launch_leaf_t<uint2, false>(p, in, out, seed, s);
    case 16: return launch_leaf_t<uint4, false>(p, in, out, seed, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace msk
