// ms_leaf.cu -- the base-block kernel: one CTA per tile of 2^d consecutive base blocks.
//
// A tile is loaded into shared memory (or generated as the identity for perm), every base block
// is shuffled by Fisher-Yates (Algorithm 1 of arXiv 1508.03167, descending form), and merge
// levels 0..d-1 of Algorithm 3 run inside shared memory with the stable random merge (Algorithm 2:
// coin interleave until one half is exhausted, leftovers in order, then random insertion).
// The tile is written back once, so this kernel is the first of the 1 + (c - d) HBM passes.
#include "ms_common.cuh"
#include "ms_device.cuh"
#include "ms_plan.h"

namespace msk {
namespace {

constexpr int kLeafThreads = 256;
constexpr int kLeafWarps = kLeafThreads / 32;

struct LeafArgs {
  const void *in;
  void *out;
  uint64_t n;
  uint64_t q;
  uint2 key;
  uint32_t c;
  uint32_t d;
  uint32_t tile_max;
  uint32_t unit_cap;
};

template <typename E>
__device__ __forceinline__ void swap_smem(E *a, uint32_t i, uint32_t j) {
  const E t = a[i];
  a[i] = a[j];
  a[j] = t;
}

// One merge level inside the tile: X holds 2^(d-lam) shuffled blocks of 2^lam base blocks each,
// Y receives 2^(d-lam-1) merged blocks.
template <typename E>
__device__ void tile_merge_level(const LeafArgs &a, uint64_t leaf0, uint64_t g0, uint32_t lam,
                                 const E *__restrict__ X, E *__restrict__ Y, uint32_t *cw,
                                 uint32_t *zw, uint32_t *m_s, uint32_t *m_n1, uint32_t *m_N,
                                 uint32_t *m_T, uint32_t *m_ZT, uint32_t *scan_scratch) {
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint32_t warp = tid >> 5;
  const uint32_t Mt = 1u << (a.d - lam - 1u);
  const uint64_t rbase = leaf0 >> (lam + 1u);  // global id of the tile's first merge
  const uint32_t Nmax = static_cast<uint32_t>(((a.n << (lam + 1u)) + a.q - 1u) >> a.c);
  const uint32_t Wm = (Nmax + 31u) >> 5;   // coin words per merge
  const uint32_t BPM = (Nmax + 127u) >> 7; // Philox blocks per merge
  const uint32_t U = Mt * Wm;

  // merge bounds (tile-relative)
  for (uint32_t r = tid; r < Mt; r += kLeafThreads) {
    const uint64_t L0 = leaf0 + (static_cast<uint64_t>(r) << (lam + 1u));
    const uint64_t s = boundary(a.n, a.c, L0);
    const uint64_t mid = boundary(a.n, a.c, L0 + (1ull << lam));
    const uint64_t e = boundary(a.n, a.c, L0 + (2ull << lam));
    m_s[r] = static_cast<uint32_t>(s - g0);
    m_n1[r] = static_cast<uint32_t>(mid - s);
    m_N[r] = static_cast<uint32_t>(e - s);
    m_T[r] = static_cast<uint32_t>(e - s);
  }
  // coin words
  for (uint32_t idx = tid; idx < Mt * BPM; idx += kLeafThreads) {
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

  // zero counts per word, exclusive prefix over the whole tile level
  {
    const uint32_t per = (U + kLeafThreads - 1u) / kLeafThreads;
    const uint32_t u0 = min(tid * per, U);
    const uint32_t u1 = min(u0 + per, U);
    uint32_t local = 0;
    for (uint32_t u = u0; u < u1; ++u) {
      const uint32_t r = u / Wm;
      const uint32_t j = u - r * Wm;
      const uint32_t N = m_N[r];
      const uint32_t valid = (32u * j >= N) ? 0u : min(32u, N - 32u * j);
      const uint32_t z = __popc(~cw[u] & low_mask(valid));
      zw[u] = z;
      local += z;
    }
    uint32_t total;
    uint32_t excl = block_exclusive_scan(local, scan_scratch, &total);
    for (uint32_t u = u0; u < u1; ++u) {
      const uint32_t z = zw[u];
      zw[u] = excl;
      excl += z;
    }
  }
  __syncthreads();

  // break step T of each merge: the (n1+1)-th zero or the (n2+1)-th one, whichever is first
  for (uint32_t u = tid; u < U; u += kLeafThreads) {
    const uint32_t r = u / Wm;
    const uint32_t j = u - r * Wm;
    const uint32_t N = m_N[r];
    if (32u * j >= N) continue;
    const uint32_t valid = min(32u, N - 32u * j);
    const uint32_t vm = low_mask(valid);
    const uint32_t word = cw[u];
    const uint32_t Zs = zw[u] - zw[r * Wm];
    const uint32_t Os = 32u * j - Zs;
    const uint32_t zeros = __popc(~word & vm);
    const uint32_t ones = valid - zeros;
    const uint32_t n1 = m_n1[r];
    const uint32_t n2 = N - n1;
    if (Zs <= n1 && n1 < Zs + zeros) atomicMin(&m_T[r], 32u * j + select_set_bit(~word & vm, n1 - Zs));
    if (Os <= n2 && n2 < Os + ones) atomicMin(&m_T[r], 32u * j + select_set_bit(word & vm, n2 - Os));
  }
  __syncthreads();
  for (uint32_t r = tid; r < Mt; r += kLeafThreads) {
    const uint32_t T = m_T[r], N = m_N[r], n1 = m_n1[r];
    uint32_t ZT = n1;
    if (T < N) {
      const uint32_t bit = (cw[r * Wm + (T >> 5)] >> (T & 31u)) & 1u;
      ZT = bit ? T - (N - n1) : n1;
    }
    m_ZT[r] = ZT;
  }
  __syncthreads();

  // stable interleave and leftover copy: lane L of a warp places step 32j + L
  for (uint32_t u = warp; u < U; u += kLeafWarps) {
    const uint32_t r = u / Wm;
    const uint32_t j = u - r * Wm;
    const uint32_t N = m_N[r];
    const uint32_t t = 32u * j + lane;
    if (t >= N) continue;
    const uint32_t s = m_s[r], n1 = m_n1[r], T = m_T[r];
    uint32_t src;
    if (t < T) {
      const uint32_t word = cw[u];
      const uint32_t Z = zw[u] - zw[r * Wm] + __popc(~word & low_mask(lane));
      src = ((word >> lane) & 1u) ? s + n1 + (t - Z) : s + Z;
    } else if (m_ZT[r] == n1) {  // first half exhausted: second half's remainder
      src = s + n1 + (t - n1);
    } else {                     // second half exhausted: first half's remainder
      src = s + (t - (N - n1));
    }
    Y[s + t] = X[min(src, s + N - 1u)];  // clamp: stays inside the merge's range
  }
  __syncthreads();

  // random insertion of positions T..N-1 (sequential per merge; draws computed 32 at a time)
  for (uint32_t r = warp; r < Mt; r += kLeafWarps) {
    const uint32_t T = m_T[r], N = m_N[r], s = m_s[r];
    const uint32_t id = static_cast<uint32_t>(rbase + r);
    for (uint32_t base = T; base < N; base += 32u) {
      const uint32_t i = base + lane;
      const uint32_t m = (i < N) ? draw_uniform(a.key, kTagTail, lam, id, i, i + 1u) : 0u;
      const uint32_t cnt = min(32u, N - base);
      for (uint32_t k = 0; k < cnt; ++k) {
        const uint32_t mk = __shfl_sync(kFullMask, m, k);
        if (lane == 0) swap_smem(Y, s + base + k, s + mk);
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

template <typename E, bool kPerm>
__global__ void __launch_bounds__(kLeafThreads) leaf_kernel(LeafArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t scan_scratch[33];
  __shared__ uint32_t m_s[kMaxTileMerges], m_n1[kMaxTileMerges], m_N[kMaxTileMerges],
      m_T[kMaxTileMerges], m_ZT[kMaxTileMerges];

  E *X = reinterpret_cast<E *>(smem_raw);
  E *Y = X + a.tile_max;
  uint32_t *cw = reinterpret_cast<uint32_t *>(Y + (a.d > 0 ? a.tile_max : 0u));
  uint32_t *zw = cw + a.unit_cap;

  const E *in = static_cast<const E *>(a.in);
  E *out = static_cast<E *>(a.out);
  const uint64_t tiles = a.q >> a.d;

  for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint64_t leaf0 = tile << a.d;
    const uint64_t g0 = boundary(a.n, a.c, leaf0);
    const uint64_t g1 = boundary(a.n, a.c, leaf0 + (1ull << a.d));
    const uint32_t len = static_cast<uint32_t>(g1 - g0);

    for (uint32_t i = threadIdx.x; i < len; i += kLeafThreads) {
      if constexpr (kPerm) {
        X[i] = static_cast<E>(g0 + i);
      } else {
        X[i] = in[g0 + i];
      }
    }
    __syncthreads();

    // Algorithm 1 on every base block of the tile (one thread per block)
    for (uint32_t k = threadIdx.x; k < (1u << a.d); k += kLeafThreads) {
      const uint64_t leaf = leaf0 + k;
      const uint32_t bs = static_cast<uint32_t>(boundary(a.n, a.c, leaf) - g0);
      const uint32_t be = static_cast<uint32_t>(boundary(a.n, a.c, leaf + 1u) - g0);
      DrawMemo memo;
      for (uint32_t i = be - bs; i-- > 1u;) {
        const uint32_t j = draw_uniform(a.key, kTagLeaf, 0u, static_cast<uint32_t>(leaf), i,
                                        i + 1u, memo);
        swap_smem(X, bs + i, bs + j);
      }
    }
    __syncthreads();

    for (uint32_t lam = 0; lam < a.d; ++lam) {
      tile_merge_level<E>(a, leaf0, g0, lam, X, Y, cw, zw, m_s, m_n1, m_N, m_T, m_ZT,
                          scan_scratch);
      E *t = X;
      X = Y;
      Y = t;
    }

    for (uint32_t i = threadIdx.x; i < len; i += kLeafThreads) out[g0 + i] = X[i];
    __syncthreads();
    // restore buffer roles for the next tile
    if (a.d & 1u) {
      E *t = X;
      X = Y;
      Y = t;
    }
  }
}

template <typename E, bool kPerm>
cudaError_t launch_leaf_t(const Plan &p, const void *in, void *out, uint64_t seed,
                          cudaStream_t s) {
  LeafArgs a;
  a.in = in;
  a.out = out;
  a.n = p.n;
  a.q = p.q;
  a.key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  a.c = p.c;
  a.d = p.d;
  a.tile_max = p.tile_max;
  a.unit_cap = p.unit_cap;
  auto kern = leaf_kernel<E, kPerm>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(p.leaf_smem));
  if (err != cudaSuccess) return err;
  const uint64_t grid = p.tiles < 1048576ull ? p.tiles : 1048576ull;
  if (p.prof) p.prof->begin(kKindLeaf, s);
  kern<<<static_cast<unsigned>(grid), kLeafThreads, p.leaf_smem, s>>>(a);
  if (p.prof) p.prof->end(s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_leaf(const Plan &p, const void *in, void *out, bool perm, uint64_t seed,
                        cudaStream_t s) {
  if (perm) return launch_leaf_t<uint32_t, true>(p, in, out, seed, s);
  switch (p.w) {
    case 4: return launch_leaf_t<uint32_t, false>(p, in, out, seed, s);
    case 8: return launch_leaf_t<uint2, false>(p, in, out, seed, s);
    case 16: return launch_leaf_t<uint4, false>(p, in, out, seed, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace msk
