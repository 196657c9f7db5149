// ms_bits.cu -- random-bit accounting of one MergeShuffle run (the random-bit model of
// Section 1 of arXiv 1508.03167; the count the paper's Table 1 reports): coin bits (T + 1 per
// merge, the terminating coin included), and for every uniform draw its tested slices times
// their width b = ceil(log2 R), for Algorithm 1's draws and for the merge tails -- or, with
// MS_FLAG_FDR, the bits the Fast Dice Roller reads from the draw's stream. The counts are a
// pure function of (n, seed, B): no data is permuted.
#include <algorithm>

#include "mergeshuffle.h"
#include "ms_merge.cuh"

namespace msk {
namespace {

constexpr int kBitThreads = 256;

// Slices tested by the rejection draw in [0, R) of stream (tag, level, id, pos): the same
// slices in the same order as the draw itself (word 0 given).
__device__ uint32_t draw_attempts(uint2 key, uint32_t tag, uint32_t level, uint32_t id,
                                  uint32_t pos, uint32_t R, uint32_t word0) {
  if (R <= 1u) return 0u;
  const uint32_t b = 32u - __clz(R - 1u);
  const uint32_t per = 32u / b;
  const uint32_t mask = (b == 32u) ? 0xFFFFFFFFu : ((1u << b) - 1u);
  uint32_t tried = 0, word = word0;
  for (uint32_t j = 0; j < (1u << 20); ++j) {
    if (j) word = pick_word(philox10(make_uint4(pos >> 2, id, (tag << 16) | level, j), key), pos & 3u);
    for (uint32_t u = 0; u < per; ++u) {
      ++tried;
      if (((word >> (u * b)) & mask) < R) return tried;
    }
  }
  return tried;
}

__device__ __forceinline__ void add_warp(unsigned long long *dst, unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFullMask, v, off);
  if ((threadIdx.x & 31u) == 0u && v) atomicAdd(dst, v);
}

// Algorithm 1's draws: one thread per (base block, quad of positions). out[1] += bits,
// out[3] += draws.
__global__ void __launch_bounds__(kBitThreads) leaf_bits_kernel(uint64_t n, uint32_t c, uint2 key,
                                                               uint32_t nq, bool fdr,
                                                               unsigned long long *out) {
  const uint64_t q = 1ull << c;
  unsigned long long bits = 0, draws = 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kBitThreads;
  for (uint64_t x = static_cast<uint64_t>(blockIdx.x) * kBitThreads + threadIdx.x; x < q * nq;
       x += stride) {
    const uint64_t k = x / nq;
    const uint32_t qd = static_cast<uint32_t>(x - k * nq);
    const uint32_t L = static_cast<uint32_t>(boundary(n, c, k + 1) - boundary(n, c, k));
    if (4u * qd >= L) continue;
    const uint4 blk = philox10(make_uint4(qd, static_cast<uint32_t>(k), kTagLeaf << 16, 0u), key);
#pragma unroll
    for (uint32_t v = 0; v < 4u; ++v) {
      const uint32_t pos = 4u * qd + v;
      if (pos >= 1u && pos < L) {
        const uint32_t R = pos + 1u;
        if (fdr) {
          uint32_t nb;
          draw_fdr(key, kTagLeaf, 0u, static_cast<uint32_t>(k), pos, R, &nb);
          bits += nb;
        } else {
          bits += static_cast<unsigned long long>(
                      draw_attempts(key, kTagLeaf, 0u, static_cast<uint32_t>(k), pos, R,
                                    pick_word(blk, v))) * (32u - __clz(R - 1u));
        }
        ++draws;
      }
    }
  }
  add_warp(out + 1, bits);
  add_warp(out + 3, draws);
}

// One level's merges, a warp per merge: out[0] += T + 1 coins, out[2] += tail bits, out[4] +=
// tail draws (positions T .. N-1), out[5] += merges.
__global__ void __launch_bounds__(kBitThreads) tail_bits_kernel(uint64_t n, uint32_t c,
                                                               uint32_t level, uint32_t M,
                                                               const uint4 *minfo, uint2 key,
                                                               bool fdr,
                                                               unsigned long long *out) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (kBitThreads / 32);
  unsigned long long coins = 0, bits = 0, draws = 0, merges = 0;
  for (uint64_t r = (static_cast<uint64_t>(blockIdx.x) * kBitThreads + threadIdx.x) >> 5; r < M;
       r += warps) {
    const uint64_t L0 = r << (level + 1u);
    const uint32_t N = static_cast<uint32_t>(boundary(n, c, L0 + (2ull << level)) -
                                             boundary(n, c, L0));
    const uint32_t T = min(minfo[r].x, N);
    if (lane == 0u) {
      coins += T + 1u;
      ++merges;
    }
    for (uint32_t i = T + lane; i < N; i += 32u) {
      const uint32_t R = i + 1u;
      if (fdr) {
        uint32_t nb;
        draw_fdr(key, kTagTail, level, static_cast<uint32_t>(r), i, R, &nb);
        bits += nb;
      } else {
        const uint4 blk = philox10(make_uint4(i >> 2, static_cast<uint32_t>(r), (kTagTail << 16) | level, 0u), key);
        bits += static_cast<unsigned long long>(
                    draw_attempts(key, kTagTail, level, static_cast<uint32_t>(r), i, R,
                                  pick_word(blk, i & 3u))) * (32u - __clz(R - 1u));
      }
      ++draws;
    }
  }
  add_warp(out + 0, coins);
  add_warp(out + 2, bits);
  add_warp(out + 4, draws);
  add_warp(out + 5, merges);
}

size_t r256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace msk

extern "C" {

size_t ms_random_bits_workspace(uint64_t n, const ms_params *params) {
  ms_params r;
  ms_default_params(&r);
  if (params) r = *params;
  if (ms_resolve_params(n, 4, &r) != MS_OK) return 0;
  if (r.B == 0 || n > 0xFFFFFFFFull) return 0;
  uint32_t c = 0;
  while ((n >> c) > r.B) ++c;
  size_t most = 0;
  for (uint32_t l = 0; l < c; ++l) {
    const uint64_t M = (1ull << c) >> (l + 1);
    const uint64_t Nmax = ((n << (l + 1)) + (1ull << c) - 1) >> c;
    const uint64_t J = (Nmax + msk::kChunk - 1) / msk::kChunk;
    most = std::max(most, msk::r256(M * J * 4) + msk::r256(M * 16));
  }
  return 256 + most;
}

ms_status ms_random_bits(uint64_t n, uint64_t seed, const ms_params *params, void *d_ws,
                         size_t ws_bytes, uint64_t *h_out, ms_stream_t stream) {
  if (!h_out) return MS_ERR_INVALID;
  for (int i = 0; i < 8; ++i) h_out[i] = 0;
  const size_t need = ms_random_bits_workspace(n, params);
  if (need == 0) return MS_ERR_INVALID;
  if (n <= 1) return MS_OK;
  if (!d_ws || ws_bytes < need || reinterpret_cast<uintptr_t>(d_ws) % 256 != 0)
    return MS_ERR_INVALID;
  ms_params r;
  ms_default_params(&r);
  if (params) r = *params;
  if (ms_resolve_params(n, 4, &r) != MS_OK) return MS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t c = 0;
  while ((n >> c) > r.B) ++c;
  const uint2 key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  char *base = static_cast<char *>(d_ws);
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(base);
  if (cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s) != cudaSuccess) return MS_ERR_CUDA;
  const uint32_t lmax = static_cast<uint32_t>((n + (1ull << c) - 1) >> c);
  const uint32_t nq = (lmax + 3u) / 4u;
  const bool fdr = (r.flags & MS_FLAG_FDR) != 0;
  msk::leaf_bits_kernel<<<152u * 8u, msk::kBitThreads, 0, s>>>(n, c, key, nq, fdr, cnt);
  if (cudaGetLastError() != cudaSuccess) return MS_ERR_CUDA;
  msk::Plan p;
  p.n = n;
  p.w = 4;
  p.B = r.B;
  p.c = c;
  p.q = 1ull << c;
  p.flags = 0;
  for (uint32_t l = 0; l < c; ++l) {
    msk::LevelPlan lv{};
    lv.level = l;
    lv.M = static_cast<uint32_t>(p.q >> (l + 1));
    lv.Nmax = static_cast<uint32_t>(((n << (l + 1)) + p.q - 1) >> c);
    lv.J = (lv.Nmax + msk::kChunk - 1) / msk::kChunk;
    msk::Buffers b{};
    b.zc = reinterpret_cast<uint32_t *>(base + 256);
    b.minfo = reinterpret_cast<uint4 *>(base + 256 +
                                        msk::r256(static_cast<size_t>(lv.M) * lv.J * 4));
    if (msk::launch_level_breaks(p, lv, b, seed, s) != cudaSuccess) return MS_ERR_CUDA;
    const uint64_t grid = std::min<uint64_t>((lv.M + 7) / 8, 152u * 16u);
    msk::tail_bits_kernel<<<static_cast<unsigned>(grid), msk::kBitThreads, 0, s>>>(
        n, c, l, lv.M, b.minfo, key, fdr, cnt);
    if (cudaGetLastError() != cudaSuccess) return MS_ERR_CUDA;
  }
  unsigned long long host[8];
  if (cudaMemcpyAsync(host, cnt, sizeof host, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MS_ERR_CUDA;
  for (int i = 0; i < 6; ++i) h_out[i] = host[i];
  h_out[6] = host[4];  // leftover = tail draws (every tail position draws, T >= 1)
  h_out[7] = c;
  return MS_OK;
}

}  // extern "C"
