// ms_device.cuh -- device-side building blocks of the MergeShuffle path (arXiv 1508.03167):
// the Philox4x32-10 block function, the coin and uniform-draw streams, and the merge-tree
// boundary arithmetic of the appendix listing. Written for sm_103a.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace msk {

// ----------------------------------------------------------------------------- Philox ------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64 products,
// xor of the high halves with the odd counter words and the round key, word permutation;
// the key is bumped by the Weyl increments between rounds.
constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kWeylA = 0x9E3779B9u;
constexpr uint32_t kWeylB = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox10(uint4 ctr, uint2 key) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo_a = kPhiloxMulA * ctr.x;
    const uint32_t hi_a = __umulhi(kPhiloxMulA, ctr.x);
    const uint32_t lo_b = kPhiloxMulB * ctr.z;
    const uint32_t hi_b = __umulhi(kPhiloxMulB, ctr.z);
    ctr = make_uint4(hi_b ^ ctr.y ^ key.x, lo_b, hi_a ^ ctr.w ^ key.y, lo_a);
    key.x += kWeylA;
    key.y += kWeylB;
  }
  return ctr;
}

__device__ __forceinline__ uint32_t pick_word(const uint4 &v, uint32_t k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

__device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

// Stream tags (the third counter word carries tag << 16 | level).
constexpr uint32_t kTagCoin = 1u;
constexpr uint32_t kTagTail = 2u;
constexpr uint32_t kTagLeaf = 3u;

// The 128 coins of steps [128*blk, 128*blk + 128) of merge `id` on `level`: word k holds steps
// 128*blk + 32*k .. +31, least significant bit first. A 0 coin takes from the first half.
__device__ __forceinline__ uint4 coin_block(uint2 key, uint32_t level, uint32_t id,
                                            uint32_t blk) {
  return philox10(make_uint4(blk, id, (kTagCoin << 16) | level, 0u), key);
}

// Uniform integer in [0, R) by rejection on b = ceil(log2 R)-bit slices; floor(32/b) slices
// per 32-bit word, word j of the stream is word pos%4 of Philox((pos/4, id, tag|level, j)).
// `memo` caches word-0 blocks across consecutive positions of one stream (pos/4 equal).
struct DrawMemo {
  uint32_t quad = 0xFFFFFFFFu;
  uint4 blk;
};

__device__ __forceinline__ uint32_t draw_uniform(uint2 key, uint32_t tag, uint32_t level,
                                                 uint32_t id, uint32_t pos, uint32_t R,
                                                 DrawMemo &memo) {
  if (R <= 1u) return 0u;
  const uint32_t b = 32u - __clz(R - 1u);
  // floor(32 / b), exact: see the note in draw_from_word
  const uint32_t slices = static_cast<uint32_t>(__fdividef(32.0f, static_cast<float>(b)));
  const uint32_t mask = (b == 32u) ? 0xFFFFFFFFu : ((1u << b) - 1u);
  const uint32_t c2 = (tag << 16) | level;
  for (uint32_t j = 0; j < (1u << 20); ++j) {
    uint4 blk;
    if (j == 0 && memo.quad == (pos >> 2)) {
      blk = memo.blk;
    } else {
      blk = philox10(make_uint4(pos >> 2, id, c2, j), key);
      if (j == 0) {
        memo.quad = pos >> 2;
        memo.blk = blk;
      }
    }
    const uint32_t word = pick_word(blk, pos & 3u);
    for (uint32_t u = 0; u < slices; ++u) {
      const uint32_t x = (word >> (u * b)) & mask;
      if (x < R) return x;
    }
  }
  return 0u;  // 2^20 rejected words: probability below 2^-(2^20); kept finite on purpose
}

__device__ __forceinline__ uint32_t draw_uniform(uint2 key, uint32_t tag, uint32_t level,
                                                 uint32_t id, uint32_t pos, uint32_t R) {
  DrawMemo memo;
  return draw_uniform(key, tag, level, id, pos, R, memo);
}

// Uniform integer in [0, R) by the Fast Dice Roller (Lumbroso 2013) on the stream's bits: word
// j of the stream (as above) read least significant bit first, j = 0, 1, ...; v doubles and c
// takes the next bit with each read; once v >= R, c < R is the value, else c - R is uniform on
// [0, v - R) and the loop goes on with v - R. *bits receives the bits read (MS_FLAG_FDR).
__device__ __forceinline__ uint32_t draw_fdr(uint2 key, uint32_t tag, uint32_t level, uint32_t id,
                                             uint32_t pos, uint32_t R, uint32_t *bits) {
  *bits = 0u;
  if (R <= 1u) return 0u;
  uint64_t v = 1u, c = 0u;
  const uint32_t c2 = (tag << 16) | level;
  for (uint32_t j = 0; j < (1u << 20); ++j) {
    const uint32_t word = pick_word(philox10(make_uint4(pos >> 2, id, c2, j), key), pos & 3u);
    for (uint32_t u = 0; u < 32u; ++u) {
      v <<= 1;
      c = (c << 1) | ((word >> u) & 1u);
      ++*bits;
      if (v >= R) {
        if (c < R) return static_cast<uint32_t>(c);
        v -= R;
        c -= R;
      }
    }
  }
  return 0u;  // 2^25 bits without a value: probability far below 2^-(2^20); kept finite
}

// ----------------------------------------------------------------------------- merge tree --
// Block boundary floor(n * i / 2^c) (appendix listing; n < 2^32 and i <= 2^c keep the product
// inside 64 bits).
__host__ __device__ __forceinline__ uint64_t boundary(uint64_t n, uint32_t c, uint64_t i) {
  return (n * i) >> c;
}

// Position of the k-th (0-based) set bit of m (m must have more than k set bits).
__device__ __forceinline__ uint32_t select_set_bit(uint32_t m, uint32_t k) {
  for (uint32_t i = 0; i < k; ++i) m &= m - 1u;
  return static_cast<uint32_t>(__ffs(static_cast<int>(m)) - 1);
}

__device__ __forceinline__ uint32_t low_mask(uint32_t bits) {  // bits in [0, 32]
  return bits >= 32u ? 0xFFFFFFFFu : ((1u << bits) - 1u);
}

}  // namespace msk
