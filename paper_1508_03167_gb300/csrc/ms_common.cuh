// ms_common.cuh -- small CTA-wide primitives shared by the MergeShuffle kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace msk {

constexpr unsigned kFullMask = 0xFFFFFFFFu;

// Inclusive warp scan (Hillis-Steele with shuffles).
__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t up = __shfl_up_sync(kFullMask, v, off);
    if (lane >= off) v += up;
  }
  return v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFullMask, v, off);
  return v;
}

// Exclusive scan of one value per thread across the CTA. `scratch` holds >= 33 words of shared
// memory. Returns the exclusive prefix; *total receives the CTA sum. All threads must call it.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *scratch,
                                                         uint32_t *total) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  const uint32_t incl = warp_inclusive_scan(v);
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < nwarps ? scratch[lane] : 0u;
    const uint32_t si = warp_inclusive_scan(s);
    scratch[lane] = si - s;  // exclusive prefix of warp totals
    if (lane == 31) scratch[32] = si;
  }
  __syncthreads();
  const uint32_t excl = scratch[warp] + incl - v;
  *total = scratch[32];
  __syncthreads();
  return excl;
}

// asynchronous global -> shared copy of one element (cp.async, L1-allocating for 4 and 8 bytes,
// L2-only for 16)
template <typename E>
__device__ __forceinline__ void cp_async_elem(E *dst, const E *src) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  if constexpr (sizeof(E) == 4) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
  } else if constexpr (sizeof(E) == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
  } else {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace msk
