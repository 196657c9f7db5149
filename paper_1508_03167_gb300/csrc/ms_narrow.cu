// ms_narrow.cu -- 1- and 2-byte elements (arXiv 1508.03167's problem statement: permute an array
// of n elements of a given width). A shuffle is its input gathered through the permutation that
// ms_perm returns for the same (n, seed, B): the result does not depend on the width. So the
// narrow widths build that permutation with the 4-byte path, then gather the elements through
// it into a scratch buffer and copy them back.
#include "mergeshuffle.h"
#include "ms_common.cuh"
#include "ms_plan.h"

namespace msk {
namespace {

constexpr uint32_t kNarrowThreads = 256;

// tmp[i] = data[idx[i]] for i < n, four positions a thread (one 16-byte load of indices, four
// element loads in flight, one packed store); then the positions of the last partial quad.
template <typename E, typename P>
__global__ void __launch_bounds__(kNarrowThreads) narrow_gather_kernel(const E *data,
                                                                      const uint32_t *idx,
                                                                      E *tmp, uint64_t n) {
  static_assert(sizeof(P) == 4 * sizeof(E), "a packed quad");
  const uint64_t quads = n / 4u;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kNarrowThreads;
  for (uint64_t q = static_cast<uint64_t>(blockIdx.x) * kNarrowThreads + threadIdx.x; q < quads;
       q += stride) {
    const uint4 j = reinterpret_cast<const uint4 *>(idx)[q];
    const E v0 = data[min(static_cast<uint64_t>(j.x), n - 1u)];
    const E v1 = data[min(static_cast<uint64_t>(j.y), n - 1u)];
    const E v2 = data[min(static_cast<uint64_t>(j.z), n - 1u)];
    const E v3 = data[min(static_cast<uint64_t>(j.w), n - 1u)];
    constexpr uint32_t kBits = 8u * sizeof(E);
    const P packed = static_cast<P>(v0) | (static_cast<P>(v1) << kBits) |
                     (static_cast<P>(v2) << (2u * kBits)) | (static_cast<P>(v3) << (3u * kBits));
    reinterpret_cast<P *>(tmp)[q] = packed;
  }
  if (blockIdx.x == 0 && threadIdx.x < n - 4u * quads) {
    const uint64_t i = 4u * quads + threadIdx.x;
    tmp[i] = data[min(static_cast<uint64_t>(idx[i]), n - 1u)];
  }
}

}  // namespace

cudaError_t launch_narrow_gather(const void *data, const uint32_t *idx, void *tmp, uint64_t n,
                                 uint32_t w, int sms, cudaStream_t s) {
  const uint64_t quads = n / 4u;
  uint64_t grid = (quads + kNarrowThreads - 1u) / kNarrowThreads;
  const uint64_t cap = static_cast<uint64_t>(sms > 0 ? sms : 1) * 8u;
  if (grid > cap) grid = cap;
  if (grid < 1u) grid = 1u;
  if (w == 1) {
    narrow_gather_kernel<uint8_t, uint32_t><<<static_cast<unsigned>(grid), kNarrowThreads, 0, s>>>(
        static_cast<const uint8_t *>(data), idx, static_cast<uint8_t *>(tmp), n);
  } else if (w == 2) {
    narrow_gather_kernel<uint16_t, unsigned long long>
        <<<static_cast<unsigned>(grid), kNarrowThreads, 0, s>>>(
            static_cast<const uint16_t *>(data), idx, static_cast<uint16_t *>(tmp), n);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace msk
