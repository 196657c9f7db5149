// ms_static.cu -- ms_perm_static: the perm entry point for callers that cannot allocate device
// memory. Its workspace (the second ping-pong buffer and the merge-level scratch) lives in a
// fixed file-scope __device__ array instead of caller-provided memory.
#include <mutex>

#include "mergeshuffle.h"

namespace {

constexpr size_t kStaticBytes = MS_STATIC_SCRATCH_BYTES;

// Shared by every call on a device; loaded with the library and held until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device. In host code the array's name is
// only a host-side stand-in, so the address is looked up once per device (with that device
// current) and cached.
ms_status scratch_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MS_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_mu);
  if (g_addr[dev] == nullptr) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr)
      return MS_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return MS_OK;
}

}  // namespace

extern "C" ms_status ms_perm_static(uint32_t *d_out, uint64_t n, uint64_t seed,
                                    const ms_params *p, ms_stream_t stream) {
  if (n > MS_STATIC_MAX_N) return MS_ERR_UNSUPPORTED;
  ms_params q;
  ms_default_params(&q);
  if (p) q = *p;
  size_t need = ms_workspace_bytes(n, 4, &q);
  if (need == 0) return MS_ERR_INVALID;
  if (need > kStaticBytes) {
    // one data pass per level needs less plan scratch (the result is the same). At this
    // version's sizes fused pairs fit (16.0 MB at 2^21 with MS_FLAG_PAIR_LEVELS), so only a
    // plan that grows reaches this; the literal, FDR and balanced-word plans do not fit either
    // way at large n and return MS_ERR_UNSUPPORTED below.
    q.flags |= MS_FLAG_SINGLE_LEVELS;
    need = ms_workspace_bytes(n, 4, &q);
  }
  if (need > kStaticBytes) return MS_ERR_UNSUPPORTED;
  if (n <= 1) return ms_perm(d_out, n, seed, nullptr, 0, &q, stream);
  void *ws = nullptr;
  const ms_status st = scratch_address(&ws);
  if (st != MS_OK) return st;
  // Nothing in the scratch has to start at zero: every kernel writes what it later reads, and
  // the merge-level hash table is reset on the stream before each level.
  return ms_perm(d_out, n, seed, ws, kStaticBytes, &q, stream);
}
