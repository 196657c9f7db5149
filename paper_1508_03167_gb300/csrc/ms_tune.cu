// ms_tune.cu -- the autotuner's lookup: which cutoff B (and fusion depth / level mode) a call
// with ms_params.B == 0 runs with. The table maps (element width, single or batched call, size
// bucket) to parameters measured fastest on the GPU by the tuner of the Python package; its
// built-in copy is ms_tune_table.h, written by that tuner. The lookup is a pure function of
// (n, w, table), so a caller who records the resolved B can reproduce the result (B is part of
// the result's definition: the block split of the appendix listing depends on it, through the
// number of levels c = min{c : floor(n / 2^c) <= B} alone).
//
// A row's B is the block size measured best at the tuner's power-of-two sizes. A single call of
// another n runs with the c whose blocks floor(n / 2^c) are nearest to it (by ratio), and
// resolves B to that block size: a row of 512 gives n = 3*10^8 blocks of 572 (c = 19), where
// the cutoff 512 itself would give blocks of 286.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "mergeshuffle.h"
#include "ms_plan.h"

namespace {

const ms_tune_entry kBuiltin[] = {
#include "ms_tune_table.h"
};

std::mutex g_mu;
std::vector<ms_tune_entry> &table() {
  static std::vector<ms_tune_entry> t(std::begin(kBuiltin), std::end(kBuiltin));
  return t;
}

uint32_t ceil_log2(uint64_t n) {
  uint32_t k = 0;
  while (k < 64 && (1ull << k) < n) ++k;
  return k;
}

bool entry_valid(const ms_tune_entry &e) {
  return (e.w == 4 || e.w == 8 || e.w == 16) && e.batch <= 1 && e.B >= 1 && e.B <= MS_MAX_B &&
         e.fuse_depth >= -1 && e.log2n_max <= 64 &&
         (e.flags & ~(MS_FLAG_CTA_LEVELS | MS_FLAG_GLOBAL_LEVELS | MS_FLAG_SINGLE_LEVELS |
                      MS_FLAG_PAIR_LEVELS)) == 0;
}

// First entry (w, batch) with ceil(log2 n) <= log2n_max, else the largest bucket of (w, batch),
// else B = 1024 with the planner's own choices.
ms_tune_entry lookup(uint64_t n, uint32_t w, uint32_t batch) {
  std::lock_guard<std::mutex> g(g_mu);
  const uint32_t lg = ceil_log2(n);
  const ms_tune_entry *best = nullptr;
  const ms_tune_entry *widest = nullptr;
  for (const ms_tune_entry &e : table()) {
    if (e.w != w || e.batch != batch) continue;
    if (lg <= e.log2n_max && (best == nullptr || e.log2n_max < best->log2n_max)) best = &e;
    if (widest == nullptr || e.log2n_max > widest->log2n_max) widest = &e;
  }
  if (best) return *best;
  if (widest) return *widest;
  ms_tune_entry d;
  std::memset(&d, 0, sizeof d);
  d.w = w;
  d.batch = batch;
  d.log2n_max = 64;
  d.B = 1024;
  d.fuse_depth = -1;
  return d;
}

// The cutoff whose blocks are nearest to `target` by ratio: floor(n / 2^c) for the c among the
// two around n / target, so that c is also the listing's smallest c with floor(n / 2^c) <= B.
uint32_t block_for(uint64_t n, uint32_t target) {
  if (n <= target) return target;  // one block (c = 0) either way
  uint32_t c0 = 0;  // n >> c0 >= target > n >> (c0 + 1)
  while ((n >> (c0 + 1)) >= target) ++c0;
  const uint64_t b0 = n >> c0, b1 = n >> (c0 + 1);
  const bool lower = b1 >= 1 && (b0 > MS_MAX_B || b0 * b1 > static_cast<uint64_t>(target) * target);
  return static_cast<uint32_t>(lower ? b1 : b0);
}

void apply(const ms_tune_entry &e, ms_params *p) {
  p->B = e.B;
  if (p->fuse_depth < 0) p->fuse_depth = e.fuse_depth;
  const uint32_t mode = MS_FLAG_CTA_LEVELS | MS_FLAG_GLOBAL_LEVELS | MS_FLAG_SINGLE_LEVELS |
                        MS_FLAG_PAIR_LEVELS;
  if ((p->flags & mode) == 0) p->flags |= e.flags;
}

}  // namespace

namespace msk {

ms_params resolve_single(uint64_t n, uint32_t w, const ms_params *p) {
  ms_params r;
  ms_default_params(&r);
  if (p) r = *p;
  if (r.B == 0) {
    apply(lookup(n, w < 4u ? 4u : w, 0), &r);  // (1- and 2-byte elements run a 4-byte perm)
    r.B = block_for(n, r.B);
  }
  return r;
}

ms_params resolve_batch(uint32_t k, const uint64_t *h_n, uint32_t w, const ms_params *p) {
  ms_params r;
  ms_default_params(&r);
  if (p) r = *p;
  if (r.B == 0) {
    // the batch runs with one B: the bucket of the median instance size
    std::vector<uint64_t> ns;
    ns.reserve(k);
    for (uint32_t i = 0; i < k && h_n; ++i) ns.push_back(h_n[i]);
    uint64_t med = 2;
    if (!ns.empty()) {
      std::nth_element(ns.begin(), ns.begin() + ns.size() / 2, ns.end());
      med = std::max<uint64_t>(ns[ns.size() / 2], 2);
    }
    apply(lookup(med, w, 1), &r);
  }
  return r;
}

}  // namespace msk

extern "C" {

ms_status ms_resolve_params(uint64_t n, uint32_t w, ms_params *inout) {
  if (!inout) return MS_ERR_INVALID;
  if (w != 1 && w != 2 && w != 4 && w != 8 && w != 16) return MS_ERR_INVALID;
  *inout = msk::resolve_single(n, w, inout);
  return MS_OK;
}

ms_status ms_resolve_batch_params(uint32_t k, const uint64_t *h_n, uint32_t w,
                                  ms_params *inout) {
  if (!inout) return MS_ERR_INVALID;
  if (w != 4 && w != 8 && w != 16) return MS_ERR_INVALID;
  if (k > 0 && h_n == nullptr) return MS_ERR_INVALID;
  *inout = msk::resolve_batch(k, h_n, w, inout);
  return MS_OK;
}

ms_status ms_tune_install(const ms_tune_entry *entries, uint32_t count) {
  if (count > 0 && entries == nullptr) return MS_ERR_INVALID;
  for (uint32_t i = 0; i < count; ++i)
    if (!entry_valid(entries[i])) return MS_ERR_INVALID;
  std::lock_guard<std::mutex> g(g_mu);
  if (count == 0)
    table().assign(std::begin(kBuiltin), std::end(kBuiltin));
  else
    table().assign(entries, entries + count);
  return MS_OK;
}

uint32_t ms_tune_table(ms_tune_entry *out, uint32_t cap) {
  std::lock_guard<std::mutex> g(g_mu);
  const uint32_t k = static_cast<uint32_t>(table().size());
  if (out)
    for (uint32_t i = 0; i < k && i < cap; ++i) out[i] = table()[i];
  return k;
}

}  // extern "C"
