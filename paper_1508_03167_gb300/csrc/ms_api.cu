// ms_api.cu -- the C ABI of libmergeshuffle (declared in include/mergeshuffle.h) and the host
// planner: block split and cutoff rule of the appendix listing of arXiv 1508.03167, the choice
// of how many low merge levels run inside shared memory, and the workspace layout.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mergeshuffle.h"
#include "ms_plan.h"

namespace msk {
namespace {

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

uint64_t ceil_scaled(uint64_t n, uint32_t shift, uint32_t c) {
  // ceil(n * 2^shift / 2^c) for shift <= c
  const uint64_t q = 1ull << c;
  return ((n << shift) + q - 1) >> c;
}

// Shared-memory layout of the base-block kernel (one CTA of 8 warps per tile of 2^d base
// blocks): buffer 0 holds the base blocks at an odd stride (conflict-free Fisher-Yates) and
// later a contiguous level; buffer 1 the other level; then the auxiliary arrays (coin words,
// their zero prefixes, precomputed tail draws) of each warp, aliased by the CTA's own.
struct LeafSmem {
  uint32_t d, dw, leaf_max, stride, buf0, tile_max;
  uint32_t ucap_w, tcap_w, ucap_c, tcap_c, aux_w;
  size_t bytes;
};

uint32_t level_units(uint64_t n, uint32_t c, uint32_t gl, uint32_t lam) {
  const uint64_t Mt = 1ull << (gl - lam - 1);
  const uint64_t Nmax = ceil_scaled(n, lam + 1, c);
  return static_cast<uint32_t>(Mt * ((Nmax + 31) / 32));
}

// levels done by single warps: at most 5 (16 merges per warp level) and a warp tile of at most
// 2048 elements
uint32_t warp_levels_max(uint32_t leaf_max) {
  uint32_t dw = 0;
  while (dw < 5 && (static_cast<uint64_t>(leaf_max) << (dw + 1)) <= 2048) ++dw;
  return dw;
}

LeafSmem leaf_smem(uint64_t n, uint32_t c, uint32_t d, uint32_t w) {
  LeafSmem L;
  const uint64_t q = 1ull << c;
  L.d = d;
  L.leaf_max = static_cast<uint32_t>((n + q - 1) >> c);
  L.stride = L.leaf_max | 1u;
  L.dw = std::min(d, warp_levels_max(L.leaf_max));
  const uint64_t tile_max = ceil_scaled(n, d, c);
  L.tile_max = static_cast<uint32_t>(tile_max);
  const uint64_t padded = (1ull << d) * L.stride;
  L.buf0 = static_cast<uint32_t>(std::max<uint64_t>(padded, tile_max));
  // coin-word capacities in multiples of four words: the arrays start 16-byte aligned
  L.ucap_w = 4;
  for (uint32_t lam = 0; lam < L.dw; ++lam)
    L.ucap_w = std::max(L.ucap_w, (level_units(n, c, L.dw, lam) + 3u) & ~3u);
  L.ucap_c = 4;
  for (uint32_t lam = L.dw; lam < d; ++lam)
    L.ucap_c = std::max(L.ucap_c, (level_units(n, c, d, lam) + 3u) & ~3u);
  const uint64_t wtile = ceil_scaled(n, L.dw, c);
  L.tcap_w = static_cast<uint32_t>((wtile / 4 + 16) & ~1ull);
  L.tcap_c = static_cast<uint32_t>((tile_max / 4 + 16) & ~1ull);
  L.aux_w = static_cast<uint32_t>(round_up(2ull * L.ucap_w * 4 + 2ull * L.tcap_w, 16));
  const size_t aux_c = round_up(2ull * L.ucap_c * 4 + 2ull * L.tcap_c, 16);
  const size_t aux = std::max<size_t>(8ull * L.aux_w, aux_c);
  L.bytes = round_up(static_cast<size_t>(L.buf0) * w + tile_max * w, 16) + round_up(aux, 16);
  return L;
}

bool leaf_fits(uint64_t n, uint32_t c, uint32_t d, uint32_t w) {
  const LeafSmem L = leaf_smem(n, c, d, w);
  return L.bytes <= kSmemLimit && L.tile_max < 65536 && d - L.dw <= 3;
}

// Shared-memory layout of the tile kernel (16-bit tile-local indices, eight warps a tile): two
// buffers (the first holds block k at k*P, P = 2 mod 64 and at least the largest block; merge r
// of level l writes at r*S[l]), then one level's (coin word, zero prefix) pairs and two sets of
// a level's tail draws (which also hold the per-thread queues of second-word Fisher-Yates
// draws: 256 threads x 4 entries x 4 bytes over both sets).
struct TileSmem {
  bool ok = false;
  uint32_t P = 0, buf = 0, wcap = 0, tcap = 0;
  uint32_t S[kTileMaxDepth] = {};
  size_t bytes = 0;
};

TileSmem tile_smem(uint64_t n, uint32_t c, uint32_t d) {
  TileSmem T;
  if (d == 0 || d > kTileMaxDepth || d > c) return T;
  const uint64_t tile_max = ceil_scaled(n, d, c);
  if (tile_max >= 65536) return T;
  const uint32_t lmax = static_cast<uint32_t>(ceil_scaled(n, 0, c));
  uint32_t P = lmax;
  while (P % 64u != 2u) ++P;
  uint64_t buf = (1ull << d) * P;
  uint64_t wcap = 4, tcap = 1024;  // (two sets of tail draws hold the 4 KiB of queues)
  for (uint32_t l = 0; l < d; ++l) {
    const uint64_t R = 1ull << (d - l - 1);
    const uint64_t Nmax = ceil_scaled(n, l + 1, c);
    const uint64_t S = (Nmax + 7) & ~7ull;
    T.S[l] = static_cast<uint32_t>(S);
    buf = std::max(buf, R * S);
    wcap = std::max(wcap, R * (Nmax / 32 + 1));
    // tail draws made ahead: the mean sum over the level's merges plus 4.8 spreads
    const double per = std::sqrt(2.0 * static_cast<double>(Nmax) / 3.14159265358979) + 2.0;
    double tc = static_cast<double>(R) * per +
                4.8 * std::sqrt(static_cast<double>(R) * static_cast<double>(Nmax)) + 64.0;
    tc = std::min(tc, static_cast<double>(R * Nmax));
    tcap = std::max<uint64_t>(tcap, static_cast<uint64_t>(tc));
  }
  T.P = P;
  T.buf = static_cast<uint32_t>((buf + 7) & ~7ull);
  T.wcap = static_cast<uint32_t>((wcap + 1) & ~1ull);
  T.tcap = static_cast<uint32_t>((tcap + 7) & ~7ull);
  // two index buffers, one set of (coin word, zero prefix) pairs, two sets of tail draws
  T.bytes = 4ull * T.buf + 8ull * T.wcap + 4ull * T.tcap;
  T.ok = T.bytes <= kSmemLimit;
  return T;
}

}  // namespace

int make_plan(uint64_t n, uint32_t w, uint32_t B, int32_t fuse_depth, uint32_t tile_bytes,
              uint32_t flags, Plan *out) {
  Plan p;
  if (w != 4 && w != 8 && w != 16) return 1;
  if (B == 0) return 1;
  if (n > 0xFFFFFFFFull) return 1;
  if (B > kMaxB) return 2;
  if ((flags & MS_FLAG_LITERAL) && (flags & MS_FLAG_BALANCED)) return 1;
  if (flags & (MS_FLAG_LITERAL | MS_FLAG_FDR | MS_FLAG_BALANCED)) {
    // the literal merge and the FDR draws run on the global levels only: no fused levels, no
    // fused pairs
    fuse_depth = 0;
    flags |= MS_FLAG_GLOBAL_LEVELS | MS_FLAG_SINGLE_LEVELS | MS_FLAG_CTA_TILES;
  }
  p.n = n;
  p.w = w;
  p.B = B;
  p.flags = flags;
  if (tile_bytes == 0) tile_bytes = kDefaultTileBytes;
  uint32_t c = 0;
  while ((n >> c) > B) ++c;
  p.c = c;
  p.q = 1ull << c;
  if (n <= 1) {
    p.ws_bytes = 256;
    *out = p;
    return 0;
  }
  // fusion depth: the deepest d whose tile fits the shared-memory budget
  const uint32_t dmax = c < kMaxFuse ? c : kMaxFuse;
  uint32_t d = 0;
  if (fuse_depth < 0) {
    for (uint32_t t = 0; t <= dmax; ++t)
      if (ceil_scaled(n, t, c) * w <= tile_bytes && leaf_fits(n, c, t, w)) d = t;
  } else {
    d = static_cast<uint32_t>(fuse_depth) < dmax ? static_cast<uint32_t>(fuse_depth) : dmax;
    while (d > 0 && !leaf_fits(n, c, d, w) &&
           ((flags & MS_FLAG_CTA_TILES) || !tile_smem(n, c, d).ok))
      --d;
  }
  p.d = d;
  const TileSmem TS = tile_smem(n, c, d);
  p.tile_mode = TS.ok && !(flags & MS_FLAG_CTA_TILES);
  if (p.tile_mode) {
    p.tile_P = TS.P;
    p.tile_buf = TS.buf;
    p.tile_wcap = TS.wcap;
    p.tile_tcap = TS.tcap;
    for (uint32_t l = 0; l < kTileMaxDepth; ++l) p.tile_S[l] = TS.S[l];
    p.tile_smem = TS.bytes;
  }
  p.tiles = p.q >> d;
  p.tile_max = static_cast<uint32_t>(ceil_scaled(n, d, c));
  const LeafSmem L = leaf_smem(n, c, d, w);
  p.dw = L.dw;
  p.leaf_max = L.leaf_max;
  p.leaf_stride = L.stride;
  p.buf0_elems = L.buf0;
  p.ucap_w = L.ucap_w;
  p.tcap_w = L.tcap_w;
  p.ucap_c = L.ucap_c;
  p.tcap_c = L.tcap_c;
  p.aux_w = L.aux_w;
  p.leaf_smem = L.bytes;
  if (d == 0) {
    // Fisher-Yates only: up to 32 blocks per one-warp CTA within 96 KiB of shared memory
    const uint64_t per_block = static_cast<uint64_t>(L.stride) * w;
    uint64_t per = (96ull * 1024) / per_block;
    if (per > 32) per = 32;
    if (per < 1) per = 1;
    p.fy_per_cta = static_cast<uint32_t>(per);
  }
  if (!p.tile_mode && p.leaf_smem > kSmemLimit) return 2;

  // HBM levels d..c-1
  p.nlevels = c - d;
  uint64_t zc_cap = 0, minfo_cap = 0, kcap_max = 0;
  uint32_t hbits_max = 0;
  for (uint32_t i = 0; i < p.nlevels; ++i) {
    LevelPlan &lv = p.levels[i];
    lv.level = d + i;
    const uint64_t M = p.q >> (lv.level + 1);
    const uint64_t Nmax = ceil_scaled(n, lv.level + 1, c);
    lv.M = static_cast<uint32_t>(M);
    lv.Nmax = static_cast<uint32_t>(Nmax);
    lv.J = static_cast<uint32_t>((Nmax + kChunk - 1) / kChunk);
    // Tail capacity: E[N - T] is about sqrt(2N/pi) per merge and its spread about sqrt(N);
    // the sum over the level's merges is bounded by the mean plus eight spreads.
    const double per = std::ceil(std::sqrt(2.0 * static_cast<double>(Nmax) / 3.14159265358979)) + 2.0;
    double kc = static_cast<double>(M) * per +
                8.0 * std::ceil(std::sqrt(static_cast<double>(M) * static_cast<double>(Nmax))) +
                1024.0;
    const double cap_all = static_cast<double>(M) * static_cast<double>(Nmax);
    if (kc > cap_all) kc = cap_all;
    lv.kcap = static_cast<uint32_t>(kc);
    uint32_t hb = 10;
    while ((1ull << hb) < 2ull * lv.kcap) ++hb;
    lv.hbits = hb;
    // local mode when a merge (and up to 16 of them) fits one CTA's staging buffer
    lv.local = false;
    lv.warp_local = false;
    lv.span = false;
    lv.warp_bytes = 0;
    lv.mlog = 0;
    // span buffers of 8 KiB (128-thread CTAs, eight an SM) when the merges fit, else 16 KiB
    // (256 threads, four an SM), else 32 KiB (two)
    const uint64_t nm = ceil_scaled(n, lv.level + 1, c);
    const uint32_t S = nm <= kSpanBytes / 4 / w   ? kSpanBytes / 4 / w
                       : nm <= kSpanBytes / 2 / w ? kSpanBytes / 2 / w
                                                  : kSpanBytes / w;
    lv.span_threads = S == kSpanBytes / 4 / w ? 128u : 256u;
    const uint32_t mode_flags = MS_FLAG_GLOBAL_LEVELS | MS_FLAG_CTA_LEVELS | MS_FLAG_WARP_LEVELS;
    // (16-byte records: a span holds too few of them to amortise the per-span work; their
    // small levels stream per warp instead)
    if (!(flags & mode_flags) && w <= 8 && ceil_scaled(n, lv.level + 1, c) <= S) {
      // streamed spans of up to 64 merges
      uint32_t m = 0;
      while ((1u << (m + 1)) <= kSpanMaxMerges && (M >> (m + 1)) >= 1 &&
             ceil_scaled(n, lv.level + 2 + m, c) <= S)
        ++m;
      lv.local = true;
      lv.span = true;
      lv.mlog = m;
      lv.span_max = S;
      lv.ucap = (level_units(n, c, lv.level + 1 + m, lv.level) + 3u) & ~3u;
      const double Mt = static_cast<double>(1u << m);
      const double per = std::sqrt(2.0 * static_cast<double>(Nmax) / 3.14159265358979) + 2.0;
      double tc = Mt * per + 4.8 * std::sqrt(Mt * static_cast<double>(Nmax)) + 64.0;
      const double span_el = static_cast<double>(ceil_scaled(n, lv.level + 1 + m, c));
      if (tc > span_el) tc = span_el;
      lv.tcap = static_cast<uint32_t>(tc);
      lv.smem = span_smem_bytes(S, w, lv.ucap, lv.tcap);
      lv.kcap = 0;
      lv.hbits = 10;
    } else if (Nmax <= kWarpMergeMax &&
               !(flags & (MS_FLAG_GLOBAL_LEVELS | MS_FLAG_CTA_LEVELS))) {
      // one warp per span of up to 16 merges (at most kWarpSpanMax elements), global to global
      uint32_t m = 0;
      while (m < kLocalMaxMergesLog && (Nmax << (m + 1)) <= kWarpSpanMax && (M >> (m + 1)) >= 1)
        ++m;
      lv.local = true;
      lv.warp_local = true;
      lv.mlog = m;
      lv.span_max = static_cast<uint32_t>(ceil_scaled(n, lv.level + 1 + m, c));
      lv.ucap = level_units(n, c, lv.level + 1 + m, lv.level);
      const double per = std::sqrt(2.0 * static_cast<double>(Nmax) / 3.14159265358979) + 2.0;
      lv.tcap = static_cast<uint32_t>((4.0 * per * (1u << m) + 64.0)) & ~1u;
      lv.warp_bytes = static_cast<uint32_t>(round_up(2ull * lv.ucap * 4 + 6ull * lv.tcap, 16));
      lv.smem = 0;
      lv.kcap = 0;
      lv.hbits = 10;
    } else if (Nmax * w <= kLocalSpanBytes && !(flags & MS_FLAG_GLOBAL_LEVELS)) {
      uint32_t m = 0;
      while (m < kLocalMaxMergesLog && (Nmax << (m + 1)) * w <= kLocalSpanBytes &&
             (M >> (m + 1)) >= 1)
        ++m;
      lv.local = true;
      lv.mlog = m;
      lv.span_max = static_cast<uint32_t>(ceil_scaled(n, lv.level + 1 + m, c));
      lv.ucap = (level_units(n, c, lv.level + 1 + m, lv.level) + 3u) & ~3u;
      lv.tcap = static_cast<uint32_t>((lv.span_max / 4 + 16) & ~1u);
      lv.smem = round_up(static_cast<size_t>(lv.span_max) * w, 16) +
                round_up(2ull * lv.ucap * 4 + 2ull * lv.tcap, 16);
      lv.kcap = 0;
      lv.hbits = 10;
    }
    if (!lv.local) {
      zc_cap = std::max<uint64_t>(zc_cap, M * lv.J);
      minfo_cap = std::max<uint64_t>(minfo_cap, M);
      kcap_max = std::max<uint64_t>(kcap_max, lv.kcap);
      hbits_max = std::max(hbits_max, lv.hbits);
    }
  }
  p.zc_cap = static_cast<uint32_t>(zc_cap);
  p.minfo_cap = static_cast<uint32_t>(minfo_cap);
  p.kcap_max = static_cast<uint32_t>(kcap_max);
  p.hbits_max = hbits_max;

  // consecutive global levels fuse in pairs (one data pass for two levels)
  uint32_t nlocal = 0, units = 0;
  uint32_t xcap_max = 0;
  for (uint32_t i = 0; i < p.nlevels; ++i) {
    p.levels[i].pair = 0;
    p.levels[i].xcap = 0;
  }
  for (uint32_t i = 0; i < p.nlevels; ++i) {
    LevelPlan &lv = p.levels[i];
    if (lv.local) {
      ++nlocal;
      continue;
    }
    if (lv.pair == 2) continue;  // second level of the pair before it
    ++units;
    // (the fused pass evaluates two interleaves and an exception test per element: worth it
    // where the pass is bound by memory, i.e. for 16-byte elements, or on request)
    const bool want_pairs = !(flags & MS_FLAG_SINGLE_LEVELS) &&
                            (w >= 16 || (flags & MS_FLAG_PAIR_LEVELS));
    if (want_pairs && i + 1 < p.nlevels && !p.levels[i + 1].local) {
      lv.pair = 1;
      p.levels[i + 1].pair = 2;
      lv.xcap = 2u * lv.kcap;
      xcap_max = std::max(xcap_max, lv.xcap);
    }
  }
  // The tile kernel of a shuffle reads its input rows after computing their order, so its
  // pass must not be in place: the passes after it must be odd in number (the last lands in
  // the caller's array). Split the last fused pair; else, on arrays well above L2, fuse the
  // last two global levels into one pass (measured on GB300 at 2^28 and 2^30 4-byte elements:
  // a fused pair costs about a third of what one level fewer in the tile costs); else fuse one
  // level less. (A perm reads nothing.)
  if (p.tile_mode && !(flags & MS_FLAG_PERM) && (nlocal + units) % 2 == 0) {
    int last = -1;
    for (uint32_t i = 0; i < p.nlevels; ++i)
      if (p.levels[i].pair == 1) last = static_cast<int>(i);
    int top = -1;  // first of the last two consecutive global levels
    if (p.nlevels >= 2 && !(flags & MS_FLAG_SINGLE_LEVELS) && n * w >= kPairParityBytes) {
      const uint32_t i = p.nlevels - 2u;
      if (!p.levels[i].local && !p.levels[i + 1].local && p.levels[i].pair == 0 &&
          p.levels[i + 1].pair == 0)
        top = static_cast<int>(i);
    }
    if (last >= 0) {
      p.levels[last].pair = 0;
      p.levels[last].xcap = 0;
      p.levels[last + 1].pair = 0;
      ++units;
      xcap_max = 0;
      for (uint32_t i = 0; i < p.nlevels; ++i) xcap_max = std::max(xcap_max, p.levels[i].xcap);
    } else if (top >= 0) {
      LevelPlan &lv = p.levels[top];
      lv.pair = 1;
      p.levels[top + 1].pair = 2;
      lv.xcap = 2u * lv.kcap;
      xcap_max = std::max(xcap_max, lv.xcap);
      --units;
    } else if (d > 0) {
      return make_plan(n, w, B, static_cast<int32_t>(d - 1), tile_bytes, flags, out);
    }
  }
  p.units = units;
  p.hbm_passes = nlocal + units;
  const bool pairs = xcap_max > 0;
  const bool literal = (flags & MS_FLAG_LITERAL) != 0;
  const bool balanced = (flags & MS_FLAG_BALANCED) != 0;
  uint32_t lcap_max = 0;
  for (uint32_t i = 0; i < p.nlevels; ++i) {
    uint32_t lg = 0;
    while ((1ull << lg) < p.levels[i].Nmax) ++lg;
    p.levels[i].lcap = literal ? std::min(lg + 12u, 64u) : 0u;
    lcap_max = std::max(lcap_max, static_cast<uint32_t>(p.levels[i].M) * p.levels[i].lcap);
  }

  size_t off = 0;
  p.off_buf = off;
  if (p.nlevels > 0) off += round_up(n * w, 256);
  if (p.nlevels > 0 && kcap_max > 0) {
    const size_t base = off;
    p.off_zc = off;     off += round_up(zc_cap * 4, 256);
    p.off_minfo = off;  off += round_up(minfo_cap * 16, 256);
    p.off_ctrl = off;   off += 256;
    p.off_mv = off;     off += round_up(kcap_max * 4, 256);
    p.off_hkeys = off;  off += round_up((1ull << hbits_max) * 8, 256);
    p.off_hvals = off;  off += round_up((1ull << hbits_max) * 4, 256);
    p.off_pdst = off;   off += round_up(2 * kcap_max * 4, 256);
    p.off_psrc = off;   off += round_up(2 * kcap_max * 4, 256);
    p.off_ptmp = off;   off += round_up(2 * kcap_max * w, 256);
    p.off_ostart = off; off += round_up((kcap_max / 1024 + 2) * 4, 256);
    p.plan_set_bytes = off - base;
    // a unit (a level or a fused pair) uses two plan sets; two units' sets, so that the next
    // unit's plan can be built during a unit's data pass
    p.plan_sets = units >= 2 ? 4u : 2u;
    off += (p.plan_sets - 1) * p.plan_set_bytes;
    // exception structures of a pair's first level, one copy per live unit (after the sets)
    if (pairs || literal || balanced) {
      const size_t ebase = off;
      p.off_zb = off - ebase;     off += round_up(zc_cap * 32ull, 256);
      if (pairs) {
        const uint64_t xblocks = (n + kXBlock - 1) / kXBlock;
        p.off_xbits = off - ebase;  off += round_up((n + 31) / 32 * 4, 256);
        p.off_xsrc = off - ebase;   off += round_up(static_cast<size_t>(xcap_max) * 4, 256);
        p.off_xval = off - ebase;   off += round_up(static_cast<size_t>(xcap_max) * 4, 256);
        p.off_xbpre = off - ebase;  off += round_up(xblocks * 4, 256);
        p.off_xtpre = off - ebase;
        off += round_up((xblocks + kXTileBlocks - 1) / kXTileBlocks * 4, 256);
        p.off_xrange = off - ebase; off += round_up(zc_cap * 128ull, 256);  // 2 x 16 words a chunk
      }
      if (literal) {
        p.off_laps = off - ebase;   off += round_up(static_cast<size_t>(lcap_max) * 8u, 256);
        p.off_ctab = off - ebase;   off += round_up(zc_cap * 128ull * 8u, 256);
      }
      if (balanced) {
        p.off_labels = off - ebase; off += round_up(n, 256);
        p.off_zlab = off - ebase;   off += round_up(zc_cap * 4ull, 256);
      }
      p.exc_base = ebase;
      p.exc_bytes = off - ebase;
      off += (p.plan_sets / 2 - 1) * p.exc_bytes;
    }
  }
  p.ws_bytes = off > 256 ? off : 256;
  *out = p;
  return 0;
}

}  // namespace msk

using msk::Plan;

namespace {
// CUDA error behind the calling thread's last MS_ERR_CUDA (ms_last_cuda_error)
thread_local cudaError_t g_last_cuda_error = cudaSuccess;
bool failed(cudaError_t e) {
  if (e == cudaSuccess) return false;
  g_last_cuda_error = e;
  return true;
}
}  // namespace

namespace msk {
// autotuner lookup (ms_tune.cu): B = 0 resolved from the tuning table
ms_params resolve_single(uint64_t n, uint32_t w, const ms_params *p);
ms_params resolve_batch(uint32_t k, const uint64_t *h_n, uint32_t w, const ms_params *p);
}  // namespace msk

namespace {

const char *const kKindNames[msk::kKindNum] = {
    "leaf", "count", "scan", "kscan", "hash_clear", "tail_insert", "tail_resolve",
    "gather", "tail_sequential", "patch_read", "patch_write", "local_level", "batch_engine",
    "pair_gather", "exceptions"};

// Process-wide event recorder used when MS_FLAG_PROFILE is set.
class EventProfiler final : public msk::Prof {
 public:
  void begin(int kind, cudaStream_t s) override {
    Rec r;
    r.kind = kind;
    r.a = take();
    r.b = take();
    cudaEventRecord(r.a, s);
    recs_.push_back(r);
  }
  void end(cudaStream_t s) override {
    if (!recs_.empty()) cudaEventRecord(recs_.back().b, s);
  }
  ms_status read(ms_profile *out, bool reset) {
    std::memset(out, 0, sizeof *out);
    out->kinds = msk::kKindNum;
    for (int k = 0; k < msk::kKindNum; ++k)
      std::strncpy(out->names[k], kKindNames[k], sizeof out->names[k] - 1);
    for (const Rec &r : recs_) {
      if (failed(cudaEventSynchronize(r.b))) return MS_ERR_CUDA;
      float ms = 0.f;
      if (failed(cudaEventElapsedTime(&ms, r.a, r.b))) return MS_ERR_CUDA;
      out->launches[r.kind] += 1;
      out->ms[r.kind] += ms;
    }
    if (reset) {
      for (const Rec &r : recs_) {
        pool_.push_back(r.a);
        pool_.push_back(r.b);
      }
      recs_.clear();
    }
    return MS_OK;
  }

 private:
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  cudaEvent_t take() {
    if (!pool_.empty()) {
      cudaEvent_t e = pool_.back();
      pool_.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  std::vector<Rec> recs_;
  std::vector<cudaEvent_t> pool_;
};

EventProfiler &profiler() {
  static EventProfiler p;
  return p;
}
std::mutex g_prof_mu;

ms_status plan_for(uint64_t n, uint32_t w, const ms_params *p, Plan *plan) {
  const ms_params r = msk::resolve_single(n, w, p);
  const int rc = msk::make_plan(n, w, r.B, r.fuse_depth, r.tile_bytes, r.flags, plan);
  if (rc == 1) return MS_ERR_INVALID;
  if (rc == 2) return MS_ERR_UNSUPPORTED;
  return MS_OK;
}

msk::Buffers buffers_for(const Plan &p, void *data, void *ws, uint32_t set) {
  char *base = static_cast<char *>(ws);
  char *ps = base + static_cast<size_t>(set) * p.plan_set_bytes;  // this plan set
  msk::Buffers b;
  b.data = data;
  b.other = base + p.off_buf;
  char *es = base + p.exc_base + static_cast<size_t>(set / 2) * p.exc_bytes;  // unit's copy
  b.zb = reinterpret_cast<uint8_t *>(es + p.off_zb);
  b.xbits = reinterpret_cast<uint32_t *>(es + p.off_xbits);
  b.xsrc = reinterpret_cast<uint32_t *>(es + p.off_xsrc);
  b.xval = reinterpret_cast<uint32_t *>(es + p.off_xval);
  b.xbpre = reinterpret_cast<uint32_t *>(es + p.off_xbpre);
  b.xtpre = reinterpret_cast<uint32_t *>(es + p.off_xtpre);
  b.xrange = reinterpret_cast<uint4 *>(es + p.off_xrange);
  b.laps = reinterpret_cast<uint2 *>(es + p.off_laps);
  b.ctab = reinterpret_cast<uint2 *>(es + p.off_ctab);
  b.labels = reinterpret_cast<uint8_t *>(es + p.off_labels);
  b.zlab = reinterpret_cast<uint32_t *>(es + p.off_zlab);
  b.zc = reinterpret_cast<uint32_t *>(ps + p.off_zc);
  b.minfo = reinterpret_cast<uint4 *>(ps + p.off_minfo);
  b.ctrl = reinterpret_cast<uint32_t *>(ps + p.off_ctrl);
  b.mv = reinterpret_cast<uint32_t *>(ps + p.off_mv);
  b.hkeys = reinterpret_cast<unsigned long long *>(ps + p.off_hkeys);
  b.hvals = reinterpret_cast<uint32_t *>(ps + p.off_hvals);
  b.pdst = reinterpret_cast<uint32_t *>(ps + p.off_pdst);
  b.psrc = reinterpret_cast<uint32_t *>(ps + p.off_psrc);
  b.ptmp = ps + p.off_ptmp;
  b.ostart = reinterpret_cast<uint32_t *>(ps + p.off_ostart);
  return b;
}

// The plan stream paired with a caller's stream (per device, created on first use), with the
// events of the two-set pipeline. It runs at the caller's priority (the lowest for a default
// stream): its short kernels fill the SMs between the data pass's blocks instead of displacing
// them (measured on GB300: one priority above the data pass, the plan kernels slowed the
// 128-thread staged gathers of a 2^30 perm by more than they saved), and a call made on a
// high-priority stream keeps its plans ahead of other callers' work. A mutex serialises the
// enqueue of one call's pipeline per caller stream.
struct PlanStream {
  int dev = -1;
  cudaStream_t caller = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr;
  cudaEvent_t planned[2] = {};
  cudaEvent_t released[2] = {};
  std::mutex mu;
};

ms_status plan_stream(cudaStream_t caller, PlanStream **out) {
  static std::mutex mu;
  static PlanStream pool[64];
  static uint32_t used = 0;
  int dev = 0;
  if (failed(cudaGetDevice(&dev))) return MS_ERR_CUDA;
  std::lock_guard<std::mutex> g(mu);
  for (uint32_t i = 0; i < used; ++i)
    if (pool[i].dev == dev && pool[i].caller == caller) {
      *out = &pool[i];
      return MS_OK;
    }
  if (used == 64) {
    *out = nullptr;  // too many distinct caller streams: the call runs without the side stream
    return MS_OK;
  }
  PlanStream &S = pool[used];
  int prio = 0;
  if (failed(cudaStreamGetPriority(caller, &prio))) return MS_ERR_CUDA;
  if (failed(cudaStreamCreateWithPriority(&S.side, cudaStreamNonBlocking, prio)))
    return MS_ERR_CUDA;
  for (int k = 0; k < 2; ++k) {
    if (failed(cudaEventCreateWithFlags(&S.planned[k], cudaEventDisableTiming)) ||
        failed(cudaEventCreateWithFlags(&S.released[k], cudaEventDisableTiming)))
      return MS_ERR_CUDA;
  }
  if (failed(cudaEventCreateWithFlags(&S.fork, cudaEventDisableTiming)))
    return MS_ERR_CUDA;
  S.dev = dev;
  S.caller = caller;
  ++used;
  *out = &S;
  return MS_OK;
}

ms_status run(void *data, bool perm, uint64_t n, uint32_t w, uint64_t seed, void *ws,
              size_t ws_bytes, const ms_params *params, cudaStream_t s);

// An NVTX range over the enqueue of one call or one of its passes (a no-op unless a profiler
// such as Nsight Systems is attached), so a timeline shows which pass launched which kernels.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// 1- and 2-byte elements: the permutation ms_perm gives for (n, seed, B) into the front of the
// workspace, the elements gathered through it into the 4-byte path's ping-pong buffer, then
// copied back (a shuffle is its input gathered through that permutation, whatever the width).
ms_status run_narrow(void *data, uint64_t n, uint32_t w, uint64_t seed, void *ws,
                     size_t ws_bytes, const ms_params *params, cudaStream_t s) {
  ms_params pp;
  ms_default_params(&pp);
  if (params) pp = *params;
  pp = msk::resolve_single(n, w, &pp);  // (narrow widths resolve as 4-byte elements)
  Plan p4;
  ms_params pp4 = pp;
  pp4.flags |= MS_FLAG_PERM;
  const ms_status ps = plan_for(n, 4, &pp4, &p4);
  if (ps != MS_OK) return ps;
  if (n <= 1) return MS_OK;
  const size_t need = ms_workspace_bytes(n, w, &pp);
  if (need == 0) return MS_ERR_INVALID;
  if (data == nullptr || reinterpret_cast<uintptr_t>(data) % w != 0) return MS_ERR_INVALID;
  if (ws == nullptr || ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return MS_ERR_INVALID;
  const size_t front = msk::round_up(n * 4u, 256);
  uint32_t *const idx = static_cast<uint32_t *>(ws);
  char *const inner = static_cast<char *>(ws) + front;
  const ms_status st = run(idx, true, n, 4, seed, inner, ws_bytes - front, &pp, s);
  if (st != MS_OK) return st;
  void *const tmp = inner + p4.off_buf;  // n * 4 bytes, free once the permutation is written
  int dev = 0, sms = 0;
  if (failed(cudaGetDevice(&dev)) ||
      failed(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
    return MS_ERR_CUDA;
  if (failed(msk::launch_narrow_gather(data, idx, tmp, n, w, sms, s))) return MS_ERR_CUDA;
  if (failed(cudaMemcpyAsync(data, tmp, n * w, cudaMemcpyDeviceToDevice, s))) return MS_ERR_CUDA;
  return MS_OK;
}

ms_status run(void *data, bool perm, uint64_t n, uint32_t w, uint64_t seed, void *ws,
              size_t ws_bytes, const ms_params *params, cudaStream_t s) {
  if (!perm && (w == 1 || w == 2)) return run_narrow(data, n, w, seed, ws, ws_bytes, params, s);
  Plan p;
  ms_params pp;
  ms_default_params(&pp);
  if (params) pp = *params;
  if (perm) pp.flags |= MS_FLAG_PERM;
  else pp.flags &= ~MS_FLAG_PERM;
  const ms_status st = plan_for(n, w, &pp, &p);
  if (st != MS_OK) return st;
  if (n <= 1) {
    if (perm && n == 1) {
      // the permutation of {0}: one zero word, stream-ordered (no host source, no sync)
      if (data == nullptr || reinterpret_cast<uintptr_t>(data) % 4 != 0) return MS_ERR_INVALID;
      if (failed(cudaMemsetAsync(data, 0, 4, s))) return MS_ERR_CUDA;
    }
    return MS_OK;
  }
  if (data == nullptr) return MS_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(data) % w != 0) return MS_ERR_INVALID;
  if (ws_bytes < p.ws_bytes) return MS_ERR_INVALID;
  if (p.ws_bytes > 256 && (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0))
    return MS_ERR_INVALID;
  const msk::Buffers b0 = buffers_for(p, data, ws, 0);
  std::unique_lock<std::mutex> prof_lock(g_prof_mu, std::defer_lock);
  if (p.flags & MS_FLAG_PROFILE) {
    prof_lock.lock();
    p.prof = &profiler();
  }
  // global units (a single level or a fused pair of levels), in order. Unit u uses plan sets
  // 2(u % 2) and 2(u % 2) + 1 (the pair's second level takes the second); its plan runs on the
  // side stream, two units ahead at most (the sets of unit u are released when unit u - 2's
  // data pass is done).
  uint32_t unit_level[33];
  uint32_t nu = 0;
  for (uint32_t i = 0; i < p.nlevels; ++i)
    if (!p.levels[i].local && p.levels[i].pair != 2) unit_level[nu++] = i;
  PlanStream *P = nullptr;
  if (nu >= 1 && p.plan_sets >= 2 && !(p.flags & MS_FLAG_SINGLE_STREAM) &&
      plan_stream(s, &P) != MS_OK)
    return MS_ERR_CUDA;
  const uint32_t slots = p.plan_sets >= 4 ? 2u : 1u;  // units whose sets can be live at once
  auto unit_sets = [&](uint32_t u, msk::Buffers *b1, msk::Buffers *b2) {
    const uint32_t base = 2u * (u % slots);
    *b1 = buffers_for(p, data, ws, base);
    *b2 = buffers_for(p, data, ws, base + 1u);
  };
  auto launch_unit_plan = [&](uint32_t u, cudaStream_t st) -> bool {
    msk::Buffers b1, b2;
    unit_sets(u, &b1, &b2);
    const msk::LevelPlan &lv = p.levels[unit_level[u]];
    if (lv.pair == 1)
      return !failed(
          msk::launch_pair_plan(p, lv, p.levels[unit_level[u] + 1], b1, b2, seed, st));
    return !failed(msk::launch_level_plan(p, lv, b1, seed, st));
  };
  auto plan_on_side = [&](uint32_t u) -> bool {
    const uint32_t k = u % 2;
    if (u >= slots && failed(cudaStreamWaitEvent(P->side, P->released[k], 0))) return false;
    if (!launch_unit_plan(u, P->side)) return false;
    return !failed(cudaEventRecord(P->planned[k], P->side));
  };
  std::unique_lock<std::mutex> pipe_lock;
  if (P) {
    pipe_lock = std::unique_lock<std::mutex>(P->mu);
    // the side stream starts after everything already on the caller's stream (earlier calls
    // may still be reading the plan sets)
    if (failed(cudaEventRecord(P->fork, s))) return MS_ERR_CUDA;
    if (failed(cudaStreamWaitEvent(P->side, P->fork, 0))) return MS_ERR_CUDA;
    for (uint32_t u = 0; u < nu && u < slots; ++u)
      if (!plan_on_side(u)) return MS_ERR_CUDA;
  }
  NvtxRange call_range(perm ? "ms_perm" : "ms_shuffle");
  void *cur = (p.hbm_passes % 2 == 0) ? data : b0.other;
  {
    NvtxRange r(p.d > 0 ? "base blocks and fused levels" : "base blocks");
    if (failed(msk::launch_leaf(p, data, cur, perm, seed, s))) return MS_ERR_CUDA;
  }
  uint32_t u = 0;  // next global unit
  for (uint32_t i = 0; i < p.nlevels; ++i) {
    const msk::LevelPlan &lv = p.levels[i];
    if (lv.pair == 2) continue;  // done with the pair's first level
    void *dst = (cur == data) ? b0.other : data;
    cudaError_t e = cudaSuccess;
    char label[48];
    std::snprintf(label, sizeof label, lv.pair == 1 ? "levels %u-%u" : "level %u", lv.level,
                  lv.level + 1u);
    NvtxRange level_range(label);
    if (lv.span) {
      e = msk::launch_span_level(p, lv, cur, dst, seed, s);
    } else if (lv.warp_local) {
      e = msk::launch_warp_level(p, lv, cur, dst, seed, s);
    } else if (lv.local) {
      e = msk::launch_local_level(p, lv, cur, dst, seed, s);
    } else {
      msk::Buffers b1, b2;
      unit_sets(u, &b1, &b2);
      if (P) {
        if (failed(cudaStreamWaitEvent(s, P->planned[u % 2], 0))) return MS_ERR_CUDA;
      } else if (!launch_unit_plan(u, s)) {
        return MS_ERR_CUDA;
      }
      e = lv.pair == 1 ? msk::launch_pair_data(p, lv, p.levels[i + 1], cur, dst, b1, b2, seed, s)
                       : msk::launch_level_data(p, lv, cur, dst, b1, seed, s);
      if (e == cudaSuccess && P) {
        if (failed(cudaEventRecord(P->released[u % 2], s))) return MS_ERR_CUDA;
        if (u + slots < nu && !plan_on_side(u + slots)) return MS_ERR_CUDA;
      }
      ++u;
    }
    if (failed(e)) return MS_ERR_CUDA;
    cur = dst;
  }
  return MS_OK;
}

// ------------------------------------------------------------------ batch layout ---------
constexpr uint32_t kEngineGrid = 320;  // persistent CTAs (2 per SM on a 152-SM GB300, spare)

struct BatchLayout {
  size_t off_table = 0, off_queue = 0, off_scratch = 0, off_large = 0, total = 0;
  std::vector<size_t> tmp_off;   // per instance: engine ping-pong buffer (SIZE_MAX otherwise)
  std::vector<uint32_t> order;   // engine instances, largest first
  std::vector<uint32_t> large;   // instances for the single-instance path
  size_t scratch_per_cta = 0;
  size_t large_ws = 0;           // one single-instance workspace
  uint32_t large_streams = 0;    // single-instance workspaces (one per side stream)
};

constexpr uint32_t kBatchSideStreams = 4;

// Which instances the engine takes: at most 2^22 elements, and -- since one CTA finishes an
// instance alone -- none much larger than the batch's average share per CTA (the rest run
// faster on the whole GPU through the single-instance path, a few of them concurrently).
ms_status batch_layout(uint32_t k, const uint64_t *h_n, uint32_t w, const ms_params *params,
                       BatchLayout *L) {
  const ms_params r = msk::resolve_batch(k, h_n, w, params);
  if (w == 1 || w == 2) return MS_ERR_UNSUPPORTED;  // (the single call takes them)
  if (w != 4 && w != 8 && w != 16) return MS_ERR_INVALID;
  if ((r.flags & MS_FLAG_PERM) && w != 4) return MS_ERR_INVALID;
  if (r.flags & (MS_FLAG_LITERAL | MS_FLAG_FDR | MS_FLAG_BALANCED)) return MS_ERR_UNSUPPORTED;
  if (r.B == 0) return MS_ERR_INVALID;
  if (r.B > MS_MAX_B) return MS_ERR_UNSUPPORTED;
  if (k > 0 && h_n == nullptr) return MS_ERR_INVALID;
  L->tmp_off.assign(k, SIZE_MAX);
  L->order.clear();
  L->large.clear();
  std::vector<uint32_t> cand;
  uint64_t cand_total = 0;
  for (uint32_t i = 0; i < k; ++i) {
    if (h_n[i] > 0xFFFFFFFFull) return MS_ERR_INVALID;
    if (h_n[i] >= 2 && h_n[i] <= msk::kEngineMaxN) {
      cand.push_back(i);
      cand_total += h_n[i];
    } else if (h_n[i] > msk::kEngineMaxN) {
      L->large.push_back(i);
    }
  }
  std::stable_sort(cand.begin(), cand.end(),
                   [&](uint32_t x, uint32_t y) { return h_n[x] > h_n[y]; });
  size_t first = 0;
  while (first < cand.size() && h_n[cand[first]] > (1u << 16) &&
         h_n[cand[first]] * kEngineGrid > 2 * cand_total) {
    cand_total -= h_n[cand[first]];
    L->large.push_back(cand[first]);
    ++first;
  }
  L->order.assign(cand.begin() + first, cand.end());
  std::sort(L->large.begin(), L->large.end());
  for (uint32_t i : L->large) {
    const size_t ws = ms_workspace_bytes(h_n[i], w, &r);
    if (ws == 0) return MS_ERR_INVALID;
    L->large_ws = std::max(L->large_ws, ws);
  }
  L->large_streams = static_cast<uint32_t>(
      std::min<size_t>(L->large.size(), kBatchSideStreams));
  size_t off = msk::round_up(static_cast<size_t>(k) * msk::engine_inst_bytes() + 1, 256);
  L->off_table = 0;
  L->off_queue = off;
  off += 256;
  for (uint32_t i : L->order) {
    L->tmp_off[i] = off;
    off += msk::round_up(h_n[i] * w, 256);
  }
  L->scratch_per_cta =
      msk::round_up((2ull << msk::kEngineHbits) * 4 + 3ull * msk::kEngineKcap * 4, 256);
  L->off_scratch = off;
  if (!L->order.empty()) off += L->scratch_per_cta * kEngineGrid;
  L->off_large = off;
  off += L->large_ws * L->large_streams;
  L->total = off;
  return MS_OK;
}

// Side streams of the batch form, one set per (device, caller stream), created on first use:
// large instances fork off the caller's stream onto them and join back before the call's work
// ends. Keying them by the caller's stream keeps unrelated callers (and captures) from being
// chained to each other; the set's mutex is held from the fork record to the last join wait,
// so two host threads on the same caller stream cannot re-record the fork event in between.
struct SideStreams {
  int dev = -1;
  cudaStream_t caller = nullptr;
  cudaStream_t s[kBatchSideStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kBatchSideStreams] = {};
  std::mutex mu;
};

ms_status side_streams(cudaStream_t caller, SideStreams **out) {
  static std::mutex mu;
  static SideStreams pool[64];
  static uint32_t used = 0;
  int dev = 0;
  if (failed(cudaGetDevice(&dev))) return MS_ERR_CUDA;
  std::lock_guard<std::mutex> g(mu);
  for (uint32_t i = 0; i < used; ++i)
    if (pool[i].dev == dev && pool[i].caller == caller) {
      *out = &pool[i];
      return MS_OK;
    }
  if (used == 64) {
    *out = nullptr;  // too many distinct caller streams: the large instances run in order
    return MS_OK;
  }
  SideStreams &S = pool[used];
  for (uint32_t i = 0; i < kBatchSideStreams; ++i) {
    if (failed(cudaStreamCreateWithFlags(&S.s[i], cudaStreamNonBlocking))) return MS_ERR_CUDA;
    if (failed(cudaEventCreateWithFlags(&S.join[i], cudaEventDisableTiming))) return MS_ERR_CUDA;
  }
  if (failed(cudaEventCreateWithFlags(&S.fork, cudaEventDisableTiming))) return MS_ERR_CUDA;
  S.dev = dev;
  S.caller = caller;
  ++used;
  *out = &S;
  return MS_OK;
}

struct BatchInstHost {  // mirrors the device descriptor of ms_batch.cu
  uint64_t data, tmp, n, seed;
  uint32_t flags, pad;
};

}  // namespace

extern "C" {

size_t ms_batch_workspace_bytes(uint32_t k, const uint64_t *h_n, uint32_t w,
                                const ms_params *p) {
  BatchLayout L;
  if (batch_layout(k, h_n, w, p, &L) != MS_OK) return 0;
  return L.total;
}

static ms_status batch_check(uint32_t k, void *const *h_ptrs, const uint64_t *h_n, uint32_t w,
                             void *d_ws, size_t ws_bytes, const ms_params *p, BatchLayout *L) {
  const ms_status st = batch_layout(k, h_n, w, p, L);
  if (st != MS_OK) return st;
  if (k > 0 && h_ptrs == nullptr) return MS_ERR_INVALID;
  if (ws_bytes < L->total || d_ws == nullptr || reinterpret_cast<uintptr_t>(d_ws) % 256 != 0)
    return MS_ERR_INVALID;
  for (uint32_t i = 0; i < k; ++i)
    if (h_n[i] > 1 && (h_ptrs[i] == nullptr || reinterpret_cast<uintptr_t>(h_ptrs[i]) % w != 0))
      return MS_ERR_INVALID;
  return MS_OK;
}

ms_status ms_batch_prepare(uint32_t k, void *const *h_ptrs, const uint64_t *h_n, uint32_t w,
                           const uint64_t *h_seeds, uint64_t base_seed, void *d_ws,
                           size_t ws_bytes, const ms_params *p, ms_stream_t stream) {
  BatchLayout L;
  const ms_status st = batch_check(k, h_ptrs, h_n, w, d_ws, ws_bytes, p, &L);
  if (st != MS_OK) return st;
  if (L.order.empty()) return MS_OK;
  if (sizeof(BatchInstHost) != msk::engine_inst_bytes()) return MS_ERR_INVALID;
  std::vector<BatchInstHost> table(L.order.size());
  char *base = static_cast<char *>(d_ws);
  for (size_t q = 0; q < L.order.size(); ++q) {
    const uint32_t i = L.order[q];
    BatchInstHost &e = table[q];
    e.data = reinterpret_cast<uintptr_t>(h_ptrs[i]);
    e.tmp = reinterpret_cast<uintptr_t>(base + L.tmp_off[i]);
    e.n = h_n[i];
    e.seed = h_seeds ? h_seeds[i] : base_seed + i;
    e.flags = 0;
    e.pad = 0;
  }
  // pageable source: the copy has consumed it when the call returns
  if (failed(cudaMemcpyAsync(base + L.off_table, table.data(), table.size() * sizeof(BatchInstHost),
                      cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream))))
    return MS_ERR_CUDA;
  return MS_OK;
}

ms_status ms_batch_run(uint32_t k, void *const *h_ptrs, const uint64_t *h_n, uint32_t w,
                       const uint64_t *h_seeds, uint64_t base_seed, void *d_ws, size_t ws_bytes,
                       const ms_params *p, ms_stream_t stream) {
  BatchLayout L;
  const ms_status st = batch_check(k, h_ptrs, h_n, w, d_ws, ws_bytes, p, &L);
  if (st != MS_OK) return st;
  // one B for the whole batch (large instances included)
  const ms_params r = msk::resolve_batch(k, h_n, w, p);
  const bool perm = (r.flags & MS_FLAG_PERM) != 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char *base = static_cast<char *>(d_ws);
  std::unique_lock<std::mutex> prof_lock(g_prof_mu, std::defer_lock);
  msk::Prof *prof = nullptr;
  if (r.flags & MS_FLAG_PROFILE) {
    prof_lock.lock();
    prof = &profiler();
  }
  if (!L.order.empty()) {
    if (failed(msk::launch_engine(w, perm, base + L.off_table, static_cast<uint32_t>(L.order.size()),
                           reinterpret_cast<uint32_t *>(base + L.off_queue), r.B,
                           base + L.off_scratch, L.scratch_per_cta, msk::kEngineKcap,
                           msk::kEngineHbits, kEngineGrid, msk::kEngineSmem, s,
                           prof)))
      return MS_ERR_CUDA;
  }
  if (prof_lock.owns_lock()) prof_lock.unlock();
  for (uint32_t i = 0; i < k; ++i) {
    if (perm && h_n[i] == 1 && failed(cudaMemsetAsync(h_ptrs[i], 0, 4, s)))
      return MS_ERR_CUDA;
  }
  if (L.large.empty()) return MS_OK;
  SideStreams *S = nullptr;
  if (L.large_streams > 1 && side_streams(s, &S) != MS_OK) return MS_ERR_CUDA;
  if (S == nullptr) {
    for (uint32_t i : L.large) {
      const uint64_t seed = h_seeds ? h_seeds[i] : base_seed + i;
      const ms_status rs = run(h_ptrs[i], perm, h_n[i], w, seed, base + L.off_large, L.large_ws,
                               &r, s);
      if (rs != MS_OK) return rs;
    }
    return MS_OK;
  }
  // several large instances: fork onto this caller's side streams, one workspace each, join back
  std::lock_guard<std::mutex> fork_lock(S->mu);
  if (failed(cudaEventRecord(S->fork, s))) return MS_ERR_CUDA;
  for (uint32_t j = 0; j < L.large_streams; ++j)
    if (failed(cudaStreamWaitEvent(S->s[j], S->fork, 0))) return MS_ERR_CUDA;
  for (size_t t = 0; t < L.large.size(); ++t) {
    const uint32_t i = L.large[t];
    const uint32_t j = static_cast<uint32_t>(t % L.large_streams);
    const uint64_t seed = h_seeds ? h_seeds[i] : base_seed + i;
    const ms_status rs = run(h_ptrs[i], perm, h_n[i], w, seed, base + L.off_large + j * L.large_ws,
                             L.large_ws, &r, S->s[j]);
    if (rs != MS_OK) return rs;
  }
  for (uint32_t j = 0; j < L.large_streams; ++j) {
    if (failed(cudaEventRecord(S->join[j], S->s[j]))) return MS_ERR_CUDA;
    if (failed(cudaStreamWaitEvent(s, S->join[j], 0))) return MS_ERR_CUDA;
  }
  return MS_OK;
}

ms_status ms_shuffle_batch(uint32_t k, void *const *h_ptrs, const uint64_t *h_n, uint32_t w,
                           const uint64_t *h_seeds, uint64_t base_seed, void *d_ws,
                           size_t ws_bytes, const ms_params *p, ms_stream_t stream) {
  const ms_status st =
      ms_batch_prepare(k, h_ptrs, h_n, w, h_seeds, base_seed, d_ws, ws_bytes, p, stream);
  if (st != MS_OK) return st;
  return ms_batch_run(k, h_ptrs, h_n, w, h_seeds, base_seed, d_ws, ws_bytes, p, stream);
}


void ms_default_params(ms_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->B = 1024;
  p->fuse_depth = -1;
  p->flags = 0;
  p->tile_bytes = 0;
}

ms_status ms_plan_info(uint64_t n, uint32_t w, const ms_params *params, ms_plan *out) {
  if (!out) return MS_ERR_INVALID;
  Plan p;
  const ms_status st = plan_for(n, w, params, &p);
  if (st != MS_OK) return st;
  std::memset(out, 0, sizeof *out);
  out->n = p.n;
  out->w = p.w;
  out->B = p.B;
  out->c = p.c;
  out->fuse_depth = p.d;
  out->hbm_levels = p.nlevels;
  out->passes = n <= 1 ? 0u : 1u + p.hbm_passes;
  out->tiles = n <= 1 ? 0u : p.tiles;
  out->tile_max = n <= 1 ? n : p.tile_max;
  out->workspace_bytes = p.ws_bytes;
  uint32_t launches = n <= 1 ? 0u : 1u;
  uint32_t global = 0;
  for (uint32_t i = 0; i < p.nlevels && n > 1; ++i) {
    const msk::LevelPlan &lv = p.levels[i];
    // global single level: 6 plan + 4 data launches (a memset among them); fused pair: 6 + 6
    // plan, 3 exception-map steps, 7 data launches (4 of them idle unless the fallback runs)
    launches += lv.local ? 1u : lv.pair == 1 ? 22u : lv.pair == 2 ? 0u : 10u;
    global += lv.local ? 0u : 1u;
  }
  out->kernel_launches = launches;
  out->global_levels = global;
  uint32_t pairs = 0;
  for (uint32_t i = 0; i < p.nlevels && n > 1; ++i) pairs += p.levels[i].pair == 1 ? 1u : 0u;
  out->fused_pairs = pairs;
  out->tile_smem = (n > 1 && p.tile_mode) ? static_cast<uint32_t>(p.tile_smem) : 0u;
  return MS_OK;
}

ms_status ms_profile_read(ms_profile *out, int reset) {
  if (!out) return MS_ERR_INVALID;
  std::lock_guard<std::mutex> g(g_prof_mu);
  return profiler().read(out, reset != 0);
}

size_t ms_workspace_bytes(uint64_t n, uint32_t w, const ms_params *params) {
  // 1- and 2-byte elements: the permutation's indices, then the 4-byte path's workspace (whose
  // ping-pong buffer later holds the gathered elements)
  if (w == 1 || w == 2) {
    const size_t inner = ms_workspace_bytes(n, 4, params);
    return inner ? msk::round_up(n * 4u, 256) + inner : 0;
  }
  // enough for ms_shuffle and (w = 4) ms_perm, whose plans may differ in how the levels after
  // the base-block pass are grouped
  ms_params pp;
  ms_default_params(&pp);
  if (params) pp = *params;
  Plan p;
  pp.flags &= ~MS_FLAG_PERM;
  if (plan_for(n, w, &pp, &p) != MS_OK) return 0;
  size_t ws = p.ws_bytes;
  if (w == 4) {
    pp.flags |= MS_FLAG_PERM;
    if (plan_for(n, w, &pp, &p) != MS_OK) return 0;
    ws = std::max(ws, p.ws_bytes);
  }
  return ws;
}

ms_status ms_shuffle(void *d_data, uint64_t n, uint32_t w, uint64_t seed, void *d_ws,
                     size_t ws_bytes, const ms_params *p, ms_stream_t stream) {
  return run(d_data, false, n, w, seed, d_ws, ws_bytes, p, static_cast<cudaStream_t>(stream));
}

ms_status ms_perm(uint32_t *d_out, uint64_t n, uint64_t seed, void *d_ws, size_t ws_bytes,
                  const ms_params *p, ms_stream_t stream) {
  return run(d_out, true, n, 4, seed, d_ws, ws_bytes, p, static_cast<cudaStream_t>(stream));
}

size_t ms_host_workspace_bytes(uint64_t n, uint32_t w, const ms_params *params) {
  const size_t inner = ms_workspace_bytes(n, w, params);
  if (inner == 0) return 0;
  return msk::round_up(n * w, 256) + inner;
}

static ms_status host_form(void *h, bool perm, uint64_t n, uint32_t w, uint64_t seed, void *d_ws,
                           size_t ws_bytes, const ms_params *params, cudaStream_t s) {
  const size_t need = ms_host_workspace_bytes(n, w, params);
  if (need == 0) return MS_ERR_INVALID;
  if (n == 0) return MS_OK;
  if (h == nullptr || d_ws == nullptr || ws_bytes < need) return MS_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0) return MS_ERR_INVALID;
  const size_t front = msk::round_up(n * w, 256);
  void *d_buf = d_ws;
  void *inner = static_cast<char *>(d_ws) + front;
  if (!perm && failed(cudaMemcpyAsync(d_buf, h, n * w, cudaMemcpyHostToDevice, s)))
    return MS_ERR_CUDA;
  const ms_status st = run(d_buf, perm, n, w, seed, inner, ws_bytes - front, params, s);
  if (st != MS_OK) return st;
  if (failed(cudaMemcpyAsync(h, d_buf, n * w, cudaMemcpyDeviceToHost, s)))
    return MS_ERR_CUDA;
  if (failed(cudaStreamSynchronize(s))) return MS_ERR_CUDA;
  return MS_OK;
}

ms_status ms_shuffle_host(void *h_data, uint64_t n, uint32_t w, uint64_t seed, void *d_ws,
                          size_t ws_bytes, const ms_params *p, ms_stream_t stream) {
  return host_form(h_data, false, n, w, seed, d_ws, ws_bytes, p,
                   static_cast<cudaStream_t>(stream));
}

ms_status ms_perm_host(uint32_t *h_out, uint64_t n, uint64_t seed, void *d_ws, size_t ws_bytes,
                       const ms_params *p, ms_stream_t stream) {
  return host_form(h_out, true, n, 4, seed, d_ws, ws_bytes, p,
                   static_cast<cudaStream_t>(stream));
}

const char *ms_status_string(ms_status s) {
  switch (s) {
    case MS_OK: return "MS_OK";
    case MS_ERR_INVALID: return "MS_ERR_INVALID";
    case MS_ERR_UNSUPPORTED: return "MS_ERR_UNSUPPORTED";
    case MS_ERR_NOMEM: return "MS_ERR_NOMEM";
    case MS_ERR_CUDA: return "MS_ERR_CUDA";
    case MS_ERR_TIMEOUT: return "MS_ERR_TIMEOUT";
  }
  return "MS_ERR_UNKNOWN";
}

int ms_last_cuda_error(void) { return static_cast<int>(g_last_cuda_error); }

const char *ms_last_cuda_error_string(void) { return cudaGetErrorString(g_last_cuda_error); }

const char *ms_version(void) { return "mergeshuffle-gb300 0.1 (MS-Philox v1, sm_103a)"; }

}  // extern "C"
