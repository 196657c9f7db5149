// ms_tile.cu -- the base blocks of a tile of 2^d consecutive base blocks and the tile's first d
// merge levels (Algorithms 1 to 3 of arXiv 1508.03167), one CTA of eight warps per tile,
// computed on 16-bit tile-local indices in shared memory; the tile is then written once (perm:
// the indices plus the tile's first element; shuffle: the input rows they name).
//
// Per tile:
//   * Algorithm 1's draws for every position of every base block (lane k of each warp: block
//     k; the warps split its positions). A draw whose first Philox word rejects all its slices
//     is queued by its thread and finished after the loop, so no lane holds its warp up with a
//     second Philox block inline;
//   * Algorithm 1's swap chain per block, reading those draws;
//   * per merge level: coin words and their zero prefix, the break step T of every merge,
//     the stable interleave (a lane places eight consecutive positions, walking the two
//     halves with one index each), the tail draws, and the random insertions of Algorithm 3's
//     second loop in order, one lane per merge. The data-independent part of level l+1 (coins,
//     prefixes, break steps by one warp, then the tail draws shared by the seven warps that do
//     not run the tails) is built while the data warp runs level l's tails;
//   * one store of the tile.
// Block k of the tile sits at k*P in the first buffer (P = 2 mod 64, so the 32 lanes at one
// position of their blocks touch 32 different banks); merge r of level l writes its output at
// r*S[l] (S[l] a multiple of eight: a lane stores its eight 16-bit results in one 16-byte store).
// The shared-memory reads of the interleave are clamped to the buffers, so an inconsistent
// plan fails the parity tests instead of reading outside shared memory.
#include "ms_merge.cuh"

namespace msk {
namespace {

// (kFailPerThread is defined with the CTA shape below)

struct TileArgs {
  const void *in;
  void *out;
  uint64_t n;
  uint2 key;
  uint32_t c, d;
  uint32_t P;     // stride of a base block in the Fisher-Yates layout
  uint32_t buf;   // 16-bit entries of each tile buffer (a multiple of eight)
  uint32_t wcap;  // coin words of one level
  uint32_t tcap;  // tail draws of one level made ahead of the data (else drawn in the loop)
  uint32_t S[kTileMaxDepth];  // output stride of one merge of level l
};

__device__ __forceinline__ uint32_t warp_exclusive(uint32_t v, uint32_t *total) {
  const uint32_t incl = warp_inclusive_scan(v);
  *total = __shfl_sync(kFullMask, incl, 31);
  return incl - v;
}

// Control data of one merge level: (coin word, zero prefix) pairs, tail draws, and per merge
// its size, break step, leftover base, first word, first tail draw and first tail quad; then
// whether the tail draws are made ahead and how many quads of them there are (a merge's half
// bases follow from its index and the level's input stride). The control warp builds level
// l+1's while the data warp finishes level l's tails: the tail draws and per-merge words come
// in two sets, the (coin word, zero prefix) pairs in one, as level l's are dead once its
// interleave is done (one set less keeps a tile of 16,384 elements at three CTAs an SM).
struct LevelCtl {
  uint2 *cz;
  uint16_t *mv;
  uint32_t *m;  // kTileCtlWords words: 6 arrays of 32, the flag "tail draws made", the quads
};
constexpr uint32_t kTileCtlWords = 6u * 32u + 2u;
__device__ __forceinline__ uint32_t *ctl_N(const LevelCtl &c) { return c.m; }
__device__ __forceinline__ uint32_t *ctl_T(const LevelCtl &c) { return c.m + 32; }
__device__ __forceinline__ uint32_t *ctl_lb(const LevelCtl &c) { return c.m + 64; }
__device__ __forceinline__ uint32_t *ctl_woff(const LevelCtl &c) { return c.m + 96; }
__device__ __forceinline__ uint32_t *ctl_koff(const LevelCtl &c) { return c.m + 128; }
__device__ __forceinline__ uint32_t *ctl_qoff(const LevelCtl &c) { return c.m + 160; }
__device__ __forceinline__ uint32_t *ctl_drawn(const LevelCtl &c) { return c.m + 192; }
__device__ __forceinline__ uint32_t *ctl_qtot(const LevelCtl &c) { return c.m + 193; }

// The data-independent part of merge level lv of the tile, by one warp: coin words, zero
// prefixes and break step of every merge, the leftover base, and the offsets of the tail draws
// (made by tail_draws). G = 32 / R lanes per merge: lane (r, sub) = (lane / G, lane % G).
__device__ __noinline__ void level_setup(uint2 key, uint32_t d, uint32_t tcap,
                                        const uint32_t *boff, uint64_t k0, uint32_t lv,
                                        uint32_t Sin, uint32_t lane, uint2 *czb, uint16_t *mvb,
                                        uint32_t *mb) {
  LevelCtl c;
  c.cz = czb;
  c.mv = mvb;
  c.m = mb;
  const uint32_t idbase = static_cast<uint32_t>(k0 >> (lv + 1u));
  const uint32_t lgG = 5u - (d - lv - 1u);  // (R = 2^(d-lv-1) <= 32)
  const uint32_t G = 1u << lgG;
  const uint32_t r = lane >> lgG;
  const uint32_t sub = lane & (G - 1u);
  const uint32_t leader = lane & ~(G - 1u);
  const uint32_t kb = (2u * r) << lv;
  const uint32_t n1 = boff[kb + (1u << lv)] - boff[kb];
  const uint32_t N = boff[kb + (2u << lv)] - boff[kb];
  const uint32_t Wm = (N >> 5) + 1u;  // coin words for steps 0..N (the break step is <= N)
  uint32_t Wtot;
  const uint32_t woff = __shfl_sync(kFullMask, warp_exclusive(sub == 0u ? Wm : 0u, &Wtot), leader);
  uint2 *const cz = c.cz + woff;
  // coin words (one Philox block: four words, 128 steps)
  const uint32_t nblk = (Wm + 3u) >> 2;
#pragma unroll 2
  for (uint32_t jb = sub; jb < nblk; jb += G) {
    const uint4 blk = coin_block(key, lv, idbase + r, jb);
    const uint32_t j = 4u * jb;
    cz[j].x = blk.x;
    if (j + 1u < Wm) cz[j + 1u].x = blk.y;
    if (j + 2u < Wm) cz[j + 2u].x = blk.z;
    if (j + 3u < Wm) cz[j + 3u].x = blk.w;
  }
  __syncwarp();
  // zeros before each word of the merge: lane (r, sub) takes a run of C words, then a scan over
  // the merge's G lanes; the same pass finds the break step, the (n1+1)-th zero or the
  // (n2+1)-th one, whichever comes first
  const uint32_t C = (Wm + G - 1u) >> lgG;
  const uint32_t j0 = min(sub * C, Wm), j1 = min(j0 + C, Wm);
  uint32_t zrun = 0;
#pragma unroll 4
  for (uint32_t j = j0; j < j1; ++j) zrun += static_cast<uint32_t>(__popc(~cz[j].x));
  uint32_t Zs = zrun;
#pragma unroll
  for (uint32_t o = 1; o < 32u; o <<= 1) {
    const uint32_t up = __shfl_up_sync(kFullMask, Zs, o, G);
    if (o < G && sub >= o) Zs += up;
  }
  Zs -= zrun;  // zeros before word j0
  const uint32_t n2 = N - n1;
  const uint32_t Z0 = Zs;
#pragma unroll 4
  for (uint32_t j = j0; j < j1; ++j) {
    cz[j].y = Zs;
    Zs += static_cast<uint32_t>(__popc(~cz[j].x));
  }
  // the break step: the (n1+1)-th zero or the (n2+1)-th one, whichever comes first. A lane
  // looks into its words only if its zero (one) ranks cover n1 (n2), at most two lanes a merge,
  // and finds the word by a binary search over the stored prefixes (zeros before word j are
  // cz[j].y, ones 32 j - cz[j].y, both non-decreasing in j)
  uint32_t T = N;
  auto find = [&](bool ones, uint32_t rank) -> uint32_t {
    uint32_t lo = j0, hi = j1;  // the last word whose count before it is at most rank
    while (hi - lo > 1u) {
      const uint32_t mid = (lo + hi) >> 1;
      const uint32_t before = ones ? 32u * mid - cz[mid].y : cz[mid].y;
      if (before <= rank) lo = mid;
      else hi = mid;
    }
    const uint32_t w = cz[lo].x;
    const uint32_t before = ones ? 32u * lo - cz[lo].y : cz[lo].y;
    return 32u * lo + select_set_bit(ones ? w : ~w, rank - before);
  };
  if (j0 < j1) {
    if (Z0 <= n1 && n1 < Zs) T = min(T, find(false, n1));
    if (32u * j0 - Z0 <= n2 && n2 < 32u * j1 - Zs) T = min(T, find(true, n2));
  }
#pragma unroll
  for (uint32_t o = 1; o < 32u; o <<= 1)
    if (o < G) T = min(T, __shfl_xor_sync(kFullMask, T, o, G));
  __syncwarp();
  const uint32_t Ab = 2u * r * Sin;
  const uint32_t Bb = Ab + Sin;
  // positions t >= T take the rest of the half that did not run out, in order; the coin at T
  // names the half that ran out (0: the first half, so t reads X[Bb + t - n1])
  uint32_t lb = Ab - n2;
  if (T < N && ((cz[T >> 5].x >> (T & 31u)) & 1u) == 0u) lb = Bb - n1;
  const uint32_t K = N - T;
  const uint32_t Q = K ? ((N - 1u) >> 2) - (T >> 2) + 1u : 0u;
  uint32_t Ktot, Qtot;
  const uint32_t koff = __shfl_sync(kFullMask, warp_exclusive(sub == 0u ? K : 0u, &Ktot), leader);
  const uint32_t qoff = __shfl_sync(kFullMask, warp_exclusive(sub == 0u ? Q : 0u, &Qtot), leader);
  if (sub == 0u) {
    ctl_N(c)[r] = N;
    ctl_T(c)[r] = T;
    ctl_lb(c)[r] = lb;
    ctl_woff(c)[r] = woff;
    ctl_koff(c)[r] = koff;
    ctl_qoff(c)[r] = qoff;
  }
  if (lane == 0) {
    *ctl_drawn(c) = Ktot <= tcap ? 1u : 0u;  // else the tails draw in their loop
    *ctl_qtot(c) = Qtot;
  }
}

// The tail draws of level lv (one Philox block per four consecutive positions of a merge's
// tail), made ahead of the data by nthreads threads (t: this thread's index among them); quad x
// of the level belongs to the last merge whose first quad is at most x.
__device__ __noinline__ void tail_draws(uint2 key, uint32_t d, uint32_t lv, uint64_t k0,
                                        uint32_t t, uint32_t nthreads, uint16_t *mvb,
                                        const uint32_t *mb) {
  LevelCtl c;
  c.cz = nullptr;
  c.mv = mvb;
  c.m = const_cast<uint32_t *>(mb);
  if (*ctl_drawn(c) == 0u) return;
  const uint32_t R = 1u << (d - lv - 1u);
  const uint32_t idbase = static_cast<uint32_t>(k0 >> (lv + 1u));
  const uint32_t Qtot = *ctl_qtot(c);
  const uint32_t *const qoff = ctl_qoff(c);
  for (uint32_t x = t; x < Qtot; x += nthreads) {
    uint32_t lo = 0, hi = R;
    while (hi - lo > 1u) {
      const uint32_t mid = (lo + hi) >> 1;
      if (qoff[mid] <= x) lo = mid;
      else hi = mid;
    }
    const uint32_t r = lo;
    const uint32_t T = ctl_T(c)[r], N = ctl_N(c)[r], koff = ctl_koff(c)[r];
    const uint32_t quad = (T >> 2) + (x - qoff[r]);
    const uint32_t id = idbase + r;
    const uint4 w0 = philox10(make_uint4(quad, id, (kTagTail << 16) | lv, 0u), key);
#pragma unroll
    for (uint32_t v = 0; v < 4u; ++v) {
      const uint32_t i = 4u * quad + v;
      if (i >= T && i < N) {
        uint32_t xv;
        if (!draw_first_word(pick_word(w0, v), i + 1u, xv))
          xv = draw_continue(key, kTagTail, lv, id, i, i + 1u);
        c.mv[koff + (i - T)] = static_cast<uint16_t>(xv);
      }
    }
  }
}

// named barrier 1 among the nthreads threads of the warps that build a level's control data
__device__ __forceinline__ void control_barrier(uint32_t nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Eight warps per tile, in three roles that rotate from tile to tile (the warps of a CTA sit on
// different SM sub-partitions, which would otherwise carry unequal loads): all of them make the
// Fisher-Yates draws and the interleaves; the data warp runs the serial parts (Algorithm 1's
// swaps, the merge tails) while the control warp builds the next level's coins, prefixes and
// break steps and the other warps join it for the tail draws.
constexpr uint32_t kTileWarps = 8;
constexpr uint32_t kTileThreads = 32u * kTileWarps;
constexpr uint32_t kTileMinBlocks = kTileWarps == 4u ? 5u : 4u;  // CTAs an SM the registers allow
// queued second-word Fisher-Yates draws per thread and block group (4 KB of queues in all)
constexpr uint32_t kFailPerThread = 32u / kTileWarps;

template <typename E, bool kPerm>
__global__ void __launch_bounds__(kTileThreads, kTileMinBlocks) tile_kernel(TileArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t boff[(1u << kTileMaxDepth) + 1u];
  __shared__ uint32_t ctlm[2][kTileCtlWords];
  __shared__ uint32_t s_S[kTileMaxDepth];  // (a.S indexed by level, without a local copy)
  uint16_t *const bufA = reinterpret_cast<uint16_t *>(smem_raw);
  uint16_t *const bufB = bufA + a.buf;
  uint2 *const cz0 = reinterpret_cast<uint2 *>(bufB + a.buf);
  uint16_t *const mv0 = reinterpret_cast<uint16_t *>(cz0 + a.wcap);
  auto ctl = [&](uint32_t set) {
    LevelCtl c;
    c.cz = cz0;
    c.mv = mv0 + set * a.tcap;
    c.m = &ctlm[0][0] + set * kTileCtlWords;
    return c;
  };
  // per-thread queues of second-word Fisher-Yates draws (aliased with the tail draws)
  uint32_t *const flist = reinterpret_cast<uint32_t *>(mv0);
  const uint32_t tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const uint32_t warp = tid >> 5;
  const uint32_t nb = 1u << a.d;
  const uint64_t tiles = (1ull << a.c) >> a.d;
  if (tid < kTileMaxDepth) {
#pragma unroll
    for (uint32_t l = 0; l < kTileMaxDepth; ++l)
      if (tid == l) s_S[l] = a.S[l];
  }
  __syncthreads();

  for (uint64_t tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
    const uint64_t k0 = tt << a.d;
    const uint64_t g0 = boundary(a.n, a.c, k0);
    for (uint32_t k = tid; k <= nb; k += kTileThreads)
      boff[k] = static_cast<uint32_t>(boundary(a.n, a.c, k0 + k) - g0);
    // roles of this tile: 0 data, 1 control, 2 and 3 helpers
    const uint32_t role = (warp - static_cast<uint32_t>(tt)) & (kTileWarps - 1u);
    __syncthreads();

    // ---- Algorithm 1's draws (warp w: quads w, w + kTileWarps, ... of every block; lane: the
    // block)
    for (uint32_t kg = 0; kg < nb; kg += 32u) {
      const uint32_t k = kg + lane;
      const bool act = k < nb;
      const uint32_t off = act ? boff[k] : 0u;
      const uint32_t L = act ? boff[k + 1u] - off : 0u;
      uint16_t *const A = bufA + k * a.P;
      uint16_t *const D = bufB + k * a.P;  // D[i]: the draw of position i
      uint32_t *const F = flist + tid * kFailPerThread;
      const uint32_t id = static_cast<uint32_t>(k0 + k);
      const uint32_t nq = L ? ((L - 1u) >> 2) + 1u : 0u;
      uint32_t nf = 0;
#pragma unroll 2
      for (uint32_t qd = warp; qd < nq; qd += kTileWarps) {
        const uint4 blk = philox10(make_uint4(qd, id, kTagLeaf << 16, 0u), a.key);
        // slice width of the quad's ranges (positions 1..3 of quad 0 take the general draw)
        const uint32_t qb = 32u - __clz(4u * qd + 1u);  // (= bits of 4qd for qd >= 1)
        const uint32_t qmask = 0xFFFFFFFFu >> (32u - qb);
#pragma unroll
        for (uint32_t v = 0; v < 4u; ++v) {
          const uint32_t pos = 4u * qd + v;
          if (pos < L) {
            A[pos] = static_cast<uint16_t>(off + pos);
            if (pos >= 1u) {
              uint32_t x;
              const uint32_t word = pick_word(blk, v);
              const bool ok = qd ? draw_first_word_b(word, pos + 1u, qb, qmask, 2u * qb, 3u * qb, x)
                                 : draw_first_word(word, pos + 1u, x);
              if (ok) {
                D[pos] = static_cast<uint16_t>(x);
              } else if (nf < kFailPerThread) {
                F[nf++] = pos;
              } else {
                D[pos] = static_cast<uint16_t>(
                    draw_continue(a.key, kTagLeaf, 0u, id, pos, pos + 1u));
              }
            }
          }
        }
      }
      // draws whose first word rejected every slice: words 1, 2, ... of their streams
      for (uint32_t e = 0; e < nf; ++e) {
        const uint32_t pos = F[e];
        D[pos] = static_cast<uint16_t>(draw_continue(a.key, kTagLeaf, 0u, id, pos, pos + 1u));
      }
    }
    __syncthreads();

    // ---- Algorithm 1's swaps, i = L-1 .. 1 (blocks 0..31: the data warp, 32..63: a helper;
    // four steps a group, the draws clamped to the block); meanwhile the control warp builds
    // level 0's control data
    if (role == 0u || role == 2u) {
      const uint32_t k = (role == 0u ? 0u : 32u) + lane;
      const uint32_t L = k < nb ? boff[k + 1u] - boff[k] : 0u;
      uint16_t *const A = bufA + k * a.P;
      const uint16_t *const D = bufB + k * a.P;
      fy_chain16(A, D, L);
    } else {
      // the other roles (1 and 3 .. kTileWarps-1): level 0's control data (role 1), then its
      // tail draws
      const LevelCtl c0 = ctl(0u);
      if (role == 1u) level_setup(a.key, a.d, a.tcap, boff, k0, 0u, a.P, lane, c0.cz, c0.mv, c0.m);
      control_barrier((kTileWarps - 2u) * 32u);
      tail_draws(a.key, a.d, 0u, k0, (role == 1u ? 0u : role - 2u) * 32u + lane,
                 (kTileWarps - 2u) * 32u, c0.mv, c0.m);
    }
    __syncthreads();

    // ---- merge levels 0 .. d-1 of the tile (Algorithm 2)
    for (uint32_t lv = 0; lv < a.d; ++lv) {
      if constexpr (!kPerm) {
        if (lv + 1u == a.d) {
          // the tile's input rows into L2 while the last level runs: its gather then reads them
          // in a random order from L2 rather than from DRAM
          const char *const rb = static_cast<const char *>(a.in) + g0 * sizeof(E);
          const uint32_t nbytes = boff[nb] * static_cast<uint32_t>(sizeof(E));
          for (uint32_t off = tid * 128u; off < nbytes; off += kTileThreads * 128u)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(rb + off));
        }
      }
      const uint16_t *const X = (lv & 1u) ? bufB : bufA;
      uint16_t *const Y = (lv & 1u) ? bufA : bufB;
      const uint32_t Sout = s_S[lv];
      const uint32_t R = nb >> (lv + 1u);
      const LevelCtl c = ctl(lv & 1u);
      // stable interleave: a thread places positions t .. t+7 of a merge. With R >= kTileWarps
      // merges a warp takes whole merges (r = w, w + kTileWarps, ...); with fewer, kTileWarps/R
      // warps share each merge
      const uint32_t wpm = R >= kTileWarps ? 1u : kTileWarps / R;  // warps per merge
      const uint32_t rstep = kTileWarps / wpm;
      const uint32_t sw = warp % wpm;
      for (uint32_t rr = warp / wpm; rr < R; rr += rstep) {
        const uint32_t Nr = ctl_N(c)[rr], Tr = ctl_T(c)[rr], lbr = ctl_lb(c)[rr];
        // (merge rr reads its halves at 2 rr Sin and 2 rr Sin + Sin, Sin the input stride)
        const uint32_t Sin = lv ? s_S[lv - 1u] : a.P;
        const uint32_t ar = 2u * rr * Sin, br = ar + Sin;
        const uint2 *const czr = c.cz + ctl_woff(c)[rr];
        uint16_t *const Yr = Y + rr * Sout;
        for (uint32_t t0 = 256u * sw; t0 < Nr; t0 += 256u * wpm) {
          const uint32_t t = t0 + 8u * lane;
          if (t >= Nr) continue;
          const uint2 wz = czr[t >> 5];
          const uint32_t sh = t & 31u;
          const uint32_t zz = wz.y + static_cast<uint32_t>(__popc(~wz.x & low_mask(sh)));
          const uint32_t bits = wz.x >> sh;
          // (reads past a clamped index stay inside shared memory: 8 entries at most)
          uint32_t pa = min(ar + zz, a.buf);
          uint32_t pb = min(br + t - zz, a.buf);
          uint32_t v[8];
          if (t + 8u <= Tr) {
#pragma unroll
            for (uint32_t i = 0; i < 8u; ++i) {
              const uint32_t bit = (bits >> i) & 1u;
              v[i] = X[bit ? pb : pa];
              pa += bit ^ 1u;
              pb += bit;
            }
          } else {
#pragma unroll
            for (uint32_t i = 0; i < 8u; ++i) {
              const uint32_t ti = t + i;
              const uint32_t bit = (bits >> i) & 1u;
              const uint32_t src = ti < Tr ? (bit ? pb : pa) : lbr + ti;
              v[i] = ti < Nr ? X[min(src, a.buf - 1u)] : 0u;
              pa += bit ^ 1u;
              pb += bit;
            }
          }
          uint4 o;
          o.x = v[0] | (v[1] << 16);
          o.y = v[2] | (v[3] << 16);
          o.z = v[4] | (v[5] << 16);
          o.w = v[6] | (v[7] << 16);
          *reinterpret_cast<uint4 *>(Yr + t) = o;
        }
      }
      __syncthreads();
      if (role == 0u) {
        // random insertion of positions T .. N-1, in order, one lane per merge
        if (lane < R) {
          const uint32_t Tq = ctl_T(c)[lane], Nq = ctl_N(c)[lane];
          uint16_t *const Cq = Y + lane * Sout;
          if (*ctl_drawn(c)) {
            // Steps i, i+1, ... of the loop, eight at a time: position i+u is untouched until
            // step i+u (earlier steps write positions below it), so its value is loaded ahead;
            // each step's two stores then need no wait, and the stores to positions i+u come
            // last. Exact unless a step of the group targets a position an earlier step of the
            // same group finished (m in [i, i+u)), a rare case that runs the swaps in order.
            const uint16_t *const mk = c.mv + ctl_koff(c)[lane];
            uint32_t i = Tq;
            for (; i + 8u <= Nq; i += 8u) {
              uint32_t m[8];
              bool clash = false;
#pragma unroll
              for (uint32_t u = 0; u < 8u; ++u) {
                m[u] = min(static_cast<uint32_t>(mk[i + u - Tq]), i + u);
                clash |= (m[u] >= i) & (m[u] < i + u);
              }
              if (clash) {
#pragma unroll
                for (uint32_t u = 0; u < 8u; ++u) swap_smem(Cq, i + u, m[u]);
                continue;
              }
              uint16_t o[8], v[8];
#pragma unroll
              for (uint32_t u = 0; u < 8u; ++u) o[u] = Cq[i + u];
#pragma unroll
              for (uint32_t u = 0; u < 8u; ++u) {
                v[u] = Cq[m[u]];
                Cq[m[u]] = o[u];
              }
#pragma unroll
              for (uint32_t u = 0; u < 8u; ++u) Cq[i + u] = v[u];
            }
            for (; i < Nq; ++i) swap_smem(Cq, i, min(static_cast<uint32_t>(mk[i - Tq]), i));
          } else {
            const uint32_t id = static_cast<uint32_t>(k0 >> (lv + 1u)) + lane;
            DrawMemo memo;
            for (uint32_t i = Tq; i < Nq; ++i)
              swap_smem(Cq, i, draw_uniform(a.key, kTagTail, lv, id, i, i + 1u, memo));
          }
        }
      } else if (lv + 1u < a.d) {
        // every role but the data warp: level lv+1's control data (role 1), then its tail draws
        const LevelCtl cn = ctl((lv + 1u) & 1u);
        if (role == 1u)
          level_setup(a.key, a.d, a.tcap, boff, k0, lv + 1u, Sout, lane, cn.cz, cn.mv, cn.m);
        control_barrier((kTileWarps - 1u) * 32u);
        tail_draws(a.key, a.d, lv + 1u, k0, (role - 1u) * 32u + lane, (kTileWarps - 1u) * 32u,
                   cn.mv, cn.m);
      }
      __syncthreads();
    }

    // ---- the tile's result (level d-1 wrote the second buffer if d is odd, else the first)
    {
      const uint16_t *const Z = (a.d & 1u) ? bufB : bufA;
      const uint32_t Lt = boff[nb];
      if constexpr (kPerm) {
        uint32_t *const o = static_cast<uint32_t *>(a.out) + g0;
        const uint32_t gb = static_cast<uint32_t>(g0);
        uint32_t t = tid;
        if ((reinterpret_cast<uintptr_t>(o) & 15u) == 0u) {
          const uint32_t n4 = Lt >> 2;
          for (uint32_t c4 = tid; c4 < n4; c4 += kTileThreads) {
            const uint2 pr = *reinterpret_cast<const uint2 *>(Z + 4u * c4);
            uint4 vv;
            vv.x = gb + (pr.x & 0xFFFFu);
            vv.y = gb + (pr.x >> 16);
            vv.z = gb + (pr.y & 0xFFFFu);
            vv.w = gb + (pr.y >> 16);
            *reinterpret_cast<uint4 *>(o + 4u * c4) = vv;
          }
          t = 4u * n4 + tid;
        }
        for (; t < Lt; t += kTileThreads) o[t] = gb + Z[t];
      } else {
        // the tile's input rows in the order of the indices: eight independent row loads per
        // thread (four of 16-byte rows) are in flight before their stores (one at a time, each
        // tile would wait out Lt / kTileThreads memory latencies in a row)
        const E *const src = static_cast<const E *>(a.in) + g0;
        E *const o = static_cast<E *>(a.out) + g0;
        constexpr uint32_t kRows = sizeof(E) >= 16u ? 4u : 8u;
        uint32_t t0 = 0;
        for (; t0 + kRows * kTileThreads <= Lt; t0 += kRows * kTileThreads) {
          E v[kRows];
#pragma unroll
          for (uint32_t u = 0; u < kRows; ++u)
            v[u] = __ldg(src + min(static_cast<uint32_t>(Z[t0 + u * kTileThreads + tid]), Lt - 1u));
#pragma unroll
          for (uint32_t u = 0; u < kRows; ++u) o[t0 + u * kTileThreads + tid] = v[u];
        }
        for (uint32_t t = t0 + tid; t < Lt; t += kTileThreads)
          o[t] = src[min(static_cast<uint32_t>(Z[t]), Lt - 1u)];
      }
    }
    __syncthreads();  // the buffers are reused by the next tile
  }
}

template <typename E, bool kPerm>
cudaError_t launch_t(const Plan &p, const void *in, void *out, uint64_t seed, cudaStream_t s) {
  TileArgs a;
  a.in = in;
  a.out = out;
  a.n = p.n;
  a.key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  a.c = p.c;
  a.d = p.d;
  a.P = p.tile_P;
  a.buf = p.tile_buf;
  a.wcap = p.tile_wcap;
  a.tcap = p.tile_tcap;
  for (uint32_t l = 0; l < kTileMaxDepth; ++l) a.S[l] = p.tile_S[l];
  auto kern = tile_kernel<E, kPerm>;
  cudaError_t err = allow_dynamic_smem(kern, p.tile_smem);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorUnknown;
  if constexpr (!kPerm) {
    // A shuffle's tile ends by reading its input rows in a random order within the tile, which
    // the L1 cache (the SM's unified memory less the shared memory of its resident CTAs) serves
    // in part: keep at least kTileMinL1 bytes of it, with as many CTAs as fit in the rest
    // (measured on GB300: at 79 KB a tile, three CTAs leave 28 KB and slow a 2^30 4-byte
    // shuffle from 39.2 to 42.0 ms; the perm reads nothing and keeps every CTA that fits).
    constexpr int kTileMinL1 = 56 * 1024;
    int sm_bytes = 0, reserved = 0;
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
            cudaSuccess ||
        cudaFuncGetAttributes(&fa, kern) != cudaSuccess)
      return cudaErrorUnknown;
    const long per_cta = static_cast<long>(p.tile_smem) + static_cast<long>(fa.sharedSizeBytes) +
                         reserved;
    long k = (static_cast<long>(sm_bytes) - kTileMinL1) / per_cta;
    if (k < 1) k = 1;
    long pct = (100 * k * per_cta + sm_bytes - 1) / sm_bytes;
    if (pct > 100) pct = 100;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                               static_cast<int>(pct));
    if (err != cudaSuccess) return err;
  }
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTileThreads, p.tile_smem);
  if (err != cudaSuccess) return err;
  const uint64_t tiles = p.q >> p.d;
  const uint64_t resident = static_cast<uint64_t>(per_sm > 0 ? per_sm : 1) * sms;
  const uint64_t grid = tiles < resident ? tiles : resident;
  if (p.prof) p.prof->begin(kKindLeaf, s);
  kern<<<static_cast<unsigned>(grid), kTileThreads, p.tile_smem, s>>>(a);
  if (p.prof) p.prof->end(s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile(const Plan &p, const void *in, void *out, bool perm, uint64_t seed,
                        cudaStream_t s) {
  if (p.d == 0 || p.d > kTileMaxDepth) return cudaErrorInvalidValue;
  if (perm) return launch_t<uint32_t, true>(p, in, out, seed, s);
  // the tile reads its input rows after computing its indices: never in place
  if (in == out) return cudaErrorInvalidValue;
  switch (p.w) {
    case 4: return launch_t<uint32_t, false>(p, in, out, seed, s);
    case 8: return launch_t<uint2, false>(p, in, out, seed, s);
    case 16: return launch_t<uint4, false>(p, in, out, seed, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace msk
