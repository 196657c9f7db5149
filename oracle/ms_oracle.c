/*
 * ms_oracle.c -- CPU oracle for MergeShuffle (arXiv 1508.03167). TEST INFRASTRUCTURE ONLY:
 * the test suite, the smoke check and the benchmark's CPU-baseline leg are its only callers.
 *
 * Plain, single-threaded, element by element. Each function names the passage it restates.
 * Nothing here is blocked, fused or reordered beyond what the paper's algorithms state; the
 * only convenience is that a random source remembers the last Philox block it computed (a
 * pure function of its counter and key), which changes no result.
 *
 * ---------------------------------------------------------------------------------------
 * MS-Philox v1: the counter-based streams (project definition; the paper leaves random_bit()
 * and random_int() unspecified -- Section 1 only says that uniform integers should be drawn
 * bit-economically).
 *   key      = (lo32(seed), hi32(seed))
 *   COIN     : coin t of merge `id` on level `level` is bit (t mod 32) of word ((t / 32) mod 4)
 *              of Philox(ctr = (t / 128, id, (1 << 16) | level, 0)).
 *   UNIFORM  : a draw in [0, R) for stream (tag, level, id, pos), R >= 2, with b = ceil(log2 R)
 *              bits per attempt and k = floor(32 / b) attempts per 32-bit word.
 *              Word j (j = 0, 1, ...) is word (pos mod 4) of
 *              Philox(ctr = (pos / 4, id, (tag << 16) | level, j)); attempt u of that word is
 *              bits [u*b, u*b + b). The first attempt below R is the value (rejection sampling).
 *              R = 1 draws nothing and returns 0.
 *   tags     : TAIL (2) for the random insertions of merge `id` on `level` (pos = position in
 *              the merged range); LEAF (3) for the Fisher-Yates draws of base block `id`
 *              (level 0, pos = the index i of Algorithm 1).
 *   splitting process (Rao-Sandelius, below): RS_COIN (4), the bit of position p on split level
 *              l is bit (p mod 32) of word ((p / 32) mod 4) of Philox((p / 128, 0, (4 << 16) | l,
 *              0)); RS_LEAF (5), the Fisher-Yates draws of the final segment starting at s
 *              (level 0, id = s, pos = i).
 * ---------------------------------------------------------------------------------------
 */
#include "ms_oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ Philox4x32-10 ------- */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11), Philox
 * with N = 4 words of W = 32 bits and 10 rounds. One round: two 32x32 -> 64-bit products of
 * the even words with the multipliers, the high halves xored with the odd words and the round
 * key, the words permuted; the key advances by the Weyl constants between rounds. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void ms_oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------ random sources ------ */
typedef struct ms_src ms_src;
struct ms_src {
  int (*coin)(ms_src *s, uint32_t level, uint32_t id, uint64_t t);
  /* a coin of another stream than the merges' (the splitting process): tag, level, id, t */
  int (*tcoin)(ms_src *s, uint32_t tag, uint32_t level, uint32_t id, uint64_t t);
  uint64_t (*uniform)(ms_src *s, uint32_t tag, uint32_t level, uint32_t id, uint64_t pos,
                      uint64_t R, uint64_t *bits);
  int failed;
  int plant; /* MS_ORACLE_PLANT_* bits; 0 in every real run */
};

/* Philox source with a one-block memo. */
typedef struct {
  ms_src base;
  uint64_t seed;
  uint32_t last_ctr[4];
  uint32_t last_out[4];
  int have_last;
} philox_src;

static const uint32_t *philox_block(philox_src *p, uint32_t c0, uint32_t c1, uint32_t c2,
                                    uint32_t c3) {
  if (!(p->have_last && p->last_ctr[0] == c0 && p->last_ctr[1] == c1 && p->last_ctr[2] == c2 &&
        p->last_ctr[3] == c3)) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    ms_oracle_philox(ctr, key, p->last_out);
    memcpy(p->last_ctr, ctr, sizeof ctr);
    p->have_last = 1;
  }
  return p->last_out;
}

static int philox_coin(ms_src *s, uint32_t level, uint32_t id, uint64_t t) {
  philox_src *p = (philox_src *)s;
  const uint32_t *blk = philox_block(p, (uint32_t)(t >> 7), id,
                                     ((uint32_t)MS_ORACLE_TAG_COIN << 16) | level, 0);
  uint32_t word = blk[(t >> 5) & 3];
  return (int)((word >> (t & 31)) & 1u);
}

static int philox_tcoin(ms_src *s, uint32_t tag, uint32_t level, uint32_t id, uint64_t t) {
  philox_src *p = (philox_src *)s;
  const uint32_t *blk = philox_block(p, (uint32_t)(t >> 7), id, (tag << 16) | level, 0);
  uint32_t word = blk[(t >> 5) & 3];
  return (int)((word >> (t & 31)) & 1u);
}

/* ceil(log2 R) for R >= 2 */
static uint32_t bits_for_range(uint64_t R) {
  uint32_t b = 0;
  while (((uint64_t)1 << b) < R) ++b;
  return b;
}

static uint64_t philox_uniform(ms_src *s, uint32_t tag, uint32_t level, uint32_t id,
                               uint64_t pos, uint64_t R, uint64_t *bits) {
  philox_src *p = (philox_src *)s;
  if (R <= 1) return 0;
  uint32_t b = bits_for_range(R);
  uint32_t per_word = 32u / b;
  uint64_t mask = (b == 32) ? 0xFFFFFFFFull : (((uint64_t)1 << b) - 1);
  for (uint32_t j = 0; j < (1u << 20); ++j) {
    const uint32_t *blk =
        philox_block(p, (uint32_t)(pos >> 2), id, (tag << 16) | level, j);
    uint32_t word = blk[pos & 3];
    for (uint32_t u = 0; u < per_word; ++u) {
      uint64_t x = ((uint64_t)word >> (u * b)) & mask;
      if (bits) *bits += b;
      if (x < R) return x;
    }
  }
  s->failed = 1; /* 2^20 rejected words in a row: never expected */
  return 0;
}

/* Fast Dice Roller (Lumbroso 2013, the optimal uniform draw Section 1 cites) on each draw's own
 * stream: the bits of word j of stream (tag, level, id, pos) -- word (pos mod 4) of
 * Philox(ctr = (pos / 4, id, (tag << 16) | level, j)) -- are read least significant first,
 * j = 0, 1, ...; v doubles and c takes the next bit with each read; once v >= R, c < R is the
 * value, else c - R is uniform on [0, v - R) and the loop continues with v - R. (The coins are
 * MS-Philox v1's; only the uniform draws change.) */
static uint64_t philox_fdr_uniform(ms_src *s, uint32_t tag, uint32_t level, uint32_t id,
                                   uint64_t pos, uint64_t R, uint64_t *bits) {
  philox_src *p = (philox_src *)s;
  if (R <= 1) return 0;
  uint64_t v = 1, c = 0;
  for (uint32_t j = 0; j < (1u << 20); ++j) {
    const uint32_t *blk = philox_block(p, (uint32_t)(pos >> 2), id, (tag << 16) | level, j);
    uint32_t word = blk[pos & 3];
    for (uint32_t u = 0; u < 32; ++u) {
      v <<= 1;
      c = (c << 1) | ((word >> u) & 1u);
      if (bits) *bits += 1;
      if (v >= R) {
        if (c < R) return c;
        v -= R;
        c -= R;
      }
    }
  }
  s->failed = 1;
  return 0;
}

/* Sequential bit stream + Fast Dice Roller (Lumbroso 2013), for bit counts only. */
typedef struct {
  ms_src base;
  uint64_t seed;
  uint64_t block;   /* index of the next Philox block of the stream */
  uint32_t buf[4];
  uint32_t avail;   /* unread bits left in buf */
} seq_src;

static uint32_t seq_bit(seq_src *q) {
  if (q->avail == 0) {
    uint32_t ctr[4] = {(uint32_t)q->block, (uint32_t)(q->block >> 32), 4u << 16, 0};
    uint32_t key[2] = {(uint32_t)q->seed, (uint32_t)(q->seed >> 32)};
    ms_oracle_philox(ctr, key, q->buf);
    q->block++;
    q->avail = 128;
  }
  uint32_t idx = 128 - q->avail;
  q->avail--;
  return (q->buf[idx >> 5] >> (idx & 31)) & 1u;
}

static int seq_coin(ms_src *s, uint32_t level, uint32_t id, uint64_t t) {
  (void)level; (void)id; (void)t;
  return (int)seq_bit((seq_src *)s);
}

static int seq_tcoin(ms_src *s, uint32_t tag, uint32_t level, uint32_t id, uint64_t t) {
  (void)tag;
  return seq_coin(s, level, id, t);
}

/* Fast Dice Roller: keep c uniform on [0, v); each bit doubles v; once v >= R, return c if
 * c < R, otherwise c - R is uniform on [0, v - R) and the loop continues from there. */
static uint64_t seq_uniform(ms_src *s, uint32_t tag, uint32_t level, uint32_t id, uint64_t pos,
                            uint64_t R, uint64_t *bits) {
  (void)tag; (void)level; (void)id; (void)pos;
  if (R <= 1) return 0;
  uint64_t v = 1, c = 0;
  for (;;) {
    v <<= 1;
    c = (c << 1) | seq_bit((seq_src *)s);
    if (bits) *bits += 1;
    if (v >= R) {
      if (c < R) return c;
      v -= R;
      c -= R;
    }
  }
}

/* ------------------------------------------------------------------ merge tree ---------- */
/* The appendix listing: c is the smallest integer with floor(n / 2^c) <= cutoff; the base
 * blocks are [floor(n*i/q), floor(n*(i+1)/q)) for i < q = 2^c. */
uint32_t ms_oracle_levels(uint64_t n, uint32_t B) {
  uint32_t c = 0;
  if (B == 0) return 0;
  while ((n >> c) > (uint64_t)B) ++c;
  return c;
}

static uint64_t boundary(uint64_t n, uint32_t c, uint64_t i) {
  return (uint64_t)(((unsigned __int128)n * i) >> c);
}

/* ------------------------------------------------------------------ element access ------ */
static void swap_elems(unsigned char *a, uint64_t i, uint64_t j, uint32_t w) {
  unsigned char tmp[64];
  if (i == j) return;
  memcpy(tmp, a + i * w, w);
  memcpy(a + i * w, a + j * w, w);
  memcpy(a + j * w, tmp, w);
}

/* ------------------------------------------------------------------ Algorithm 1 --------- */
/* Fisher-Yates, Durstenfeld's descending form: for i = n-1 down to 0, j uniform in {0..i},
 * swap T[i] and T[j]. The i = 0 step has range 1 and draws nothing. */
static void fisher_yates(ms_src *src, unsigned char *a, uint64_t len, uint32_t w, uint32_t leaf,
                         ms_oracle_stats *st) {
  for (uint64_t i = len; i-- > 1;) {
    uint64_t bits = 0;
    uint64_t R = (src->plant & MS_ORACLE_PLANT_FY_RANGE) ? i : i + 1;
    uint64_t j = src->uniform(src, MS_ORACLE_TAG_LEAF, 0, leaf, i, R, &bits);
    st->leaf_bits += bits;
    st->leaf_draws += 1;
    swap_elems(a, i, j, w);
  }
}

/* ------------------------------------------------------------------ Algorithm 3 --------- */
/* Random insertion that finishes every merge ("one list is depleted; use Fisher-Yates to finish
 * merging"): for i = T .. N-1, m uniform in {0..i}, swap C[i] and C[m]. */
static void merge_tail(ms_src *src, unsigned char *c, uint64_t T, uint64_t N, uint32_t w,
                       uint32_t level, uint32_t id, ms_oracle_stats *st) {
  if (src->plant & MS_ORACLE_PLANT_NO_TAIL) return;
  for (uint64_t i = T; i < N; ++i) {
    uint64_t bits = 0;
    uint64_t R = (src->plant & MS_ORACLE_PLANT_TAIL_RANGE) && i > 0 ? i : i + 1;
    uint64_t m = src->uniform(src, MS_ORACLE_TAG_TAIL, level, id, i, R, &bits);
    st->tail_bits += bits;
    if (i + 1 > 1) st->tail_draws += 1;
    swap_elems(c, i, m, w);
  }
}

/* Stable placement. Coin t = 0 takes the next unused element of the first half A, coin 1 the
 * next unused element of the second half B; the loop stops at the first coin that asks for an
 * element of an exhausted half (that flip is drawn and counted). The remaining elements of the
 * other half follow in order, then the random insertion runs over positions T..N-1. */
static uint64_t merge_stable(ms_src *src, const unsigned char *A, uint64_t n1,
                             const unsigned char *Bh, uint64_t n2, unsigned char *out,
                             uint32_t w, uint32_t level, uint32_t id, ms_oracle_stats *st) {
  uint64_t z = 0, o = 0, t = 0;
  for (;;) {
    int bit = src->coin(src, level, id, t);
    if (bit == 0) {
      if (z == n1) break;
      memcpy(out + t * w, A + z * w, w);
      ++z;
    } else {
      if (o == n2) break;
      memcpy(out + t * w, Bh + o * w, w);
      ++o;
    }
    ++t;
  }
  uint64_t T = t;
  st->coin_bits += T + 1;
  while (z < n1) { memcpy(out + t * w, A + z * w, w); ++z; ++t; }
  while (o < n2) { memcpy(out + t * w, Bh + o * w, w); ++o; ++t; }
  merge_tail(src, out, T, n1 + n2, w, level, id, st);
  st->merges += 1;
  st->leftover += n1 + n2 - T;
  return T;
}

/* Algorithm 3 as printed (in place): i walks the output, j the second half; a 1-coin swaps
 * T[i] with T[j] and advances j; either way i advances unless the requested half is empty. */
static uint64_t merge_literal(ms_src *src, unsigned char *a, uint64_t n1, uint64_t n2,
                              uint32_t w, uint32_t level, uint32_t id, ms_oracle_stats *st) {
  uint64_t i = 0, j = n1, n = n1 + n2, t = 0;
  for (;;) {
    int bit = src->coin(src, level, id, t);
    if (bit == 0) {
      if (i == j) break;
    } else {
      if (j == n) break;
      swap_elems(a, i, j, w);
      ++j;
    }
    ++i;
    ++t;
  }
  uint64_t T = t; /* == i */
  st->coin_bits += T + 1;
  merge_tail(src, a, T, n, w, level, id, st);
  st->merges += 1;
  st->leftover += n - T;
  return T;
}

/* Merge driven by a balanced word (Section 3's idea; its correctness lemma: a uniform word in
 * C(n1 + n2, n1) interleaving two uniformly shuffled lists gives a uniform permutation). The
 * word: the labels (0 for the first half, 1 for the second) merged by this merge's own coin loop
 * and random insertions -- uniform over C(N, n1) by the Merge lemma, drawn from the same
 * streams as the stable merge, with the same bits. The data is then interleaved stably by the
 * word: no insertion moves an element. */
static uint64_t merge_balanced(ms_src *src, const unsigned char *A, uint64_t n1,
                               const unsigned char *Bh, uint64_t n2, unsigned char *out,
                               uint32_t w, uint32_t level, uint32_t id, ms_oracle_stats *st) {
  uint64_t N = n1 + n2;
  unsigned char *lab = (unsigned char *)calloc(2 * N + 2, 1);
  if (!lab) { src->failed = 1; return 0; }
  unsigned char *word = lab + N + 1;
  for (uint64_t i = 0; i < N; ++i) lab[i] = i < n1 ? 0 : 1;
  uint64_t T = merge_stable(src, lab, n1, lab + n1, n2, word, 1, level, id, st);
  uint64_t z = 0, o = 0;
  for (uint64_t t = 0; t < N; ++t) {
    if (word[t] == 0) memcpy(out + t * w, A + (z++) * w, w);
    else memcpy(out + t * w, Bh + (o++) * w, w);
  }
  free(lab);
  return T;
}

/* ------------------------------------------------------------------ Algorithm 2 --------- */
/* Split into q = 2^c blocks, Fisher-Yates each block, then merge adjacent blocks level by level:
 * on level l (p = 2^l) merge r joins [b(2pr), b(2pr+p)) and [b(2pr+p), b(2pr+2p)). */
static int run_mergeshuffle(ms_src *src, unsigned char *data, uint64_t n, uint32_t w, uint32_t B,
                            int literal, ms_oracle_stats *st, int balanced) {
  if (n <= 1) return 0;
  uint32_t c = ms_oracle_levels(n, B);
  uint64_t q = (uint64_t)1 << c;
  st->levels = c;
  for (uint64_t k = 0; k < q; ++k) {
    uint64_t s = boundary(n, c, k), e = boundary(n, c, k + 1);
    fisher_yates(src, data + s * w, e - s, w, (uint32_t)k, st);
  }
  if (literal) {
    for (uint32_t level = 0; level < c; ++level) {
      uint64_t p = (uint64_t)1 << level;
      for (uint64_t r = 0; r < (q >> (level + 1)); ++r) {
        uint64_t s = boundary(n, c, 2 * p * r);
        uint64_t mid = boundary(n, c, 2 * p * r + p);
        uint64_t e = boundary(n, c, 2 * p * r + 2 * p);
        merge_literal(src, data + s * w, mid - s, e - mid, w, level, (uint32_t)r, st);
      }
    }
    return src->failed ? 1 : 0;
  }
  unsigned char *other = NULL;
  if (c > 0) {
    other = (unsigned char *)malloc(n * w);
    if (!other) return 2;
  }
  unsigned char *cur = data, *nxt = other;
  for (uint32_t level = 0; level < c; ++level) {
    uint64_t p = (uint64_t)1 << level;
    for (uint64_t r = 0; r < (q >> (level + 1)); ++r) {
      uint64_t s = boundary(n, c, 2 * p * r);
      uint64_t mid = boundary(n, c, 2 * p * r + p);
      uint64_t e = boundary(n, c, 2 * p * r + 2 * p);
      if (balanced)
        merge_balanced(src, cur + s * w, mid - s, cur + mid * w, e - mid, nxt + s * w, w, level,
                       (uint32_t)r, st);
      else
        merge_stable(src, cur + s * w, mid - s, cur + mid * w, e - mid, nxt + s * w, w, level,
                     (uint32_t)r, st);
    }
    unsigned char *t = cur; cur = nxt; nxt = t;
  }
  if (cur != data) memcpy(data, cur, n * w);
  free(other);
  return src->failed ? 1 : 0;
}

/* ------------------------------------------------------------------ splitting process --- */
/* The Rao-Sandelius splitting process (the introduction's passage on splitting processes, after
 * Flajolet et al.; Table 1's third row), with R = 2 parts and a Fisher-Yates cutoff B (the
 * paper names the cutoff idea for MergeShuffle; here it plays the same role):
 *   start with the single segment [0, n); on level l = 0, 1, ..., every segment [s, e) with more
 *   than B elements draws one fair bit per element, the bit of its current position p
 *   (stream RS_COIN: bit p mod 32 of word (p / 32) mod 4 of Philox((p / 128, 0,
 *   (RS_COIN << 16) | l, 0))), and is split stably: the elements with bit 0 keep their order
 *   and come first, then those with bit 1. Segments of at most B elements no longer change. Once
 *   no segment has more than B elements, each segment [s, e) is shuffled by Algorithm 1 with the
 *   draws of stream (RS_LEAF, level 0, id = s, pos = i).
 * Each element draws an independent fresh bit per level while its segment splits (its position
 * is a function of earlier bits only), so the ordered partition into segments is exchangeable
 * and the shuffled segments make a uniform permutation. Levels stop after max_levels with code
 * 5 if a segment is still above B (the walk below bounds its depth that way). */
static void rs_fisher_yates(ms_src *src, unsigned char *a, uint64_t len, uint32_t w, uint32_t id,
                            ms_oracle_stats *st) {
  for (uint64_t i = len; i-- > 1;) {
    uint64_t bits = 0;
    uint64_t R = (src->plant & MS_ORACLE_PLANT_FY_RANGE) ? i : i + 1;
    uint64_t j = src->uniform(src, MS_ORACLE_TAG_RS_LEAF, 0, id, i, R, &bits);
    st->leaf_bits += bits;
    st->leaf_draws += 1;
    swap_elems(a, i, j, w);
  }
}

static int run_rao_sandelius(ms_src *src, unsigned char *data, uint64_t n, uint32_t w,
                             uint32_t B, uint32_t max_levels, ms_oracle_stats *st) {
  if (n <= 1) return 0;
  /* segment boundaries in order: seg[0] = 0 < ... < seg[count] = n (empty segments dropped) */
  uint64_t cap = 2, count = 1;
  uint64_t *seg = (uint64_t *)malloc((cap + 1) * sizeof(uint64_t));
  unsigned char *tmp = (unsigned char *)malloc(n * w);
  unsigned char *bitv = (unsigned char *)malloc(n);
  if (!seg || !tmp || !bitv) { free(seg); free(tmp); free(bitv); return 2; }
  seg[0] = 0;
  seg[1] = n;
  int rc = 0;
  for (uint32_t level = 0;; ++level) {
    int active = 0;
    for (uint64_t k = 0; k < count; ++k)
      if (seg[k + 1] - seg[k] > B) active = 1;
    if (!active) break;
    if (level >= max_levels) { rc = 5; break; }
    uint64_t *next = (uint64_t *)malloc((2 * count + 1) * sizeof(uint64_t));
    if (!next) { rc = 2; break; }
    uint64_t m = 0;
    next[m] = 0;
    for (uint64_t k = 0; k < count; ++k) {
      uint64_t s = seg[k], e = seg[k + 1];
      if (e - s > B) {
        /* stable split by the bit of each position: zeros to the front, ones after them */
        uint64_t z = 0;
        for (uint64_t p = s; p < e; ++p) {  /* each bit drawn once, in position order */
          bitv[p] = (unsigned char)src->tcoin(src, MS_ORACLE_TAG_RS_COIN, level, 0, p);
          if (bitv[p] == 0) ++z;
        }
        uint64_t zi = s, oi = s + z;
        for (uint64_t p = s; p < e; ++p)
          memcpy(tmp + (bitv[p] ? oi++ : zi++) * w, data + p * w, w);
        memcpy(data + s * w, tmp + s * w, (e - s) * w);
        st->coin_bits += e - s;
        st->merges += 1; /* splits */
        if (z > 0) next[++m] = s + z;
        if (z < e - s) next[++m] = e;
      } else {
        next[++m] = e;
      }
    }
    free(seg);
    seg = next;
    count = m;
    st->levels = level + 1;
  }
  if (rc == 0)
    for (uint64_t k = 0; k < count; ++k)
      rs_fisher_yates(src, data + seg[k] * w, seg[k + 1] - seg[k], w, (uint32_t)seg[k], st);
  free(seg);
  free(tmp);
  free(bitv);
  if (rc == 0 && src->failed) rc = 1;
  return rc;
}

static void init_philox(philox_src *p, uint64_t seed) {
  memset(p, 0, sizeof *p);
  p->base.coin = philox_coin;
  p->base.tcoin = philox_tcoin;
  p->base.uniform = philox_uniform;
  p->seed = seed;
}

static void init_seq(seq_src *q, uint64_t seed) {
  memset(q, 0, sizeof *q);
  q->base.coin = seq_coin;
  q->base.tcoin = seq_tcoin;
  q->base.uniform = seq_uniform;
  q->seed = seed;
}

/* ------------------------------------------------------------------ public entry points - */
int ms_oracle_coin(uint64_t seed, uint32_t level, uint32_t id, uint64_t t) {
  philox_src p;
  init_philox(&p, seed);
  return philox_coin(&p.base, level, id, t);
}

uint64_t ms_oracle_draw(uint64_t seed, uint32_t tag, uint32_t level, uint32_t id, uint64_t pos,
                        uint64_t R, uint64_t *bits) {
  philox_src p;
  init_philox(&p, seed);
  if (bits) *bits = 0;
  return philox_uniform(&p.base, tag, level, id, pos, R, bits);
}

uint64_t ms_oracle_draw_fdr(uint64_t seed, uint32_t tag, uint32_t level, uint32_t id,
                            uint64_t pos, uint64_t R, uint64_t *bits) {
  philox_src p;
  init_philox(&p, seed);
  if (bits) *bits = 0;
  return philox_fdr_uniform(&p.base, tag, level, id, pos, R, bits);
}

int ms_oracle_shuffle(void *data, uint64_t n, uint32_t w, uint64_t seed, uint32_t B, int mode,
                      ms_oracle_stats *st) {
  ms_oracle_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof *st);
  if (w == 0 || w > 64 || B == 0) return 3;
  if (n > 0xFFFFFFFFull) return 3;
  int literal = (mode & MS_ORACLE_LITERAL) != 0;
  if (mode & MS_ORACLE_SEQFDR) {
    seq_src q;
    init_seq(&q, seed);
    return run_mergeshuffle(&q.base, (unsigned char *)data, n, w, B, literal, st,
                            (mode & MS_ORACLE_BALANCED) != 0);
  }
  philox_src p;
  init_philox(&p, seed);
  if (mode & MS_ORACLE_FDR) p.base.uniform = philox_fdr_uniform;
  return run_mergeshuffle(&p.base, (unsigned char *)data, n, w, B, literal, st,
                          (mode & MS_ORACLE_BALANCED) != 0);
}

int ms_oracle_perm(uint32_t *out, uint64_t n, uint64_t seed, uint32_t B, int mode,
                   ms_oracle_stats *st) {
  for (uint64_t i = 0; i < n; ++i) out[i] = (uint32_t)i;
  return ms_oracle_shuffle(out, n, 4, seed, B, mode, st);
}

int ms_oracle_merge(uint32_t *a, uint64_t n1, uint64_t n2, uint64_t seed, uint32_t level,
                    uint32_t id, int mode, uint64_t *T_out, ms_oracle_stats *st) {
  ms_oracle_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof *st);
  philox_src p;
  seq_src q;
  ms_src *src;
  if (mode & MS_ORACLE_SEQFDR) { init_seq(&q, seed); src = &q.base; }
  else {
    init_philox(&p, seed);
    if (mode & MS_ORACLE_FDR) p.base.uniform = philox_fdr_uniform;
    src = &p.base;
  }
  uint64_t T;
  if (mode & MS_ORACLE_LITERAL) {
    T = merge_literal(src, (unsigned char *)a, n1, n2, 4, level, id, st);
  } else if (mode & MS_ORACLE_BALANCED) {
    uint32_t *out = (uint32_t *)malloc((n1 + n2 + 1) * sizeof(uint32_t));
    if (!out) return 2;
    T = merge_balanced(src, (unsigned char *)a, n1, (unsigned char *)(a + n1), n2,
                       (unsigned char *)out, 4, level, id, st);
    memcpy(a, out, (n1 + n2) * sizeof(uint32_t));
    free(out);
  } else {
    uint32_t *out = (uint32_t *)malloc((n1 + n2 + 1) * sizeof(uint32_t));
    if (!out) return 2;
    T = merge_stable(src, (unsigned char *)a, n1, (unsigned char *)(a + n1), n2,
                     (unsigned char *)out, 4, level, id, st);
    memcpy(a, out, (n1 + n2) * sizeof(uint32_t));
    free(out);
  }
  if (T_out) *T_out = T;
  return src->failed ? 1 : 0;
}

int ms_oracle_rs_shuffle(void *data, uint64_t n, uint32_t w, uint64_t seed, uint32_t B, int mode,
                         ms_oracle_stats *st) {
  ms_oracle_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof *st);
  if (w == 0 || w > 64 || B == 0) return 3;
  if (n > 0xFFFFFFFFull) return 3;
  if (mode & MS_ORACLE_SEQFDR) {
    seq_src q;
    init_seq(&q, seed);
    return run_rao_sandelius(&q.base, (unsigned char *)data, n, w, B, 4096, st);
  }
  philox_src p;
  init_philox(&p, seed);
  return run_rao_sandelius(&p.base, (unsigned char *)data, n, w, B, 4096, st);
}

int ms_oracle_rs_perm(uint32_t *out, uint64_t n, uint64_t seed, uint32_t B, int mode,
                      ms_oracle_stats *st) {
  for (uint64_t i = 0; i < n; ++i) out[i] = (uint32_t)i;
  return ms_oracle_rs_shuffle(out, n, 4, seed, B, mode, st);
}

/* ------------------------------------------------------------------ exhaustive walk ----- */
/* A source that, instead of drawing, walks the decision tree depth first: every coin is a
 * 2-way choice and every uniform draw an R-way choice (rejection collapsed to its exact
 * 1/R outcome). Each run follows a forced prefix of choices and takes choice 0 beyond it;
 * the odometer then advances to the next leaf. The weight of a leaf is 1 / prod(arity). */
#define ENUM_MAXD 512

typedef struct {
  ms_src base;
  uint32_t choice[ENUM_MAXD];
  uint32_t arity[ENUM_MAXD];
  uint32_t depth;   /* choices taken in the current run */
  uint32_t forced;  /* length of the forced prefix */
  unsigned __int128 prod;
  int overflow;
} enum_src;

static uint32_t enum_take(enum_src *e, uint32_t arity) {
  if (e->depth >= ENUM_MAXD) { e->overflow = 1; return 0; }
  uint32_t c;
  if (e->depth < e->forced) {
    c = e->choice[e->depth];
  } else {
    c = 0;
    e->choice[e->depth] = 0;
    e->arity[e->depth] = arity;
  }
  e->depth++;
  e->prod *= arity;
  return c;
}

static int enum_coin(ms_src *s, uint32_t level, uint32_t id, uint64_t t) {
  (void)level; (void)id; (void)t;
  return (int)enum_take((enum_src *)s, 2);
}

static int enum_tcoin(ms_src *s, uint32_t tag, uint32_t level, uint32_t id, uint64_t t) {
  (void)tag;
  return enum_coin(s, level, id, t);
}

static uint64_t enum_uniform(ms_src *s, uint32_t tag, uint32_t level, uint32_t id, uint64_t pos,
                             uint64_t R, uint64_t *bits) {
  (void)tag; (void)level; (void)id; (void)pos; (void)bits;
  if (R <= 1) return 0;
  return enum_take((enum_src *)s, (uint32_t)R);
}

/* advance the odometer; returns 0 when every leaf has been visited */
static int enum_next(enum_src *e) {
  uint32_t len = e->depth;
  while (len > 0 && e->choice[len - 1] + 1 >= e->arity[len - 1]) --len;
  if (len == 0) return 0;
  e->choice[len - 1] += 1;
  e->forced = len;
  return 1;
}

/* common denominator: 2^80 * 3^8 * 5^4 * 7^4 (every leaf weight of the supported sizes
 * divides it; checked at run time) */
static unsigned __int128 enum_denominator(void) {
  unsigned __int128 d = (unsigned __int128)1 << 80;
  for (int i = 0; i < 8; ++i) d *= 3;
  for (int i = 0; i < 4; ++i) d *= 5;
  for (int i = 0; i < 4; ++i) d *= 7;
  return d;
}

static uint64_t lehmer_rank(const uint32_t *p, uint32_t n) {
  uint64_t rank = 0;
  for (uint32_t i = 0; i < n; ++i) {
    uint64_t smaller = 0;
    for (uint32_t j = i + 1; j < n; ++j) smaller += p[j] < p[i];
    rank = rank * (n - i) + smaller;
  }
  return rank;
}

int ms_oracle_enumerate(uint32_t n, uint32_t B, int mode, uint64_t *num, uint64_t *den,
                        uint64_t *paths) {
  if (n == 0 || n > 8 || B == 0) return 3;
  uint64_t nfact = 1;
  for (uint32_t i = 2; i <= n; ++i) nfact *= i;
  unsigned __int128 D = enum_denominator();
  unsigned __int128 *acc = (unsigned __int128 *)calloc(nfact, sizeof(unsigned __int128));
  if (!acc) return 2;
  enum_src e;
  memset(&e, 0, sizeof e);
  e.base.coin = enum_coin;
  e.base.tcoin = enum_tcoin;
  e.base.uniform = enum_uniform;
  e.base.plant = mode & (MS_ORACLE_PLANT_FY_RANGE | MS_ORACLE_PLANT_TAIL_RANGE |
                         MS_ORACLE_PLANT_NO_TAIL);
  uint64_t leaves = 0;
  int rc = 0;
  for (;;) {
    uint32_t perm[8];
    ms_oracle_stats st;
    memset(&st, 0, sizeof st);
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    e.depth = 0;
    e.prod = 1;
    run_mergeshuffle(&e.base, (unsigned char *)perm, n, 4, B, (mode & MS_ORACLE_LITERAL) != 0,
                     &st, (mode & MS_ORACLE_BALANCED) != 0);
    if (e.overflow || D % e.prod != 0) { rc = 4; break; }
    acc[lehmer_rank(perm, n)] += D / e.prod;
    ++leaves;
    if (!enum_next(&e)) break;
  }
  for (uint64_t r = 0; r < nfact; ++r) {
    num[2 * r] = (uint64_t)(acc[r] >> 64);
    num[2 * r + 1] = (uint64_t)acc[r];
  }
  den[0] = (uint64_t)(D >> 64);
  den[1] = (uint64_t)D;
  if (paths) *paths = leaves;
  free(acc);
  return rc;
}

int ms_oracle_enumerate_merge(uint32_t a, uint32_t b, int mode, uint64_t *num, uint64_t *den,
                              uint64_t *paths) {
  uint32_t n = a + b;
  if (n == 0 || n > 10) return 3; /* tail ranges up to 10 keep every weight a divisor of D */
  unsigned __int128 D = enum_denominator();
  uint64_t nmask = (uint64_t)1 << n;
  unsigned __int128 *acc = (unsigned __int128 *)calloc(nmask, sizeof(unsigned __int128));
  if (!acc) return 2;
  enum_src e;
  memset(&e, 0, sizeof e);
  e.base.coin = enum_coin;
  e.base.tcoin = enum_tcoin;
  e.base.uniform = enum_uniform;
  e.base.plant = mode & (MS_ORACLE_PLANT_FY_RANGE | MS_ORACLE_PLANT_TAIL_RANGE |
                         MS_ORACLE_PLANT_NO_TAIL);
  uint64_t leaves = 0;
  int rc = 0;
  uint32_t in[10], out[10];
  for (;;) {
    ms_oracle_stats st;
    memset(&st, 0, sizeof st);
    for (uint32_t i = 0; i < n; ++i) in[i] = i;
    e.depth = 0;
    e.prod = 1;
    if (mode & MS_ORACLE_LITERAL) {
      merge_literal(&e.base, (unsigned char *)in, a, b, 4, 0, 0, &st);
      memcpy(out, in, sizeof in);
    } else if (mode & MS_ORACLE_BALANCED) {
      merge_balanced(&e.base, (unsigned char *)in, a, (unsigned char *)(in + a), b,
                     (unsigned char *)out, 4, 0, 0, &st);
    } else {
      merge_stable(&e.base, (unsigned char *)in, a, (unsigned char *)(in + a), b,
                   (unsigned char *)out, 4, 0, 0, &st);
    }
    if (e.overflow || D % e.prod != 0) { rc = 4; break; }
    uint64_t mask = 0;
    for (uint32_t i = 0; i < n; ++i)
      if (out[i] < a) mask |= (uint64_t)1 << i;
    acc[mask] += D / e.prod;
    ++leaves;
    if (!enum_next(&e)) break;
  }
  for (uint64_t r = 0; r < nmask; ++r) {
    num[2 * r] = (uint64_t)(acc[r] >> 64);
    num[2 * r + 1] = (uint64_t)acc[r];
  }
  den[0] = (uint64_t)(D >> 64);
  den[1] = (uint64_t)D;
  if (paths) *paths = leaves;
  free(acc);
  return rc;
}

/* The same walk for the splitting process, cut at max_levels levels: paths that still have a
 * segment above B after max_levels levels are not counted (their mass goes to *unres, as a
 * numerator over the same denominator). The counted mass of every permutation must be the same. */
int ms_oracle_enumerate_rs(uint32_t n, uint32_t B, uint32_t max_levels, int mode, uint64_t *num,
                           uint64_t *den, uint64_t *paths, uint64_t *unres) {
  if (n == 0 || n > 6 || B == 0) return 3;
  uint64_t nfact = 1;
  for (uint32_t i = 2; i <= n; ++i) nfact *= i;
  unsigned __int128 D = enum_denominator();
  unsigned __int128 *acc = (unsigned __int128 *)calloc(nfact, sizeof(unsigned __int128));
  if (!acc) return 2;
  unsigned __int128 lost = 0;
  enum_src e;
  memset(&e, 0, sizeof e);
  e.base.coin = enum_coin;
  e.base.tcoin = enum_tcoin;
  e.base.uniform = enum_uniform;
  e.base.plant = mode & MS_ORACLE_PLANT_FY_RANGE;
  uint64_t leaves = 0;
  int rc = 0;
  for (;;) {
    uint32_t perm[8];
    ms_oracle_stats st;
    memset(&st, 0, sizeof st);
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    e.depth = 0;
    e.prod = 1;
    int r = run_rao_sandelius(&e.base, (unsigned char *)perm, n, 4, B, max_levels, &st);
    if (e.overflow || D % e.prod != 0 || (r != 0 && r != 5)) { rc = 4; break; }
    if (r == 5) lost += D / e.prod;
    else acc[lehmer_rank(perm, n)] += D / e.prod;
    ++leaves;
    if (!enum_next(&e)) break;
  }
  for (uint64_t k = 0; k < nfact; ++k) {
    num[2 * k] = (uint64_t)(acc[k] >> 64);
    num[2 * k + 1] = (uint64_t)acc[k];
  }
  den[0] = (uint64_t)(D >> 64);
  den[1] = (uint64_t)D;
  unres[0] = (uint64_t)(lost >> 64);
  unres[1] = (uint64_t)lost;
  if (paths) *paths = leaves;
  free(acc);
  return rc;
}
