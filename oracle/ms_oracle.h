/*
 * ms_oracle.h -- CPU oracle for MergeShuffle (Bacher, Bodini, Hollender, Lumbroso,
 * "MergeShuffle: A Very Fast, Parallel Random Permutation Algorithm", arXiv 1508.03167).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg call this library. The product path (the CUDA library) never links, loads or calls it,
 * and the two share no source: this directory has its own Philox, its own merge tree and its
 * own merge procedure.
 *
 * The oracle is a plain, single-threaded restatement of the paper:
 *   - Algorithm 1 (Fisher-Yates, descending form) on each base block,
 *   - Algorithm 2 (MergeShuffle driver) with the block split of the appendix listing
 *     (q = 2^c blocks, c the smallest integer with floor(n / 2^c) <= cutoff, boundaries
 *     floor(n * i / q)),
 *   - Algorithm 3 (Merge): coin loop until one side is exhausted, then random insertion
 *     of every remaining position (the second loop of the merge, Fisher-Yates steps over the
 *     tail).
 *
 * Two merge placements are provided:
 *   MS_ORACLE_STABLE  -- the coin word interleaves the two halves in their order (output
 *                        position t takes the next unused element of the first half when coin t
 *                        is 0, of the second half when it is 1); the first half's and second
 *                        half's leftovers keep their order. Uniform by the bijection argument of
 *                        the BalancedShuffle correctness lemma (Section 3.2) and by the Merge
 *                        lemma's conditioning argument (Section 2.1). This is the definition the
 *                        GPU path reproduces bit for bit.
 *   MS_ORACLE_LITERAL -- Algorithm 3 exactly as printed: in-place swaps, which rotate the
 *                        unconsumed part of the first half. Same coins, same break step, same
 *                        tail draws, so the same number of random bits; different output.
 *
 * Random sources:
 *   MS_ORACLE_PHILOX  -- counter-based streams ("MS-Philox v1"), every coin and every uniform
 *                        draw addressed by (seed, tag, level, id, position); see ms_oracle.c.
 *   MS_ORACLE_SEQFDR  -- one sequential bit stream; uniform integers by Lumbroso's Fast Dice
 *                        Roller (Section 1, "optimal way of drawing discrete uniform
 *                        variables"). Used only to compare bit counts with Table 1.
 *   MS_ORACLE_FDR     -- the Philox streams, but every uniform draw by the Fast Dice Roller on
 *                        its own stream ("MS-Philox-FDR"); the GPU's MS_FLAG_FDR mode.
 */
#ifndef MS_ORACLE_H
#define MS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MS_ORACLE_STABLE = 0,
  MS_ORACLE_LITERAL = 1,
  MS_ORACLE_PHILOX = 0,
  MS_ORACLE_SEQFDR = 2,
  MS_ORACLE_FDR = 4, /* Philox streams, uniform draws by the Fast Dice Roller on each draw's
                        own stream (MS-Philox-FDR; coins unchanged) */
  MS_ORACLE_BALANCED = 8, /* merges driven by a balanced word: the labels merged by the coin
                             loop and insertions, then a stable interleave of the data */
  /* Planted mistakes, for tests that show the pins catch them (never used otherwise):
   * Sattolo-style off-by-one ranges in Algorithm 1 or in the merge tail, or no tail at all. */
  MS_ORACLE_PLANT_FY_RANGE = 16,
  MS_ORACLE_PLANT_TAIL_RANGE = 32,
  MS_ORACLE_PLANT_NO_TAIL = 64
};

/* Stream tags of MS-Philox v1. */
enum {
  MS_ORACLE_TAG_COIN = 1,
  MS_ORACLE_TAG_TAIL = 2,
  MS_ORACLE_TAG_LEAF = 3,
  MS_ORACLE_TAG_RS_COIN = 4, /* splitting process: the bit of position p on level l */
  MS_ORACLE_TAG_RS_LEAF = 5  /* splitting process: Fisher-Yates of the final segment at s */
};

typedef struct {
  uint64_t coin_bits;   /* flips drawn by all coin loops, terminating flips included */
  uint64_t leaf_bits;   /* bits consumed by the Fisher-Yates draws of the base blocks */
  uint64_t tail_bits;   /* bits consumed by the random insertions that finish each merge */
  uint64_t leaf_draws;  /* number of uniform draws with range > 1 in the base blocks */
  uint64_t tail_draws;  /* number of uniform draws with range > 1 in merge tails */
  uint64_t merges;      /* number of Merge calls */
  uint64_t leftover;    /* sum over merges of N - T (positions placed by random insertion) */
  uint64_t levels;      /* c */
} ms_oracle_stats;

/* Philox4x32-10 block function (Salmon, Moraes, Dror, Shaw, SC'11). */
void ms_oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Coin t of merge (level, id) under seed: 0 takes from the first half, 1 from the second. */
int ms_oracle_coin(uint64_t seed, uint32_t level, uint32_t id, uint64_t t);

/* Uniform integer in [0, R) of stream (tag, level, id, pos); *bits receives the bits used. */
uint64_t ms_oracle_draw(uint64_t seed, uint32_t tag, uint32_t level, uint32_t id, uint64_t pos,
                        uint64_t R, uint64_t *bits);

/* The same draw by the Fast Dice Roller on the draw's own stream (mode MS_ORACLE_FDR). */
uint64_t ms_oracle_draw_fdr(uint64_t seed, uint32_t tag, uint32_t level, uint32_t id,
                            uint64_t pos, uint64_t R, uint64_t *bits);

/* Number of base-block levels c for n elements and cutoff B (B >= 1). */
uint32_t ms_oracle_levels(uint64_t n, uint32_t B);

/* Permute n elements of w bytes (w in 1..64) in place. Returns 0 on success. */
int ms_oracle_shuffle(void *data, uint64_t n, uint32_t w, uint64_t seed, uint32_t B, int mode,
                      ms_oracle_stats *st);

/* Fill out[0..n) with the permutation MergeShuffle applies to the identity. */
int ms_oracle_perm(uint32_t *out, uint64_t n, uint64_t seed, uint32_t B, int mode,
                   ms_oracle_stats *st);

/* The Rao-Sandelius splitting process with a Fisher-Yates cutoff B (see ms_oracle.c): segments
 * above B split stably by one fresh bit per element and level (stream RS_COIN) until every
 * segment has at most B elements, then each segment [s, e) is shuffled by Algorithm 1 with the
 * draws of stream (RS_LEAF, 0, s, i). Stats: coin_bits = bits drawn by the splits, merges = the
 * number of splits, levels = split levels, leaf_* = the Fisher-Yates draws. mode: MS_ORACLE_PHILOX
 * or MS_ORACLE_SEQFDR (one sequential stream, Fast Dice Roller draws; bit counts only).
 * Returns 0 on success. */
int ms_oracle_rs_shuffle(void *data, uint64_t n, uint32_t w, uint64_t seed, uint32_t B, int mode,
                         ms_oracle_stats *st);
int ms_oracle_rs_perm(uint32_t *out, uint64_t n, uint64_t seed, uint32_t B, int mode,
                      ms_oracle_stats *st);

/* One Merge of the adjacent ranges a[0..n1) and a[n1..n1+n2), as merge `id` of `level`.
 * *T_out receives the break step (number of flips before the terminating one). */
int ms_oracle_merge(uint32_t *a, uint64_t n1, uint64_t n2, uint64_t seed, uint32_t level,
                    uint32_t id, int mode, uint64_t *T_out, ms_oracle_stats *st);

/* Exhaustive walk of every coin and draw outcome (exact probabilities; rejection collapsed to
 * an exact 1/R choice) of MergeShuffle on the identity of size n <= 8 with cutoff B.
 * num[2*rank], num[2*rank+1] receive the high and low 64 bits of the probability numerator
 * of the output permutation with Lehmer rank `rank`, over the common denominator returned in
 * den[0] (high), den[1] (low). *paths receives the number of decision-tree leaves.
 * Returns 0 on success, nonzero if the tree is deeper than the walker supports. */
int ms_oracle_enumerate(uint32_t n, uint32_t B, int mode, uint64_t *num, uint64_t *den,
                        uint64_t *paths);

/* Same walk for one Merge of a first half of size a and a second half of size b (a+b <= 10),
 * inputs in their given order: num[2*mask..] accumulates the probability that the set of output
 * positions holding first-half elements is `mask`. */
int ms_oracle_enumerate_merge(uint32_t a, uint32_t b, int mode, uint64_t *num, uint64_t *den,
                              uint64_t *paths);

/* Exhaustive walk of the splitting process on the identity of size n <= 6, cut at max_levels
 * split levels: num[2*rank..] receives the probability numerator of each output permutation over
 * paths that finish within max_levels levels, unres[0..1] the numerator of the paths cut off
 * (high, low), den the common denominator. mode: 0, or MS_ORACLE_PLANT_FY_RANGE (tests only). */
int ms_oracle_enumerate_rs(uint32_t n, uint32_t B, uint32_t max_levels, int mode, uint64_t *num,
                           uint64_t *den, uint64_t *paths, uint64_t *unres);

#ifdef __cplusplus
}
#endif
#endif
