"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU needed).

Each test pins the oracle to something other than itself:
  - Philox4x32-10 against cuRAND's host generator (an independent library routine),
  - exact uniformity of the whole algorithm and of one Merge by exhaustive enumeration
    (Merge lemma, Section 2.1; bijection F, Section 3.2),
  - the break-step distribution against the sums of the bit-count lemma (Section 2.1),
  - expected random bits against those sums plus the rejection-sampling cost, and the
    n log2 n + Theta(n) law (Section 2.2),
  - Fisher-Yates with the Fast Dice Roller against the printed Table 1 row (Section 4),
  - special cases that reduce to a textbook Fisher-Yates (Algorithm 1).
"""
from __future__ import annotations

import ctypes
import ctypes.util
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats as sstats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------- Philox -------
def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if path and os.path.exists(path) if path.startswith("/") else path:
            try:
                return ctypes.CDLL(path)
            except OSError:
                continue
    return None


def _curand_host_philox(lib, seed: int, count: int) -> np.ndarray:
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(count)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 7, 0x123456789ABCDEF, 2**64 - 1])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox4x32-10 generator lays block j out at counter
    (j >> 16, 0, j & 0xffff, 0) under key (lo32(seed), hi32(seed)); every block must match."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    nblk = 65536 + 300
    got = _curand_host_philox(lib, seed, 4 * nblk).reshape(-1, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in list(range(0, 40)) + [4095, 4096, 65535, 65536, 65537, 65536 + 299]:
        want = oracle.philox([j >> 16, 0, j & 0xFFFF, 0], key)
        assert np.array_equal(got[j], want), (seed, j)


# ---------------------------------------------------------------------------- exact walks --
@pytest.mark.parametrize("mode", [oracle.STABLE, oracle.LITERAL])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_exact_uniformity_all_cutoffs(n, mode):
    """Every one of the n! outputs has probability exactly 1/n!, for every cutoff B in 1..n
    (Merge lemma, Section 2.1; induction over Algorithm 2)."""
    for B in range(1, n + 1):
        num, den, paths = oracle.enumerate_perm(n, B, mode)
        assert den % math.factorial(n) == 0
        target = den // math.factorial(n)
        assert all(x == target for x in num), (n, B, mode)
        assert sum(num) == den
        assert paths >= math.factorial(n)


@pytest.mark.parametrize("B,mode", [(2, oracle.STABLE), (3, oracle.LITERAL), (4, oracle.STABLE),
                                    (7, oracle.STABLE)])
def test_exact_uniformity_n7(B, mode):
    num, den, _ = oracle.enumerate_perm(7, B, mode)
    assert set(num) == {den // 5040}


@pytest.mark.parametrize("mode", [oracle.STABLE, oracle.LITERAL])
def test_merge_position_sets_uniform(mode):
    """For one Merge of halves of sizes a and b, the set of output positions holding
    first-half elements is uniform over all C(a+b, a) sets (Section 3.2, bijection F)."""
    for a in range(0, 6):
        for b in range(0, 6):
            if a + b == 0 or a + b > 10:
                continue
            num, den, _ = oracle.enumerate_merge(a, b, mode)
            nsets = math.comb(a + b, a)
            for mask, x in enumerate(num):
                if bin(mask).count("1") == a:
                    assert x * nsets == den, (a, b, mask)
                else:
                    assert x == 0, (a, b, mask)


@pytest.mark.parametrize("plant", [oracle.PLANT_FY_RANGE, oracle.PLANT_TAIL_RANGE,
                                   oracle.PLANT_NO_TAIL])
def test_exact_walk_catches_planted_mistakes(plant):
    """The walk is a real check: an off-by-one draw range in Algorithm 1 or in the merge tail,
    or a merge without its random insertion, makes some output's probability differ from
    1/n! (the mistakes are planted in the oracle on the CPU, behind test-only mode bits)."""
    bad = False
    for n, B in ((3, 1), (4, 2), (5, 2), (4, 4)):
        num, den, _ = oracle.enumerate_perm(n, B, oracle.STABLE | plant)
        bad |= len(set(num)) > 1
    assert bad


# ---------------------------------------------------------------------------- sampled ------
def _lehmer(p) -> int:
    n = len(p)
    r = 0
    for i in range(n):
        r = r * (n - i) + sum(1 for j in range(i + 1, n) if p[j] < p[i])
    return r


@pytest.mark.parametrize("n,B,runs", [(4, 1, 24000), (5, 2, 60000), (6, 2, 144000)])
def test_chi_square_over_consecutive_seeds(n, B, runs):
    """Philox streams over consecutive seeds: the n! outcomes are uniform (no bias from
    neighbouring keys). Chi-square at p = 1e-6."""
    counts = np.zeros(math.factorial(n), dtype=np.int64)
    for seed in range(runs):
        p, _ = oracle.perm(n, seed, B)
        counts[_lehmer(p)] += 1
    chi2, pval = sstats.chisquare(counts)
    assert pval > 1e-6, (chi2, pval)


def _break_distribution(n1: int, n2: int) -> dict:
    """P(T = t, side) from the sums of the bit-count lemma (Section 2.1): the first half runs
    out after i ones with probability C(n1+i, n1) / 2^(n1+1+i), the second symmetrically.
    side 0: first half exhausted (terminating coin 0), 1: second half; T = N counted apart."""
    N = n1 + n2
    dist = {}
    for i in range(0, n2 + 1):
        t = n1 + i
        key = ("N", None) if t == N else (t, 0)
        dist[key] = dist.get(key, Fraction(0)) + Fraction(math.comb(n1 + i, n1), 2 ** (n1 + 1 + i))
    for i in range(0, n1 + 1):
        t = n2 + i
        key = ("N", None) if t == N else (t, 1)
        dist[key] = dist.get(key, Fraction(0)) + Fraction(math.comb(n2 + i, n2), 2 ** (n2 + 1 + i))
    return dist


@pytest.mark.parametrize("n1,n2", [(16, 16), (20, 9), (5, 27), (1, 1)])
def test_break_step_distribution(n1, n2):
    dist = _break_distribution(n1, n2)
    assert sum(dist.values()) == 1
    runs = 40000
    N = n1 + n2
    obs = {}
    vals = np.arange(N, dtype=np.uint32)
    for seed in range(runs):
        _, T, st = oracle.merge(vals, n1, seed, level=3, merge_id=seed % 97)
        assert st.coin_bits == T + 1
        if T == N:
            key = ("N", None)
        else:
            key = (T, oracle.coin(seed, 3, seed % 97, T))
        obs[key] = obs.get(key, 0) + 1
    assert set(obs) <= set(dist)
    # pool sparse cells
    exp, got, pool_e, pool_o = [], [], 0.0, 0
    for key, p in dist.items():
        e = float(p) * runs
        if e < 20:
            pool_e += e
            pool_o += obs.get(key, 0)
        else:
            exp.append(e)
            got.append(obs.get(key, 0))
    if pool_e > 0:
        exp.append(pool_e)
        got.append(pool_o)
    exp = np.array(exp) * (runs / sum(exp))
    chi2, pval = sstats.chisquare(got, exp)
    assert pval > 1e-6, (chi2, pval)


def test_mean_leftover_matches_sqrt_law():
    """E[N - T] for a balanced merge of N = 2^10, from the same sums: close to sqrt(2N/pi)
    (about 25), and the oracle's mean over seeds agrees within 5 sigma."""
    n1 = n2 = 512
    N = 1024
    dist = _break_distribution(n1, n2)
    mean = sum(float(p) * (N - (N if k[0] == "N" else k[0])) for k, p in dist.items())
    assert abs(mean - math.sqrt(2 * N / math.pi)) < 1.5
    vals = np.arange(N, dtype=np.uint32)
    left = [N - oracle.merge(vals, n1, s)[1] for s in range(3000)]
    se = np.std(left) / math.sqrt(len(left))
    assert abs(np.mean(left) - mean) < 5 * se


# ---------------------------------------------------------------------------- bits ---------
def _bits_per_draw(R: int) -> float:
    """Expected bits of one rejection-sampled draw with b = ceil(log2 R) bits per attempt."""
    if R <= 1:
        return 0.0
    b = (R - 1).bit_length()
    return b * (2 ** b) / R


def _expected_total_bits(n: int, B: int) -> float:
    c = 0
    while (n >> c) > B:
        c += 1
    q = 1 << c
    bnd = [(n * i) >> c for i in range(q + 1)]
    fy = [0.0]
    for R in range(2, B + 3):
        fy.append(fy[-1] + _bits_per_draw(R))
    total = 0.0
    for k in range(q):
        L = bnd[k + 1] - bnd[k]
        total += fy[L - 1] if L >= 2 else 0.0
    for level in range(c):
        p = 1 << level
        for r in range(q >> (level + 1)):
            s, mid, e = bnd[2 * p * r], bnd[2 * p * r + p], bnd[2 * p * r + 2 * p]
            n1, n2 = mid - s, e - mid
            N = n1 + n2
            suffix = [0.0] * (N + 2)  # suffix[T] = sum_{i=T}^{N-1} bits(i+1)
            for i in range(N - 1, -1, -1):
                suffix[i] = suffix[i + 1] + _bits_per_draw(i + 1)
            for key, pr in _break_distribution(n1, n2).items():
                T = N if key[0] == "N" else key[0]
                total += float(pr) * (T + 1 + suffix[T])
    return total


@pytest.mark.parametrize("n,B", [(300, 7), (1000, 64), (4133, 64)])
def test_expected_bits_consumed(n, B):
    want = _expected_total_bits(n, B)
    got = []
    for seed in range(400):
        _, st = oracle.perm(n, seed, B)
        got.append(st.total_bits)
    got = np.array(got, dtype=float)
    se = got.std() / math.sqrt(len(got))
    assert abs(got.mean() - want) < 5 * se + 1e-9, (got.mean(), want, se)


def test_bits_are_n_log_n_plus_linear():
    """(bits - n log2 n) / n stays bounded as n grows (Section 2.2)."""
    ratios = []
    for k in (10, 13, 16, 18):
        n = 1 << k
        _, st = oracle.perm(n, 11, 32)
        ratios.append((st.total_bits - n * k) / n)
    assert all(0.0 < r < 4.0 for r in ratios), ratios
    assert max(ratios) - min(ratios) < 0.5, ratios


def test_fisher_yates_bits_cross_check():
    """A single block (n <= B) is plain Fisher-Yates: its mean bit count matches the sum of the
    per-draw expectations."""
    n = 1500
    want = sum(_bits_per_draw(R) for R in range(2, n + 1))
    got = np.array([oracle.perm(n, s, n)[1].leaf_bits for s in range(300)], dtype=float)
    assert abs(got.mean() - want) < 5 * got.std() / math.sqrt(len(got))


def _table1():
    rows = {}
    with open(os.path.join(GOLDEN, "table1_random_bits.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, n, bits = line.split()
            rows[(name, int(n))] = int(bits)
    return rows


@pytest.mark.parametrize("n,trials", [(100000, 100), (1000000, 12)])
def test_table1_fisher_yates_row(n, trials):
    """Fisher-Yates with Lumbroso's draws (Table 1, first row): the oracle's mean bit count
    agrees with the printed 100-trial mean within the combined sampling error."""
    paper = _table1()[("fisher_yates", n)]
    got = np.array([oracle.perm(n, s, n, oracle.SEQFDR)[1].leaf_bits for s in range(trials)],
                   dtype=float)
    sd = got.std()
    se = math.sqrt(sd ** 2 / trials + sd ** 2 / 100)
    assert abs(got.mean() - paper) < 4.5 * se, (got.mean(), paper, se)


# ---------------------------------------------------------------------------- structure ----
@pytest.mark.parametrize("n", [2, 17, 1024])
def test_single_block_is_textbook_fisher_yates(n):
    """n <= B: no merge; the result is Algorithm 1 driven by the LEAF stream of block 0."""
    seed = 99
    got, st = oracle.perm(n, seed, B=n)
    assert st.merges == 0 and st.levels == 0
    a = list(range(n))
    for i in range(n - 1, 0, -1):
        j, _ = oracle.draw(seed, oracle.TAG_LEAF, 0, 0, i, i + 1)
        a[i], a[j] = a[j], a[i]
    assert got.tolist() == a


def test_two_elements_one_merge():
    """n = 2, B = 1: two one-element blocks and one Merge, worked by hand from Algorithm 3:
    the first coin picks which element leads; the second either takes the other element
    (no tail) or breaks, leaving one element for the random insertion at position 1."""
    for seed in range(200):
        p, st = oracle.perm(2, seed, 1)
        c0 = oracle.coin(seed, 0, 0, 0)
        c1 = oracle.coin(seed, 0, 0, 1)
        if c0 == 0:
            out, T = [0], 1
            if c1 == 1:
                out, T = [0, 1], 2
        else:
            out, T = [1], 1
            if c1 == 0:
                out, T = [1, 0], 2
        rest = [x for x in (0, 1) if x not in out]
        out = out + rest
        for i in range(T, 2):
            m, _ = oracle.draw(seed, oracle.TAG_TAIL, 0, 0, i, i + 1)
            out[i], out[m] = out[m], out[i]
        assert p.tolist() == out, seed


@pytest.mark.parametrize("n,B", [(1, 1), (5, 1), (1000, 7), (4099, 64), (70000, 1024)])
def test_output_is_permutation_and_modes_share_bits(n, B):
    a, sa = oracle.perm(n, 3, B, oracle.STABLE)
    b, sb = oracle.perm(n, 3, B, oracle.LITERAL)
    assert np.array_equal(np.sort(a), np.arange(n))
    assert np.array_equal(np.sort(b), np.arange(n))
    assert sa.as_dict() == sb.as_dict()  # same coins, same T, same tail draws


def test_shuffle_is_data_oblivious():
    """shuffle(X) = X[perm(n)] for records of any width (the decisions never look at data)."""
    n, B, seed = 5003, 32, 21
    rng = np.random.default_rng(0)
    rec = rng.integers(0, 2**63, size=(n, 2), dtype=np.uint64)
    got, _ = oracle.shuffle(rec, seed, B)
    p, _ = oracle.perm(n, seed, B)
    assert np.array_equal(got, rec[p])


def test_cutoff_rule_follows_listing():
    """c is the smallest integer with floor(n / 2^c) <= B (appendix listing)."""
    assert oracle.levels(2**20, 1024) == 10
    assert oracle.levels(2049, 1024) == 1
    assert oracle.levels(2048, 1024) == 1
    assert oracle.levels(1024, 1024) == 0
    assert oracle.levels(300_000_017, 1024) == 19
    assert oracle.levels(2**30, 1024) == 20
