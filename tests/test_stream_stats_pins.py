"""Pins for the oracle's parallel-stream statistics (oracle/stream_stats.py).

The statistics are plain definitions (Knuth, TAOCP vol. 2, §3.3.2), so they
are pinned by:
  * brute-force Python loops on tiny inputs (tuples, gaps, spacings);
  * hand-worked examples with known counts;
  * the stream fed in pieces giving the same gap counts as in one piece;
  * their known distributions on words from numpy's PCG64 (independent of
    every generator under test): uniform cells, geometric gaps, and birthday
    spacings with mean close to lambda = n^3 / (4 m);
  * planted mistakes that the tests must catch: micro-streams that ignore
    the particle id (every particle draws the same words), and a stream
    whose low bit alternates.
And the concatenated micro-stream layout is pinned to the oracle's already
pinned per-stream words.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import stream_stats as S

PCG = np.random.default_rng(20231030)


def pcg_words(n, rng=None):
    return (rng or PCG).integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)


# ------------------------------------------------------------- tuples ----

def brute_tuples(words, t, bits, shift, stride):
    counts = [0] * (1 << (t * bits))
    m = 0
    while m * stride + t <= len(words):
        cell = 0
        for i in range(t):
            cell = (cell << bits) | ((int(words[m * stride + i]) >> shift) & ((1 << bits) - 1))
        counts[cell] += 1
        m += 1
    return np.array(counts, np.uint64)


@pytest.mark.parametrize("n,t,bits,shift,stride", [(0, 1, 8, 24, 1), (2, 3, 4, 28, 3), (97, 1, 8, 24, 1),
                                                   (97, 2, 6, 26, 2), (101, 3, 4, 0, 3), (50, 2, 3, 5, 1)])
def test_tuples_match_brute_force(n, t, bits, shift, stride):
    w = pcg_words(n)
    assert np.array_equal(S.tuple_counts(w, t, bits, shift, stride), brute_tuples(w, t, bits, shift, stride))


def test_tuples_hand_example():
    w = np.array([0x00000000, 0xFFFFFFFF, 0x80000000, 0x7FFFFFFF], np.uint32)
    assert S.tuple_counts(w, 1, 1, 31, 1).tolist() == [2, 2]
    # pairs (0,1), (1,0): cells 0b01 and 0b10
    assert S.tuple_counts(w, 2, 1, 31, 2).tolist() == [0, 1, 1, 0]
    # overlapping pairs (0,1), (1,1), (1,0)
    assert S.tuple_counts(w, 2, 1, 31, 1).tolist() == [0, 1, 1, 1]
    # low byte: 0x00, 0xFF, 0x00, 0xFF
    c = S.tuple_counts(w, 1, 8, 0, 1)
    assert c[0] == 2 and c[255] == 2 and c.sum() == 4


def test_tuples_uniform_on_pcg64():
    c = S.tuple_counts(pcg_words(3 << 18), 3, 4, 28, 3)
    assert stats.chisquare(c.astype(float)).pvalue > 1e-4


# --------------------------------------------------------------- gaps ----

def brute_gaps(words, lo, hi, t_max):
    counts = [0] * (t_max + 1)
    last = None
    for i, x in enumerate(words):
        if lo <= int(x) < hi:
            if last is not None:
                counts[min(i - last - 1, t_max)] += 1
            last = i
    return np.array(counts, np.uint64)


def test_gaps_hand_example():
    # hits at 0, 3, 5, 6: gaps 2, 1, 0
    w = np.array([0, 5, 5, 0, 5, 0, 0], np.uint32)
    c, carry = S.gap_counts(w, 0, 1, 4)
    assert c.tolist() == [1, 1, 1, 0, 0] and carry == 0
    # a trailing run of non-hits becomes the carry
    c, carry = S.gap_counts(np.array([7, 0, 7, 7], np.uint32), 0, 1, 4)
    assert c.sum() == 0 and carry == 2
    # no hit at all: the carry stays "no hit yet"
    c, carry = S.gap_counts(np.array([7, 7], np.uint32), 0, 1, 4)
    assert c.sum() == 0 and carry is None


@pytest.mark.parametrize("lo,hi,t_max", [(0, 1 << 28, 40), (3 << 30, 1 << 32, 8), (12345, 12345 + (1 << 27), 100)])
def test_gaps_match_brute_force(lo, hi, t_max):
    w = pcg_words(3000)
    c, _ = S.gap_counts(w, lo, hi, t_max)
    assert np.array_equal(c, brute_gaps(w, lo, hi, t_max))


def test_gaps_in_pieces_equal_one_piece():
    w = pcg_words(5000)
    lo, hi, t_max = 0, 1 << 29, 30
    whole, _ = S.gap_counts(w, lo, hi, t_max)
    rng = np.random.default_rng(4)
    cuts = np.sort(rng.integers(0, w.size, 40))
    total = np.zeros(t_max + 1, np.uint64)
    carry = None
    for a, b in zip(np.concatenate([[0], cuts]), np.concatenate([cuts, [w.size]])):
        c, carry = S.gap_counts(w[a:b], lo, hi, t_max, carry)
        total += c
    assert np.array_equal(total, whole)


def test_gaps_geometric_on_pcg64():
    p, t_max = 1 / 16, 64
    c, _ = S.gap_counts(pcg_words(1 << 20), 0, 1 << 28, t_max)
    probs = np.array([p * (1 - p) ** r for r in range(t_max)] + [(1 - p) ** t_max])
    assert stats.chisquare(c.astype(float), probs * c.sum()).pvalue > 1e-4


# ----------------------------------------------------------- birthday ----

def test_birthday_hand_examples():
    # n = 4 birthdays in m = 16 days
    assert S.birthday_counts(np.array([1, 5, 9, 13], np.uint32), 2, 4, 0, 8).tolist()[3] == 1   # S = 4,4,4,4
    assert S.birthday_counts(np.array([0, 0, 0, 0], np.uint32), 2, 4, 0, 8).tolist()[2] == 1    # S = 0,0,0,16
    assert S.birthday_counts(np.array([3, 1, 2, 7], np.uint32), 2, 4, 0, 8).tolist()[1] == 1    # S = 1,1,4,10
    # r_max pools: R = 3 counted in counts[2]
    assert S.birthday_counts(np.array([1, 5, 9, 13], np.uint32), 2, 4, 0, 2).tolist() == [0, 0, 1]
    # shift and bits pick the field; incomplete samples are ignored
    c = S.birthday_counts(np.array([1 << 20, 5 << 20, 9 << 20, 13 << 20, 99], np.uint32), 2, 4, 20, 8)
    assert c.tolist()[3] == 1 and c.sum() == 1


def brute_birthday_r(ys, m):
    y = sorted(ys)
    sp = sorted([y[i + 1] - y[i] for i in range(len(y) - 1)] + [y[0] + m - y[-1]])
    return sum(1 for j in range(1, len(sp)) if sp[j] == sp[j - 1])


def test_birthday_matches_brute_force():
    rng = np.random.default_rng(11)
    w = rng.integers(0, 2**32, size=64 * 40, dtype=np.uint64).astype(np.uint32)
    got = S.birthday_counts(w, 6, 10, 22, 40)
    want = np.zeros(41, np.uint64)
    for s in range(40):
        ys = [(int(x) >> 22) & 1023 for x in w[s * 64:(s + 1) * 64]]
        want[min(brute_birthday_r(ys, 1024), 40)] += 1
    assert np.array_equal(got, want)


def test_birthday_mean_is_lambda_on_pcg64():
    # n = 4096, m = 2^32: lambda = 2^36 / 2^34 = 4
    n_samples = 400
    c = S.birthday_counts(pcg_words(4096 * n_samples), 12, 32, 0, 40)
    mean = float(np.dot(np.arange(41), c)) / n_samples
    assert abs(mean - 4.0) < 5 * math.sqrt(4.0 / n_samples)


# ------------------------------------------------- micro-stream layout ----

def test_micro_stream_layout(orc):
    w = S.micro_stream_words(orc.PHILOX, 0x5EED, 5, 3, 7, 4)
    assert w.shape == (4 * 5 * 3,)
    for j in range(4):
        for s in range(5):
            ref = orc.stream_words(orc.PHILOX, 0x5EED ^ s, 7 + j, 0, 3)
            assert np.array_equal(w[(j * 5 + s) * 3:(j * 5 + s + 1) * 3], ref)


# ---------------------------------------------------- planted mistakes ----

def test_planted_identical_micro_streams_fail(orc):
    """Every particle drawing the same words (the particle id dropped from the
    key) repeats each iteration's 3 words 16,000 times: the triple test
    (and the gap test) must reject it outright."""
    words = np.concatenate([np.tile(orc.stream_words(orc.PHILOX, 0x5EED, j, 0, 3), 16000) for j in range(6)])
    c = S.tuple_counts(words, 3, 4, 28, 3)
    assert stats.chisquare(c.astype(float)).pvalue < 1e-30
    p, t_max = 1 / 16, 64
    g, _ = S.gap_counts(words, 0, 1 << 28, t_max)
    probs = np.array([p * (1 - p) ** r for r in range(t_max)] + [(1 - p) ** t_max])
    if g.sum():
        assert stats.chisquare(g.astype(float), probs * g.sum()).pvalue < 1e-30


def test_planted_low_bit_alternation_fails():
    w = pcg_words(1 << 16)
    w = (w & np.uint32(0xFFFFFFFE)) | (np.arange(w.size, dtype=np.uint32) & np.uint32(1))
    # low bits of overlapping pairs: only cells 01 and 10 occur
    c = S.tuple_counts(w, 2, 1, 0, 1)
    assert c[0] == 0 and c[3] == 0
    assert stats.chisquare(c.astype(float)).pvalue < 1e-30


# ------------------------------------------- host-side evaluation (product) ----

def test_evaluate_matches_scipy_and_flags_failures():
    """The harness's p-values (paper_2310_19925_b300.stream_tests.evaluate)
    against scipy's tests on the same counts, and its verdicts on good and
    planted-bad counts from the oracle."""
    from paper_2310_19925_b300 import stream_tests as ST

    w = pcg_words(48000 * 40)
    for name, kind, prm in ST.BATTERY:
        if kind == "tuples":
            c = S.tuple_counts(w, prm["t"], prm["bits"], prm["shift"], prm["stride"])
        elif kind == "gaps":
            c, _ = S.gap_counts(w, prm["lo"], prm["hi"], prm["t_max"])
        else:
            c = S.birthday_counts(w, prm["log2_n"], prm["bits"], prm["shift"], prm["r_max"])
        r = ST.evaluate(kind, prm, c)
        assert r["verdict"] == "pass", (name, r["p"])
        if kind == "birthday":
            y = int(np.dot(np.arange(c.size), c.astype(np.int64)))
            mu = c.sum() * ST.birthday_mean(prm["log2_n"], prm["bits"])
            assert r["p"] == pytest.approx(min(1, 2 * min(stats.poisson.cdf(y, mu), stats.poisson.sf(y - 1, mu))))
            continue
        probs = ST.expected_probabilities(kind, prm)
        assert abs(probs.sum() - 1.0) < 1e-12
        exp = probs * c.sum()
        if exp.min() >= 5:
            assert r["p"] == pytest.approx(stats.chisquare(c.astype(float), exp).pvalue, rel=1e-9)
    bad = np.zeros(256, np.uint64)
    bad[:128] = 1000
    assert ST.evaluate("tuples", dict(t=1, bits=8, shift=24, stride=1), bad)["verdict"] == "fail"


def test_birthday_mean_against_brute_force():
    """E[R] = n (n-1)^2 / (4m) - n (n-1)^2 (n-2)^2 / (18 m^2), the mean the
    harness tests against, pinned by the oracle's own counts where the two
    corrections to Knuth's n^3 / (4m) are large: n = 64, m = 2^16 (lambda = 1;
    pairs 0.96899 minus triples 0.01263 gives 0.95636), 400,000 samples
    (standard error 0.0015)."""
    from paper_2310_19925_b300 import stream_tests as ST

    rng = np.random.default_rng(2024)
    n_samples = 400_000
    c = S.birthday_counts(pcg_words(64 * n_samples, rng), 6, 16, 0, 200)
    mean = float(np.dot(np.arange(201), c)) / n_samples
    se = math.sqrt(1.0 / n_samples)
    want = ST.birthday_mean(6, 16)
    assert abs(want - 0.95636) < 1e-5
    assert abs(mean - want) < 4 * se
    assert abs(mean - 1.0) > 10 * se          # Knuth's first-order mean is off by > 10 standard errors
