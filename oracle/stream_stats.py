"""Plain CPU definitions of the parallel-stream correlation test.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it; the product path never does and shares no code with it.

The paper's statistical evaluation (§5, Statistical Evaluation) checks
parallel streams after Anderson et al. (HOOMD-blue, 2020): 16,000
particles each draw a micro-stream of three numbers, the micro-streams are
concatenated into one stream, and the stream is lengthened over successive
iterations.  Here particle s of iteration j draws the first `draws` words of
the stream with key seed ^ s and counter counter_first + j (§3: the seed
names the processing element, the counter the iteration), and the words of
iteration j follow those of iteration j - 1.

The batteries the paper ran (TestU01, PractRand) are not available, so the
concatenated stream is checked with three classical tests, each written out
here from its textbook definition (Knuth, TAOCP vol. 2, §3.3.2):
  * tuple frequencies (serial test): non-overlapping t-tuples of b-bit
    fields, counted in 2^(t b) cells;
  * the gap test: lengths of the runs of words outside [lo, hi) between
    consecutive words inside it;
  * birthday spacings (Marsaglia; Knuth's form): n birthdays in m days,
    sorted, with the n spacings including the wrap-around one; R = the
    number of equal adjacent values among the sorted spacings.
Only integer counts come out; p-values are computed from them elsewhere.
"""
from __future__ import annotations

import numpy as np

from . import U32, fill


def micro_stream_words(gen: int, seed: int, n_streams: int, draws: int, counter_first: int,
                       n_counters: int) -> np.ndarray:
    """The concatenated stream: iteration j (counter counter_first + j) puts
    the `draws` words of particles 0..n_streams-1 one after the other; the
    iterations follow each other.  Returns n_counters * n_streams * draws u32."""
    parts = [fill(gen, U32, seed, counter_first + j, n_streams, draws) for j in range(n_counters)]
    if not parts:
        return np.zeros(0, np.uint32)
    return np.concatenate(parts).astype(np.uint32)


def tuple_counts(words, t: int, bits: int, shift: int, stride: int) -> np.ndarray:
    """Counts of the 2^(t*bits) cells.  Tuple m is words[m*stride : m*stride + t]
    for every m with m*stride + t <= n; each word contributes its field
    (w >> shift) & (2^bits - 1), the first word in the highest position."""
    w = np.asarray(words, dtype=np.uint64)
    n = w.size
    n_tuples = 0 if n < t else (n - t) // stride + 1
    cell = np.zeros(n_tuples, dtype=np.uint64)
    starts = np.arange(n_tuples, dtype=np.int64) * stride
    mask = np.uint64((1 << bits) - 1)
    for i in range(t):
        field = (w[starts + i] >> np.uint64(shift)) & mask
        cell = (cell << np.uint64(bits)) | field
    return np.bincount(cell.astype(np.int64), minlength=1 << (t * bits)).astype(np.uint64)


def gap_counts(words, lo: int, hi: int, t_max: int, carry=None):
    """Gap test.  A word is a hit when lo <= w < hi (hi may be 2^32).  Each
    hit after the first closes a gap: the number of non-hit words since the
    previous hit.  counts[r] for r < t_max, gaps of t_max or more pooled in
    counts[t_max].  `carry` is the number of non-hit words after the last
    hit of the stream's earlier part (None: no hit yet), so a stream fed in
    pieces gives the same counts as in one piece.  Returns (counts, carry)."""
    w = np.asarray(words, dtype=np.uint64)
    hits = np.flatnonzero((w >= lo) & (w < hi))
    gaps = np.diff(hits) - 1
    if carry is not None and hits.size:
        gaps = np.concatenate([[carry + hits[0]], gaps])
    counts = np.bincount(np.minimum(gaps, t_max).astype(np.int64), minlength=t_max + 1).astype(np.uint64)
    if hits.size:
        carry = int(w.size - 1 - hits[-1])
    elif carry is not None:
        carry = int(carry + w.size)
    return counts, carry


def birthday_counts(words, log2_n: int, bits: int, shift: int, r_max: int) -> np.ndarray:
    """Birthday spacings.  Sample s takes the n = 2^log2_n words
    words[s*n : (s+1)*n] (whole samples only); birthday = (w >> shift) &
    (2^bits - 1) in a year of m = 2^bits days.  With the birthdays sorted,
    Y(1) <= ... <= Y(n), the spacings are Y(i+1) - Y(i) and Y(1) + m - Y(n);
    sorted, R counts the j with S(j) == S(j-1).  Returns counts[min(R, r_max)]."""
    n = 1 << log2_n
    w = np.asarray(words, dtype=np.uint64)
    n_samples = w.size // n
    counts = np.zeros(r_max + 1, dtype=np.uint64)
    if n_samples == 0:
        return counts
    y = (w[: n_samples * n].reshape(n_samples, n) >> np.uint64(shift)) & np.uint64((1 << bits) - 1)
    y = np.sort(y.astype(np.int64), axis=1)
    wrap = y[:, :1] + (1 << bits) - y[:, -1:]
    s = np.sort(np.concatenate([np.diff(y, axis=1), wrap], axis=1), axis=1)
    r = np.sum(s[:, 1:] == s[:, :-1], axis=1)
    np.add.at(counts, np.minimum(r, r_max), 1)
    return counts
