"""The device header's per-thread engine classes (orand::Philox, Threefry,
Squares, Tyche): the paper's draw interface (§3; Fig. 1 builds
`RNG rng(p.pid, counter)` in the thread and draws from it).

On the GPU, orand_engine_draws runs six draw methods in a fixed interleaving
(12 words a round, so draws straddle Philox/Threefry's 4-word blocks) and
every value is compared with the oracle's words and maps: words and uniforms
bit-exact, normals within 4 ulp.  On the host, orand_host_engine_words draws
through the same classes: the random-access engines start at any word and
wrap at the 2^32-word period, Tyche starts at word 0.
"""
import numpy as np
import pytest

from helpers import ulp_distance_f32

import paper_2310_19925_b300 as orand
from paper_2310_19925_b300 import workloads as W

M32 = 2**32
REC = np.dtype(orand.ENGINE_RECORD_FIELDS)


def _words(orc, gen, key, counter, first, n):
    """Words first .. first + n - 1 of a stream, positions taken modulo 2^32."""
    out, pos = [], first
    while n:
        k = min(n, M32 - pos)
        out.append(orc.stream_words(gen, key, counter, pos, k))
        n -= k
        pos = (pos + k) % M32
    return np.concatenate(out)


def _expected(orc, words):
    """The record fields from one thread's words (12 per round)."""
    w = words.reshape(-1, 12)
    f64 = lambda hi, lo: orc.map_words(W.F64_UNIFORM, np.stack([hi, lo], 1).ravel())
    f32 = lambda x: orc.map_words(W.F32_UNIFORM, x)
    return {"w": w[:, 0], "d1": f64(w[:, 1], w[:, 2]), "n": orc.box_muller_array(w[:, 3], w[:, 4]),
            "u": f32(w[:, 5]), "d2": np.stack([f64(w[:, 6], w[:, 7]), f64(w[:, 8], w[:, 9])], 1),
            "u2": np.stack([f32(w[:, 10]), f32(w[:, 11])], 1)}


CASES = [(0x5EED, 0, 0), (2**64 - 1, 2**32 - 1, 1), (0x0123456789ABCDEF, 77, 2**32 - 7)]


@pytest.mark.gpu
@pytest.mark.parametrize("gen", [W.PHILOX, W.THREEFRY, W.SQUARES, W.TYCHE])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_engine_draws_match_oracle(orc, gen, case):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    seed, counter, first = CASES[case]
    if gen == W.TYCHE and first:
        first = 0                                    # Tyche is sequential from word 0
    n_threads, n_rounds = 1000, 5                    # several blocks and a ragged tail
    out = orand.engine_draws(gen, seed, counter, n_threads, n_rounds, first_word=first)
    torch.cuda.synchronize()
    rec = out.cpu().numpy()[:n_threads * n_rounds * REC.itemsize].view(REC).reshape(n_threads, n_rounds)
    for t in list(range(0, n_threads, 7)) + [n_threads - 1]:
        exp = _expected(orc, _words(orc, gen, seed ^ t, counter, first, 12 * n_rounds))
        r = rec[t]
        assert np.array_equal(r["w"], exp["w"]), t
        assert np.array_equal(r["d1"], exp["d1"]) and np.array_equal(r["d2"], exp["d2"]), t
        assert np.array_equal(r["u"].astype(np.float64), exp["u"]), t
        assert np.array_equal(r["u2"].astype(np.float64), exp["u2"]), t
        assert ulp_distance_f32(r["n"], exp["n"]).max() <= 4, t


def test_engine_draws_reject_bad_arguments():
    """Argument checks run on the host before anything touches the device."""
    lib = orand._lib()
    assert lib.orand_engine_draws(4, 0, 0, 0, 1, 1, 16, None) == -1          # unknown generator
    assert lib.orand_engine_draws(3, 0, 0, 5, 1, 1, 16, None) == -1          # Tyche from word 5
    assert lib.orand_engine_draws(0, 0, 0, 0, 1, 1, 8, None) == -3           # out not 16-byte aligned
    assert lib.orand_engine_draws(0, 0, 0, 0, 2**62, 2**10, 16, None) == -2  # size overflows
    assert lib.orand_engine_draws(3, 0, 0, 0, 1, 2**30, 16, None) == -2      # Tyche past 2^32 words
    assert lib.orand_engine_draws(0, 0, 0, 0, 0, 5, 0, None) == 0            # nothing to do


@pytest.mark.parametrize("gen", [W.PHILOX, W.THREEFRY, W.SQUARES])
def test_host_engines_start_anywhere_and_wrap_at_the_period(orc, gen):
    for seed, counter in [(0x5EED, 0), (2**64 - 1, 2**32 - 1), (12345, 678)]:
        for first in (0, 1, 2, 3, 5, M32 - 3, M32 - 1):
            got = orand.host_engine_words(gen, seed, counter, 9, first_word=first)
            assert np.array_equal(got, _words(orc, gen, seed, counter, first, 9)), (seed, counter, first)


def test_host_tyche_engine(orc):
    for seed, counter in [(0x5EED, 0), (2**64 - 1, 2**32 - 1)]:
        assert np.array_equal(orand.host_engine_words(W.TYCHE, seed, counter, 100),
                              orc.stream_words(W.TYCHE, seed, counter, 0, 100))
    with pytest.raises(orand.OrandError):
        orand.host_engine_words(W.TYCHE, 1, 2, 4, first_word=1)
