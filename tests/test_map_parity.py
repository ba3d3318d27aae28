"""Exhaustive GPU checks of the word -> value maps against the oracle.

The Box-Muller map is checked on every possible input of each half:
  * all 2^24 values of u1 with u2 = 0, so z0 is the radius alone and z1 is 0;
  * all 2^24 values of u2 at one fixed radius (this includes the exact zeros
    at u2 = 0, 1/4, 1/2, 3/4);
  * 2^24 random word pairs.
The bar for normals is 4 ulp (ordered-integer distance to the FP64 value
rounded to FP32).  The components are held to 2 ulp.  The uniform maps are
bit-exact: the FP32 map over all 2^24 distinct values, the FP64 map on
random words.
"""
import numpy as np
import pytest

from helpers import ordered_f32, to_numpy, ulp_distance_f32

import paper_2310_19925_b300 as orand
from paper_2310_19925_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_normals(torch, w0, w1):
    words = np.empty(2 * len(w0), np.uint32)
    words[0::2], words[1::2] = w0, w1
    t = torch.from_numpy(words.view(np.int32)).cuda()
    z = orand.map_words(W.F32_NORMAL, t)
    torch.cuda.synchronize()
    return to_numpy(z).reshape(-1, 2)


def test_radius_all_u1(torch_cuda, orc):
    rng = np.random.default_rng(1)
    k = np.arange(1 << 24, dtype=np.uint32)
    w0 = (k << 8) | rng.integers(0, 256, k.size, dtype=np.uint32)
    w1 = rng.integers(0, 256, k.size, dtype=np.uint32)           # u2 = 0
    z = gpu_normals(torch_cuda, w0, w1)
    ref = orc.box_muller_array(w0, w1)
    assert np.all(z[:, 1] == 0.0)
    d = ulp_distance_f32(z[:, 0], ref[:, 0])
    assert d.max() <= 2, "radius max ulp %d at k=%d" % (d.max(), int(k[d.argmax()]))
    assert z[-1, 0] == 0.0 and not np.signbit(z[-1, 0])          # u1 = 1 gives +0


def test_trig_all_u2(torch_cuda, orc):
    m = np.arange(1 << 24, dtype=np.uint32)
    w1 = m << 8
    w0 = np.full(m.size, 0x7FFFFF00, np.uint32)                  # u1 = 1/2: r = sqrt(2 ln 2)
    z = gpu_normals(torch_cuda, w0, w1)
    ref = orc.box_muller_array(w0, w1)
    for c in (0, 1):
        d = ulp_distance_f32(z[:, c], ref[:, c])
        assert d.max() <= 4, "component %d max ulp %d at m=%d" % (c, d.max(), int(m[d.argmax()]))
    quarter = np.array([0, 1 << 22, 2 << 22, 3 << 22])
    assert np.all(ordered_f32(z[quarter, 0][[1, 3]]) == 0) and np.all(ordered_f32(z[quarter, 1][[0, 2]]) == 0)


def test_normals_random_pairs(torch_cuda, orc):
    rng = np.random.default_rng(2)
    w = rng.integers(0, 2**32, (1 << 24, 2), dtype=np.uint64).astype(np.uint32)
    z = gpu_normals(torch_cuda, w[:, 0], w[:, 1])
    ref = orc.box_muller_array(w[:, 0], w[:, 1])
    d = ulp_distance_f32(z.ravel(), ref.ravel())
    assert d.max() <= 4
    # Measured with the SFU's square root in the radius: 3 ulp at most, on
    # 1.3e-5 of the components.
    assert (d > 2).mean() < 1e-4


def test_uniform_maps_exact(torch_cuda, orc):
    torch = torch_cuda
    rng = np.random.default_rng(3)
    k = np.arange(1 << 24, dtype=np.uint32)
    w = (k << 8) | rng.integers(0, 256, k.size, dtype=np.uint32)
    got = to_numpy(orand.map_words(W.F32_UNIFORM, torch.from_numpy(w.view(np.int32)).cuda()))
    assert np.array_equal(got.astype(np.float64), orc.map_words(W.F32_UNIFORM, w))
    w2 = rng.integers(0, 2**32, 1 << 22, dtype=np.uint64).astype(np.uint32)
    w2[:8] = [0, 0, 0, 0x800, 0xFFFFFFFF, 0xFFFFFFFF, 0x80000000, 0]
    got = to_numpy(orand.map_words(W.F64_UNIFORM, torch.from_numpy(w2.view(np.int32)).cuda()))
    assert np.array_equal(got, orc.map_words(W.F64_UNIFORM, w2))
    got = to_numpy(orand.map_words(W.U32, torch.from_numpy(w2.view(np.int32)).cuda()))
    assert np.array_equal(got, w2)


def test_f64_map_every_leading_bit(torch_cuda, orc):
    """The FP64 map takes a short path when the high word is >= 2^20 and the
    general one otherwise, chosen per pair of values.  Every position of the
    high word's leading bit (and a zero high word), with random low words,
    each paired with a partner from both paths, is bit-exact."""
    torch = torch_cuda
    rng = np.random.default_rng(4)
    his = [0]
    for p in range(32):
        his += [int(v) | (1 << p) for v in rng.integers(0, 1 << p, 64, dtype=np.uint64)] if p else [1] * 64
    his = np.array(his, np.uint64).astype(np.uint32)
    n = his.size
    partner = np.where(np.arange(n) % 2 == 0, rng.integers(1 << 20, 2**32, n, dtype=np.uint64),
                       rng.integers(0, 1 << 20, n, dtype=np.uint64)).astype(np.uint32)
    w = np.empty((n, 4), np.uint32)
    w[:, 0], w[:, 2] = his, partner
    w[:, 1] = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    w[:, 3] = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    w[::3, 1] = 0x7FF                                             # the bits the >> 11 drops
    w[1::3, 1] = 0xFFFFF800
    for words in (w.ravel(), w[:, [2, 3, 0, 1]].ravel()):       # each word in both slots
        got = to_numpy(orand.map_words(W.F64_UNIFORM, torch.from_numpy(words.view(np.int32)).cuda()))
        assert np.array_equal(got, orc.map_words(W.F64_UNIFORM, words))


def test_map_words_odd_counts_match_fill(torch_cuda, orc):
    torch = torch_cuda
    for dtype in range(4):
        for n in (1, 3, 5, 18):
            words = orc.stream_words(W.PHILOX, 9, 2, 0, orc.words_for(dtype, n))
            got = to_numpy(orand.map_words(dtype, torch.from_numpy(words.view(np.int32)).cuda(), n_values=n))
            ref = orc.fill(W.PHILOX, dtype, 9, 2, 1, n)
            if dtype == W.F32_NORMAL:
                assert ulp_distance_f32(got, ref).max() <= 4
            else:
                assert np.array_equal(got.astype(ref.dtype), ref)


# ------------------------------------------------ the walks' normal map ----

def walk_normals(torch, w0, w1):
    words = np.empty(2 * len(w0), np.uint32)
    words[0::2], words[1::2] = w0, w1
    z = orand.walk_normals(torch.from_numpy(words.view(np.int32)).cuda())
    torch.cuda.synchronize()
    return to_numpy(z).reshape(-1, 2).astype(np.float64)


def test_walk_map_radius_all_u1(torch_cuda, orc):
    """Every u1 at u2 = 1/4 (cosine 0, sine 1): z1 is the radius, within
    1e-6 relative of the FP64 value (measured 5.8e-7), and finite, non-negative
    up to the cosine term, everywhere including u1 = 1."""
    k = np.arange(1 << 24, dtype=np.uint32)
    w0 = k << 8
    w1 = np.full(k.size, 1 << 30, np.uint32)                     # u2 = 1/4
    z = walk_normals(torch_cuda, w0, w1)
    ref = orc.box_muller_array(w0, w1)
    assert np.all(np.isfinite(z))
    err = np.abs(z[:, 1] - ref[:, 1])
    assert np.all(err <= 1e-6 * ref[:, 1] + 1e-30), "radius rel err %.3g at k=%d" % (
        (err / np.maximum(ref[:, 1], 1e-30)).max(), int(k[err.argmax()]))
    assert np.all(np.abs(z[:, 0]) <= 5e-7 * np.maximum(ref[:, 1], 1.0))   # r cos(pi/2) ~ 0
    assert z[-1, 1] == 0.0                                       # u1 = 1 gives r = 0


def test_walk_map_trig_all_u2(torch_cuda, orc):
    """Every u2 at r = sqrt(2 ln 2): cos and sin within 4e-7 absolute of the
    FP64 values times the radius, plus the radius error.  And no mean error:
    a walk of T steps of size s drifts by T s E[r] times the mean error of
    the cosine or sine, so it is held below 2e-10 (about 1e-7 over the 10^4
    steps of the 2D workload)."""
    m = np.arange(1 << 24, dtype=np.uint32)
    w1 = m << 8
    w0 = np.full(m.size, 0x7FFFFF00, np.uint32)                  # u1 = 1/2
    z = walk_normals(torch_cuda, w0, w1)
    ref = orc.box_muller_array(w0, w1)
    r = np.sqrt(2 * np.log(2))
    bound = 4e-7 * r + 1e-6 * np.abs(ref)
    assert np.all(np.abs(z - ref) <= bound)
    bias = (z - ref).mean(axis=0) / r
    assert np.all(np.abs(bias) < 2e-10), bias


def test_walk_map_random_pairs_and_moments(torch_cuda, orc):
    rng = np.random.default_rng(3)
    w = rng.integers(0, 2**32, size=(1 << 22, 2), dtype=np.uint64).astype(np.uint32)
    z = walk_normals(torch_cuda, w[:, 0], w[:, 1])
    ref = orc.box_muller_array(w[:, 0], w[:, 1])
    rr = np.sqrt(ref[:, 0] ** 2 + ref[:, 1] ** 2)
    assert np.all(np.abs(z - ref) <= (1e-6 + 4e-7) * rr[:, None] + 1e-12)
    zz = z.ravel()
    n = zz.size
    assert abs(zz.mean()) < 5 / np.sqrt(n) and abs(zz.var() - 1) < 5 * np.sqrt(2 / n)
