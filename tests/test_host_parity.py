"""Host-side generation against the oracle (CPU, no GPU needed).

The host streams come from the device header's generator source compiled
for the CPU; they must equal the oracle's words bit for bit, which also
shows the shared source computes the same streams the GPU parity tests
check on the device.  The micro-benchmark is checked for its contract
(finite, positive times; streams of every length drawn).
"""
import ctypes

import numpy as np
import pytest

import paper_2310_19925_b300 as orand
from paper_2310_19925_b300 import workloads as W

GENS = [W.PHILOX, W.THREEFRY, W.SQUARES, W.TYCHE]


@pytest.fixture(scope="module")
def lib():
    from paper_2310_19925_b300 import build

    build.build()
    return orand._lib()


@pytest.mark.parametrize("gen", GENS)
@pytest.mark.parametrize("seed,counter,n_streams,dps", [(0x5EED, 0, 37, 18), (2**63 + 12345, 2**32 - 1, 5, 33),
                                                        (0, 7, 1, 1), (42, 3, 64, 64)])
def test_host_fill_bit_exact(lib, orc, gen, seed, counter, n_streams, dps):
    got = orand.host_fill_u32(gen, seed, counter, n_streams, dps)
    assert np.array_equal(got, orc.fill(gen, orc.U32, seed, counter, n_streams, dps))


def test_host_arguments_rejected(lib):
    assert lib.orand_host_fill_u32(9, 0, 0, 1, 1, 16) == -1               # unknown generator
    assert lib.orand_host_fill_u32(0, 0, 0, 1, 2**32 + 1, 16) == -2       # longer than a stream
    assert lib.orand_host_fill_u32(0, 0, 0, 2**40, 2**30, 16) == -2       # size product overflows
    assert lib.orand_host_fill_u32(0, 0, 0, 0, 5, None) == 0              # empty
    assert lib.orand_host_fill_u32(0, 0, 0, 1, 1, None) == -1             # NULL output
    assert lib.orand_host_fill_u32(0, 0, 0, 1, 1, 2) == -3                # misaligned
    L = (ctypes.c_uint64 * 1)(0)
    ns = (ctypes.c_double * 1)()
    sink = (ctypes.c_uint32 * 1)()
    assert lib.orand_host_microbench(7, L, 1, 10, ns, sink) == -1         # unknown generator
    assert lib.orand_host_microbench(0, L, 1, 10, ns, sink) == -1         # length 0
    assert lib.orand_host_microbench(0, None, 0, 10, None, None) == 0     # nothing to time


def test_microbench_contract(lib):
    lengths = [1, 16, 1024]
    for g in GENS + [orand.HOST_MT19937]:
        ns = orand.host_microbench(g, lengths, words_per_length=1 << 14)
        assert ns.shape == (3,) and np.all(np.isfinite(ns)) and np.all(ns > 0)
        assert ns[2] > ns[0]          # a 1024-word stream takes longer than a 1-word one
