"""C-ABI checks that need no GPU: the library loads, exports every entry
point the public header declares, and rejects bad arguments on the host
before any launch."""
import ctypes
import os
import re

import pytest

import paper_2310_19925_b300 as orand

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def _declared_functions():
    names = set()
    for h in sorted(os.listdir(INCLUDE)):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(INCLUDE, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(orand_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2310_19925_b300 import build

    build.build()
    return orand._lib()


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert "orand_fill_u32" in declared and "orand_stat_gaps" in declared and len(declared) >= 8
    for name in declared:
        assert hasattr(lib, name), name
        assert name in orand._SIGS, "binding lacks " + name


def test_status_strings(lib):
    for code, name in orand.STATUS_NAMES.items():
        assert lib.orand_status_string(code).decode().startswith(name)
    assert lib.orand_version() >= 100


@pytest.mark.parametrize("gen,dtype", [(4, 0), (-1, 0), (0, 4), (0, -2)])
def test_bad_enums_rejected(lib, gen, dtype):
    assert lib.orand_fill(gen, dtype, 1, 0, 4, 4, 16, None) == -1


def test_stream_range_overflow_rejected(lib):
    assert lib.orand_fill_streams(0, 0, 1, 0, 2**64 - 10, 11, 4, 16, None) == -2   # stream ids pass 2^64
    assert lib.orand_fill_streams(0, 0, 1, 0, 2**62, 2**62, 16, 16, None) == -2     # (first + n) * dps overflows
    assert lib.orand_fill_streams(0, 0, 1, 0, 2**64 - 10, 0, 4, None, None) == 0    # empty range


def test_overflow_rejected(lib):
    assert lib.orand_fill(0, 0, 1, 0, 2**40, 2**30, 16, None) == -2          # n*dps overflows
    assert lib.orand_fill(0, 0, 1, 0, 2**62, 2, 16, None) == -2              # bytes overflow
    assert lib.orand_fill(0, 0, 1, 0, 1, 2**32 + 1, 16, None) == -2          # > 2^32 words
    assert lib.orand_fill(0, 2, 1, 0, 1, 2**31 + 1, 16, None) == -2          # f64 needs 2 words each


def test_null_and_alignment_rejected(lib):
    assert lib.orand_fill(0, 0, 1, 0, 4, 4, None, None) == -1
    assert lib.orand_fill(0, 0, 1, 0, 4, 4, 2, None) == -3                   # u32 at 2-byte offset
    assert lib.orand_fill(0, 2, 1, 0, 4, 4, 4, None) == -3                   # f64 at 4-byte offset


def test_empty_fill_is_a_noop(lib):
    assert lib.orand_fill(0, 0, 1, 0, 0, 5, None, None) == 0
    assert lib.orand_fill(3, 3, 1, 0, 7, 0, None, None) == 0


def test_python_errors_raise(lib):
    with pytest.raises(orand.OrandError):
        orand.orand_fill(9, 0, 1, 0, 1, 1, 16, 0)


def test_walk_arguments_rejected_on_host(lib):
    W2 = orand.walk2d_params
    assert lib.orand_brownian_walk(None, None, None) == -1
    assert lib.orand_brownian_walk(ctypes.byref(W2(0, 10)), None, None) == 0            # empty: no-op
    assert lib.orand_brownian_walk(ctypes.byref(W2(4, 10, dt=-1.0)), None, None) == -1
    assert lib.orand_brownian_walk(ctypes.byref(W2(4, 10, D=float("nan"))), None, None) == -1
    assert lib.orand_brownian_walk(ctypes.byref(W2(4, 10)), None, None) == -1           # NULL output
    assert lib.orand_brownian_walk(ctypes.byref(W2(4, 10)), 4, None) == -3              # not 8-byte aligned
    assert lib.orand_brownian_walk(ctypes.byref(W2(8, 10, p_first=2**64 - 4)), 8, None) == -2
    assert lib.orand_brownian_walk(ctypes.byref(W2(8, 2**32 - 1)), 8, None) == -2        # counter 2^32 - 1 limit
    assert lib.orand_walk2d_curand_state_bytes() >= 48
    assert lib.orand_walk2d_curand_setup(ctypes.byref(W2(4, 10)), None, 8, 0, None) == -1   # NULL states
    assert lib.orand_walk2d_curand_setup(ctypes.byref(W2(4, 10)), 8, 8, 0, None) == -3      # misaligned states
    assert lib.orand_walk2d_curand_run(ctypes.byref(W2(4, 10)), 16, 4, None) == -3          # misaligned pos
    assert lib.orand_walk2d_curand_fused(ctypes.byref(W2(4, 10, dt=-1.0)), 8, 0, None) == -1
    p3 = orand.walk3d_params(10, 5)
    assert lib.orand_walk3d_fwd(None, ctypes.byref(p3), None, 16, None, None, None) == -1  # no context
    assert lib.orand_walk3d_fwd(None, None, None, 16, None, None, None) == -1
    bad = orand.walk3d_params(10, 5, sigma=-0.5)
    assert lib.orand_walk3d_bwd(None, ctypes.byref(bad), 16, None, None, 16, 16, None, None, None) == -1
    ou = orand.walk3d_params(10, 5, kappa=1.0)
    assert lib.orand_walk3d_stored_fwd(None, ctypes.byref(ou), None, 16, 16, None, None) == -1   # kappa != 0
    assert lib.orand_walk3d_stored_bwd(None, ctypes.byref(ou), 16, 16, None, 16, 16, None, None) == -1
    big = orand.walk3d_params(2**40, 5)
    assert lib.orand_walk3d_init(ctypes.byref(big), 16, None) == -2                      # grid too large
    steps_max = orand.walk3d_params(1, 2**32 - 1)
    assert lib.orand_walk3d_init(ctypes.byref(steps_max), 16, None) == -2


def test_context_needs_a_device_or_succeeds(lib):
    import torch

    h = ctypes.c_void_p()
    st = lib.orand_ctx_create(ctypes.byref(h))
    if torch.cuda.is_available():
        assert st == 0 and h.value
        assert lib.orand_ctx_destroy(h) == 0
    else:
        assert st in (-5, -7) and not h.value
    assert lib.orand_ctx_create(None) == -1
    assert lib.orand_ctx_destroy(None) == -1


def _reqs(rows):
    import numpy as np

    from paper_2310_19925_b300.workloads import REQUEST_DTYPE

    a = np.zeros(len(rows), REQUEST_DTYPE)
    for i, r in enumerate(rows):
        for k, v in r.items():
            a[i][k] = v
    return a


def test_ragged_arguments_rejected_on_host(lib):
    ok = dict(gen=0, dtype=0, seed=1, counter=2, length=8, out_offset_bytes=0)
    serial = lib.orand_fill_ragged_serial
    r = _reqs([ok])
    assert serial(r.ctypes.data, 0, None, 0, None) == 0                                  # empty batch
    assert serial(None, 3, 16, 64, None) == -1
    for bad, code in [(dict(ok, gen=4), -1), (dict(ok, dtype=9), -1), (dict(ok, reserved=1), -1),
                      (dict(ok, length=2**32 + 1), -2), (dict(ok, dtype=2, length=2**31 + 1), -2),
                      (dict(ok, out_offset_bytes=232), -2), (dict(ok, out_offset_bytes=2**64 - 8), -2),
                      (dict(ok, out_offset_bytes=2), -3), (dict(ok, dtype=2, out_offset_bytes=4), -3)]:
        rr = _reqs([ok, bad])
        assert serial(rr.ctypes.data, 2, 16, 256, None) == code, bad
    assert lib.orand_fill_ragged(None, r.ctypes.data, 1, 16, 64, None) == -1            # no context
    cfg = orand.RaggedConfig(256, 8192, 16, 0)
    assert lib.orand_ragged_set_config(None, ctypes.byref(cfg)) == -1


def test_langevin_arguments_rejected_on_host(lib):
    P = orand.langevin2d_params
    assert lib.orand_langevin2d_init(None, 16, None) == -1
    assert lib.orand_langevin2d_step(ctypes.byref(P(0)), None, 1, None) == 0              # empty: no-op
    assert lib.orand_langevin2d_step(ctypes.byref(P(4, mass=0.0)), 16, 1, None) == -1
    assert lib.orand_langevin2d_step(ctypes.byref(P(4, dt=-1e-3)), 16, 1, None) == -1
    assert lib.orand_langevin2d_step(ctypes.byref(P(4, gamma=float("nan"))), 16, 1, None) == -1
    assert lib.orand_langevin2d_step(ctypes.byref(P(4)), None, 1, None) == -1
    assert lib.orand_langevin2d_step(ctypes.byref(P(4)), 4, 1, None) == -3                # not 8-byte aligned
    assert lib.orand_langevin2d_fused(ctypes.byref(P(4)), 16, 2**32 - 5, 10, None) == -2  # counters wrap
    assert lib.orand_langevin2d_curand_setup(ctypes.byref(P(4)), 16, None, 1984, None) == -1
    assert lib.orand_langevin2d_curand_state_bytes() >= 48


def test_stream_statistics_arguments_rejected_on_host(lib):
    L = lib
    assert L.orand_fill_micro_streams(9, 0, 10, 3, 0, 1, 16, None) == -1          # unknown generator
    assert L.orand_fill_micro_streams(0, 0, 10, 0, 0, 1, 16, None) == -1          # draws = 0
    assert L.orand_fill_micro_streams(0, 0, 10, 65, 0, 1, 16, None) == -1         # draws > 64
    assert L.orand_fill_micro_streams(0, 0, 10, 3, 2**32 - 2, 3, 16, None) == -2  # counters wrap
    assert L.orand_fill_micro_streams(0, 0, 2**62, 3, 0, 2, 16, None) == -2       # size overflow
    assert L.orand_fill_micro_streams(0, 0, 10, 3, 0, 0, None, None) == 0         # empty: no-op
    assert L.orand_fill_micro_streams(0, 0, 10, 3, 0, 1, None, None) == -1        # NULL output
    assert L.orand_fill_micro_streams(0, 0, 10, 3, 0, 1, 2, None) == -3           # misaligned output
    assert L.orand_stat_tuples(16, 100, 0, 8, 24, 1, 16, None) == -1              # t = 0
    assert L.orand_stat_tuples(16, 100, 3, 5, 0, 3, 16, None) == -1               # 15 bits of cells
    assert L.orand_stat_tuples(16, 100, 1, 8, 25, 1, 16, None) == -1              # field past bit 31
    assert L.orand_stat_tuples(16, 100, 1, 8, 24, 0, 16, None) == -1              # stride 0
    assert L.orand_stat_tuples(16, 100, 1, 8, 24, 1, 4, None) == -3               # counts misaligned
    assert L.orand_stat_tuples(None, 0, 1, 8, 24, 1, 16, None) == 0               # no tuple: no-op
    assert L.orand_stat_gaps(None, 16, 10, 5, 5, 8, 16, 16, None) == -1           # lo >= hi
    assert L.orand_stat_gaps(None, 16, 10, 0, 2**32 + 1, 8, 16, 16, None) == -1   # hi > 2^32
    assert L.orand_stat_gaps(None, 16, 10, 0, 16, 0, 16, 16, None) == -1          # t_max = 0
    assert L.orand_stat_gaps(None, 16, 10, 0, 16, 8, 16, None, None) == -1        # NULL carry
    assert L.orand_stat_gaps(None, 16, 10, 0, 16, 8, 16, 16, None) == -1          # NULL context
    assert L.orand_stat_birthday(16, 100, 1, 32, 0, 8, 16, None) == -1            # log2_n < 2
    assert L.orand_stat_birthday(16, 100, 13, 32, 0, 8, 16, None) == -1           # log2_n > 12
    assert L.orand_stat_birthday(16, 100, 4, 24, 9, 8, 16, None) == -1            # field past bit 31
    assert L.orand_stat_birthday(16, 100, 4, 24, 8, 0, 16, None) == -1            # r_max = 0
    assert L.orand_stat_birthday(16, 15, 4, 24, 8, 8, 16, None) == 0              # no whole sample


def test_injected_allocation_failure_in_ctx_create(lib, monkeypatch):
    """With ORAND_FAIL_ALLOC=1 every library allocation is refused before the
    allocator runs; orand_ctx_create reports ORAND_ERR_ALLOC (its host object
    is allocated before the device is queried) and leaves the handle NULL."""
    h = ctypes.c_void_p(12345)
    monkeypatch.setenv("ORAND_FAIL_ALLOC", "1")
    assert lib.orand_ctx_create(ctypes.byref(h)) == -4
    assert h.value is None
    monkeypatch.delenv("ORAND_FAIL_ALLOC")
    st = lib.orand_ctx_create(ctypes.byref(h))
    assert st != -4                       # ORAND_OK on a GPU; a device error without one
    if st == 0:
        assert lib.orand_ctx_destroy(h) == 0


def test_nvtx_ranges_leave_results_unchanged():
    """ORAND_NVTX=1 wraps each launching call in an NVTX range (for
    profilers); the calls return what they return without it."""
    import subprocess
    import sys

    code = ("import ctypes, paper_2310_19925_b300 as o; L = o._lib(); "
            "assert L.orand_fill(4, 0, 1, 0, 4, 4, 16, None) == -1; "
            "assert L.orand_fill_streams(0, 0, 1, 0, 2**64 - 10, 11, 4, 16, None) == -2; "
            "assert L.orand_engine_draws(0, 0, 0, 0, 0, 5, 0, None) == 0; print('ok')")
    env = dict(os.environ, ORAND_NVTX="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr
