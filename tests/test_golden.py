"""Stored expected values (tests/golden/, written by make_golden.py from the
oracle; each file's header cites the passage it follows).

On the CPU the oracle must reproduce every stored value exactly, so a later
change to its arithmetic cannot pass unnoticed.  On the GPU the library is
checked against the stored values directly, with the oracle out of the loop:
words and uniforms bit-exact, normals within 4 ulp of the FP64 value, walk
positions within 1e-5 relative (floor 1).
"""
import os

import numpy as np
import pytest

from helpers import to_numpy, ulp_distance_f32

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GEN_IDS = {"philox4x32_10": 0, "threefry4x32_20": 1, "squares32": 2, "tyche": 3}

WALK2D = dict(seed=0x77, n=8, steps=37, dt=float(np.float32(1e-3)), D=1.0)
WALK3D = dict(seed=0, n=6, steps=65, K=16, dt=float(np.float32(1e-3)), mu=(0.1, -0.2, 0.05), sigma=0.5,
              p_first=3)


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def stream_rows():
    return [(GEN_IDS[p[0]], int(p[1], 16), int(p[2], 16), np.array([int(x, 16) for x in p[3:]], np.uint32))
            for p in _lines("stream_words.txt")]


def map_rows():
    f32, pairs = [], []
    for p in _lines("value_maps.txt"):
        if p[0] == "f32":
            f32.append((int(p[1], 16), int(p[2], 16)))
        else:
            pairs.append((int(p[1], 16), int(p[2], 16), float.fromhex(p[3]), float.fromhex(p[4]),
                          float.fromhex(p[5])))
    return f32, pairs


def walk_rows():
    w2, w3 = {}, {}
    for p in _lines("walk_positions.txt"):
        v = np.array([float.fromhex(x) for x in p[2:]])
        (w2 if p[0] == "walk2d" else w3)[int(p[1])] = v
    return w2, w3


def test_golden_files_cover_every_generator():
    rows = stream_rows()
    assert sorted({r[0] for r in rows}) == [0, 1, 2, 3]
    assert all(len(r[3]) == 16 for r in rows) and len(rows) == 60
    f32, pairs = map_rows()
    assert len(f32) == 64 and len(pairs) == 32
    w2, w3 = walk_rows()
    assert len(w2) == 8 and len(w3) == 6


# ----------------------------------------------------------------- CPU ----

def test_oracle_reproduces_stored_stream_words(orc):
    for gen, key, ctr, words in stream_rows():
        assert np.array_equal(orc.stream_words(gen, key, ctr, 0, 16), words), (gen, hex(key), ctr)


def test_oracle_reproduces_stored_maps(orc):
    f32, pairs = map_rows()
    w = np.array([a for a, _ in f32], np.uint32)
    got = orc.map_words(orc.F32_UNIFORM, w)
    assert [int(np.float32(v).view(np.uint32)) for v in got] == [b for _, b in f32]
    pw = np.array([[a, b] for a, b, *_ in pairs], np.uint32)
    f64 = orc.map_words(orc.F64_UNIFORM, pw.ravel())
    assert np.array_equal(f64, np.array([p[2] for p in pairs]))
    z = orc.box_muller_array(pw[:, 0], pw[:, 1])
    assert np.array_equal(z, np.array([[p[3], p[4]] for p in pairs]))


def test_oracle_reproduces_stored_walks(orc):
    w2, w3 = walk_rows()
    c2, c3 = WALK2D, WALK3D
    _, xT = orc.walk2d(c2["seed"], c2["n"], c2["steps"], c2["dt"], c2["D"])
    assert np.array_equal(xT, np.array([w2[i] for i in range(c2["n"])]))
    yT, _ = orc.walk3d_forward(c3["seed"], c3["n"], c3["steps"], c3["K"], c3["dt"], c3["mu"], c3["sigma"],
                               p_first=c3["p_first"])
    assert np.array_equal(yT, np.array([w3[c3["p_first"] + i] for i in range(c3["n"])]))


# ----------------------------------------------------------------- GPU ----

@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.gpu
def test_gpu_matches_stored_stream_words(torch_cuda):
    import paper_2310_19925_b300 as orand

    for gen, key, ctr, words in stream_rows():
        # One stream of the fill keyed by seed = key64 (stream 0: key64 ^ 0).
        got = to_numpy(orand.fill(gen, orand.U32, key, ctr, 1, 16))
        assert np.array_equal(got, words), (gen, hex(key), ctr)


@pytest.mark.gpu
def test_gpu_matches_stored_maps(torch_cuda):
    import paper_2310_19925_b300 as orand

    torch = torch_cuda
    f32, pairs = map_rows()
    w = torch.from_numpy(np.array([a for a, _ in f32], np.uint32).view(np.int32)).cuda()
    got = to_numpy(orand.map_words(orand.F32_UNIFORM, w))
    assert [int(v) for v in got.view(np.uint32)] == [b for _, b in f32]
    pw = torch.from_numpy(np.array([[a, b] for a, b, *_ in pairs], np.uint32).ravel().view(np.int32)).cuda()
    f64 = to_numpy(orand.map_words(orand.F64_UNIFORM, pw))
    assert np.array_equal(f64, np.array([p[2] for p in pairs]))
    z = to_numpy(orand.map_words(orand.F32_NORMAL, pw)).reshape(-1, 2)
    ref = np.array([[p[3], p[4]] for p in pairs])
    assert ulp_distance_f32(z.ravel(), ref.ravel()).max() <= 4


@pytest.mark.gpu
def test_gpu_matches_stored_walks(torch_cuda):
    import paper_2310_19925_b300 as orand

    w2, w3 = walk_rows()
    c2, c3 = WALK2D, WALK3D
    got2 = to_numpy(orand.brownian_walk(c2["n"], c2["steps"], c2["dt"], c2["D"], c2["seed"])).astype(np.float64)
    ref2 = np.array([w2[i] for i in range(c2["n"])])
    assert np.all(np.abs(got2 - ref2) <= 1e-5 * np.maximum(np.abs(ref2), 1.0))
    p = orand.walk3d_params(c3["n"], c3["steps"], dt=c3["dt"], mu=c3["mu"], sigma=c3["sigma"], k=2.0,
                            seed=c3["seed"], ckpt_every=c3["K"], p_first=c3["p_first"])
    xT, _, _ = orand.walk3d_forward(p)
    got3 = to_numpy(xT).astype(np.float64)
    ref3 = np.array([w3[c3["p_first"] + i] for i in range(c3["n"])])
    assert np.all(np.abs(got3 - ref3) <= 1e-5 * np.maximum(np.abs(ref3), 1.0))
