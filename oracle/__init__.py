"""CPU oracle for the counter-based generation hot path (OpenRAND, arXiv 2310.19925).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2310_19925_b300``) never does and shares no code with it.

The arithmetic lives in ``orand_oracle.c`` (plain C, FP64 for floating point),
compiled with gcc into ``liborand_oracle.so`` next to it; this module only
marshals numpy arrays through ctypes.  ctypes releases the GIL during foreign
calls, so ``fill(..., threads=N)`` runs N plain C loops side by side over
disjoint stream ranges (a timing convenience, no change to the arithmetic).

Each function names the passage it follows; the generator definitions come
from the publications the paper cites for them (§3): Philox/Threefry (Salmon
et al. 2011), Squares (Widynski 2020), Tyche (Neves & Araujo 2011).
Parity unpinned: the Threefry4x32-20 round function and the Squares round
order (no outside implementation to compare against in this environment).
The Squares key derivation (MurmurHash3's 64-bit finaliser) is pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orand_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborand_oracle.so")

PHILOX, THREEFRY, SQUARES, TYCHE = 0, 1, 2, 3
U32, F32_UNIFORM, F64_UNIFORM, F32_NORMAL = 0, 1, 2, 3
GENERATORS = (PHILOX, THREEFRY, SQUARES, TYCHE)
DTYPES = (U32, F32_UNIFORM, F64_UNIFORM, F32_NORMAL)


def build(force: bool = False) -> str:
    """Compile orand_oracle.c with gcc (no fast-math) into liborand_oracle.so."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_threefry4x32_20.argtypes = [u32p, u32p, u32p]
        L.orc_squares32.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_squares32.restype = ctypes.c_uint32
        L.orc_squares_key.argtypes = [ctypes.c_uint64]
        L.orc_squares_key.restype = ctypes.c_uint64
        L.orc_tyche_mix.argtypes = [u32p]
        L.orc_tyche_init.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u32p]
        L.orc_stream_words.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_uint64, u32p]
        L.orc_stream_words.restype = ctypes.c_int
        L.orc_f32_uniform.argtypes = [ctypes.c_uint32]
        L.orc_f32_uniform.restype = ctypes.c_double
        L.orc_f64_uniform.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.orc_f64_uniform.restype = ctypes.c_double
        L.orc_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, dp]
        L.orc_box_muller_array.argtypes = [u32p, u32p, ctypes.c_uint64, dp]
        L.orc_map_words.argtypes = [ctypes.c_int, u32p, ctypes.c_uint64, ctypes.c_void_p]
        L.orc_map_words.restype = ctypes.c_int
        L.orc_fill.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                               ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                               ctypes.c_void_p, u32p]
        L.orc_fill.restype = ctypes.c_int
        L.orc_walk2d.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                 ctypes.c_float, ctypes.c_float, dp, dp]
        L.orc_langevin2d.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.orc_walk3d_ou_forward.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_float, fp, ctypes.c_float, ctypes.c_float,
                                            dp, dp, dp, dp]
        L.orc_walk3d_ou_adjoint.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_float, ctypes.c_float, dp, ctypes.c_double, ctypes.c_double,
                                            dp, dp, dp, dp]
        L.orc_walk3d_init.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, dp]
        L.orc_walk3d_forward.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_uint32, ctypes.c_uint32, ctypes.c_float, fp,
                                         ctypes.c_float, dp, dp, dp]
        L.orc_walk3d_loss.argtypes = [dp, ctypes.c_uint64, ctypes.c_double, ctypes.c_double]
        L.orc_walk3d_loss.restype = ctypes.c_double
        L.orc_walk3d_adjoint.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_uint32, ctypes.c_float, dp, ctypes.c_double,
                                         ctypes.c_double, dp, dp, dp]
        _lib = L
    return _lib


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u32arr(vals, n):
    a = np.ascontiguousarray(np.asarray(vals, dtype=np.uint64) & 0xFFFFFFFF, dtype=np.uint32)
    assert a.shape == (n,)
    return a


# --- generator cores (§3: Philox, Threefry, Squares, Tyche) -----------------

def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (Salmon et al. 2011): 4 counter words, 2 key words."""
    c, k, o = _u32arr(ctr, 4), _u32arr(key, 2), np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_u32p(c), _u32p(k), _u32p(o))
    return [int(v) for v in o]


def threefry4x32_20(ctr, key):
    """One Threefry4x32-20 block (Salmon et al. 2011): 4 counter words, 4 key words."""
    c, k, o = _u32arr(ctr, 4), _u32arr(key, 4), np.zeros(4, np.uint32)
    lib().orc_threefry4x32_20(_u32p(c), _u32p(k), _u32p(o))
    return [int(v) for v in o]


def squares32(ctr: int, key: int) -> int:
    """Squares, 32-bit output, 4 rounds (Widynski 2020)."""
    return int(lib().orc_squares32(ctr & (2**64 - 1), key & (2**64 - 1)))


def squares_key(key64: int) -> int:
    """Per-stream Squares key: fmix64(key64) | 1 (a reading: the paper's
    library takes 32-bit seeds for Squares)."""
    return int(lib().orc_squares_key(key64 & (2**64 - 1)))


def tyche_mix(state):
    """One Tyche MIX (the ChaCha quarter-round) on (a, b, c, d)."""
    s = _u32arr(state, 4)
    lib().orc_tyche_mix(_u32p(s))
    return [int(v) for v in s]


def tyche_init(key64: int, counter: int):
    """Tyche state after seeding (a=hi, b=lo, c=2654435769, d=1367130551^counter) and 20 MIX."""
    s = np.zeros(4, np.uint32)
    lib().orc_tyche_init(key64 & (2**64 - 1), counter & 0xFFFFFFFF, _u32p(s))
    return [int(v) for v in s]


def stream_words(gen: int, key64: int, counter: int, first: int, n: int) -> np.ndarray:
    """Words [first, first+n) of the stream (gen, key64, counter)."""
    out = np.zeros(max(n, 1), np.uint32)
    rc = lib().orc_stream_words(gen, key64 & (2**64 - 1), counter & 0xFFFFFFFF, first, n, _u32p(out))
    if rc != 0:
        raise ValueError("oracle: bad generator or word range")
    return out[:n]


# --- maps (§4 Fig. 1 / Fig. 3 draw helpers) ---------------------------------

def f32_uniform(w: int) -> float:
    return float(lib().orc_f32_uniform(w & 0xFFFFFFFF))


def f64_uniform(hi: int, lo: int) -> float:
    return float(lib().orc_f64_uniform(hi & 0xFFFFFFFF, lo & 0xFFFFFFFF))


def box_muller(w0: int, w1: int):
    z = np.zeros(2, np.float64)
    lib().orc_box_muller(w0 & 0xFFFFFFFF, w1 & 0xFFFFFFFF, _dp(z))
    return float(z[0]), float(z[1])


def box_muller_array(w0, w1) -> np.ndarray:
    """Box-Muller of word pairs: returns (n, 2) float64."""
    a = np.ascontiguousarray(w0, np.uint32)
    b = np.ascontiguousarray(w1, np.uint32)
    z = np.zeros((len(a), 2), np.float64)
    lib().orc_box_muller_array(_u32p(a), _u32p(b), len(a), _dp(z))
    return z


def map_words(dtype: int, words) -> np.ndarray:
    """Apply a dtype's word->value map to a word array (uint32 or float64 out)."""
    w = np.ascontiguousarray(words, np.uint32)
    n = len(w) // 2 if dtype == F64_UNIFORM else len(w)
    out = np.zeros(n, np.uint32 if dtype == U32 else np.float64)
    if n and lib().orc_map_words(dtype, _u32p(w), n, out.ctypes.data_as(ctypes.c_void_p)) != 0:
        raise ValueError("oracle: bad dtype")
    return out


def words_for(dtype: int, dps: int) -> int:
    if dtype == F64_UNIFORM:
        return 2 * dps
    if dtype == F32_NORMAL:
        return 2 * ((dps + 1) // 2)
    return dps


# --- bulk fill (§3: one stream per processing element) ----------------------

def _fill_range(gen, dtype, seed, counter, s_first, n_streams, dps, out):
    scratch = np.zeros(max(words_for(dtype, dps), 1), np.uint32)
    rc = lib().orc_fill(gen, dtype, seed & (2**64 - 1), counter & 0xFFFFFFFF, s_first, n_streams, dps,
                        out.ctypes.data_as(ctypes.c_void_p), _u32p(scratch))
    if rc != 0:
        raise ValueError("oracle: bad fill arguments")


def fill(gen: int, dtype: int, seed: int, counter: int, n_streams: int, dps: int,
         s_first: int = 0, threads: int = 1) -> np.ndarray:
    """Stream-major fill: out[i*dps + j] = value j of stream s_first+i (key64 = seed ^ s).

    Returns uint32 for U32, float64 for the float dtypes (FP32 uniforms exact,
    normals unrounded FP64)."""
    out = np.zeros(n_streams * dps, np.uint32 if dtype == U32 else np.float64)
    if n_streams * dps == 0:
        return out
    threads = max(1, min(threads, n_streams))
    if threads == 1:
        _fill_range(gen, dtype, seed, counter, s_first, n_streams, dps, out)
        return out
    bounds = np.linspace(0, n_streams, threads + 1).astype(np.int64)
    with ThreadPoolExecutor(threads) as ex:
        futs = [ex.submit(_fill_range, gen, dtype, seed, counter, s_first + int(a), int(b - a), dps,
                          out[int(a) * dps:int(b) * dps]) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        for f in futs:
            f.result()
    return out


def ragged(requests) -> list:
    """Ragged batch: each request (gen, dtype, seed, counter, length) is the
    single stream key64 = seed (stream id 0), i.e. fill(..., n_streams=1).
    A request is a 5-tuple in that order or a record with those field names
    (the batcher's request layout has more fields)."""
    out = []
    for r in requests:
        names = getattr(getattr(r, "dtype", None), "names", None)
        if names:
            g, d, s, c, n = (int(r[k]) for k in ("gen", "dtype", "seed", "counter", "length"))
        else:
            g, d, s, c, n = (int(x) for x in r[:5])
        out.append(fill(g, d, s, c, 1, n))
    return out


# --- walks (§4 Fig. 1 structure; §5 macro-benchmark) -------------------------

def _split(n, threads):
    threads = max(1, min(threads, n))
    b = np.linspace(0, n, threads + 1).astype(np.int64)
    return [(int(x), int(y)) for x, y in zip(b[:-1], b[1:]) if y > x]


def walk2d(seed: int, n: int, steps: int, dt: float, D: float, p_first: int = 0, threads: int = 1):
    """FP64 2D Brownian walk of particles p_first..p_first+n-1; returns (x0, xT), each (n, 2)."""
    x0 = np.zeros((n, 2), np.float64)
    xT = np.zeros((n, 2), np.float64)

    def run(a, b):
        lib().orc_walk2d(seed, p_first + a, b - a, steps, dt, D, _dp(x0[a:b]), _dp(xT[a:b]))

    parts = _split(n, threads)
    if len(parts) <= 1:
        for a, b in parts:
            run(a, b)
    else:
        with ThreadPoolExecutor(len(parts)) as ex:
            for f in [ex.submit(run, a, b) for a, b in parts]:
                f.result()
    return x0, xT


def langevin2d(seed, n, steps, dt=1e-3, gamma=1.0, mass=1.0, p_first=0, threads=1):
    """The paper's FP64 Brownian-dynamics benchmark (Fig. 1): returns (n, 4) = x, y, vx, vy."""
    st = np.zeros((n, 4), np.float64)

    def run(a, b):
        lib().orc_langevin2d(seed, p_first + a, b - a, steps, dt, gamma, mass, _dp(st[a:b]))

    parts = _split(n, threads)
    if len(parts) <= 1:
        for a, b in parts:
            run(a, b)
    else:
        with ThreadPoolExecutor(len(parts)) as ex:
            for f in [ex.submit(run, a, b) for a, b in parts]:
                f.result()
    return st


def walk3d_init(seed: int, n: int, p_first: int = 0) -> np.ndarray:
    x0 = np.zeros((n, 3), np.float64)
    lib().orc_walk3d_init(seed, p_first, n, _dp(x0))
    return x0


def walk3d_forward(seed, n, steps, K, dt, mu, sigma, x0=None, p_first=0, want_ckpt=False, threads=1):
    """FP64 3D drift walk; returns (xT (n,3), ckpt (ceil(steps/K), n, 3) or None)."""
    xT = np.zeros((n, 3), np.float64)
    n_ck = (steps + K - 1) // K if K else 0
    ck = np.zeros((n_ck, n, 3), np.float64) if want_ckpt else None
    mu_a = (ctypes.c_float * 3)(*[float(m) for m in mu])
    x0c = None if x0 is None else np.ascontiguousarray(x0, np.float64)

    def run(a, b):
        ck_part = None
        if ck is not None:
            ck_part = np.zeros((n_ck, b - a, 3), np.float64)
        lib().orc_walk3d_forward(seed, p_first + a, b - a, steps, K, dt, mu_a, sigma,
                                 None if x0c is None else _dp(x0c[a:b]), _dp(xT[a:b]),
                                 None if ck_part is None else _dp(ck_part))
        if ck is not None:
            ck[:, a:b, :] = ck_part

    parts = _split(n, threads)
    if len(parts) <= 1:
        for a, b in parts:
            run(a, b)
    else:
        with ThreadPoolExecutor(len(parts)) as ex:
            for f in [ex.submit(run, a, b) for a, b in parts]:
                f.result()
    return xT, ck


def walk3d_loss(xT: np.ndarray, k: float, P: float) -> float:
    xT = np.ascontiguousarray(xT, np.float64)
    return float(lib().orc_walk3d_loss(_dp(xT), xT.shape[0], k, P))


def walk3d_adjoint(seed, n, steps, dt, xT, k, P, p_first=0, threads=1):
    """Stepped reverse-mode adjoint; returns (dmu (3,), dsigma, dx0 (n,3))."""
    xT = np.ascontiguousarray(xT, np.float64)
    dx0 = np.zeros((n, 3), np.float64)
    parts = _split(n, threads)
    partial = []

    def run(a, b):
        dmu = np.zeros(3, np.float64)
        ds = np.zeros(1, np.float64)
        lib().orc_walk3d_adjoint(seed, p_first + a, b - a, steps, dt, _dp(xT[a:b]), k, P,
                                 _dp(dmu), _dp(ds), _dp(dx0[a:b]))
        return dmu, float(ds[0])

    if len(parts) <= 1:
        partial = [run(a, b) for a, b in parts]
    else:
        with ThreadPoolExecutor(len(parts)) as ex:
            partial = [f.result() for f in [ex.submit(run, a, b) for a, b in parts]]
    dmu = np.sum([p[0] for p in partial], axis=0) if partial else np.zeros(3)
    dsig = float(np.sum([p[1] for p in partial])) if partial else 0.0
    return dmu, dsig, dx0


def walk3d_ou_forward(seed, n, steps, K, dt, mu, sigma, kappa, x0=None, p_first=0, want_ckpt=False):
    """FP64 3D walk with drift mu - kappa x; returns (xT (n,3), ckpt or None, xs (steps+1, n, 3))."""
    xT = np.zeros((n, 3), np.float64)
    n_ck = (steps + K - 1) // K if K else 0
    ck = np.zeros((n_ck, n, 3), np.float64) if want_ckpt else None
    xs = np.zeros((steps + 1, n, 3), np.float64)
    mu_a = (ctypes.c_float * 3)(*[float(m) for m in mu])
    x0c = None if x0 is None else np.ascontiguousarray(x0, np.float64)
    lib().orc_walk3d_ou_forward(seed, p_first, n, steps, K, dt, mu_a, sigma, kappa,
                                None if x0c is None else _dp(x0c), _dp(xT), None if ck is None else _dp(ck), _dp(xs))
    return xT, ck, xs


def walk3d_ou_adjoint(seed, n, steps, dt, kappa, xs, k, P, p_first=0):
    """Stepped adjoint of the OU walk; returns (dmu (3,), dsigma, dkappa, dx0 (n,3))."""
    xs = np.ascontiguousarray(xs, np.float64)
    dmu = np.zeros(3, np.float64)
    ds = np.zeros(1, np.float64)
    dk = np.zeros(1, np.float64)
    dx0 = np.zeros((n, 3), np.float64)
    lib().orc_walk3d_ou_adjoint(seed, p_first, n, steps, dt, kappa, _dp(xs), k, P, _dp(dmu), _dp(ds), _dp(dk),
                                _dp(dx0))
    return dmu, float(ds[0]), float(dk[0]), dx0
