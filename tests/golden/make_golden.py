"""Write the stored expected values under tests/golden/ from the CPU oracle.

The paper prints no known-answer values for its generators or maps, so the
fixtures here come from the oracle alone (this script imports nothing but
``oracle`` and numpy).  They freeze the oracle's outputs: a later change to
its arithmetic shows up as a fixture mismatch on the CPU
(``tests/test_golden.py``), and the GPU path is checked against the stored
values without running the oracle (``-m gpu`` tests in the same file).

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

GEN_NAMES = {0: "philox4x32_10", 1: "threefry4x32_20", 2: "squares32", 3: "tyche"}

# Stream keys: seed 0x5EED with stream ids 0, 1 and 2^24 - 1 (the fill
# workload's first, second and last streams), and keys using all 64 bits.
KEYS = (0x5EED, 0x5EED ^ 1, 0x5EED ^ (2**24 - 1), 0x0123456789ABCDEF, 2**64 - 1)
COUNTERS = (0, 1, 2**32 - 1)
N_WORDS = 16

# Word-map inputs: edge cases of each map, then seeded random words.
EDGE_WORDS = (0x00000000, 0x000000FF, 0x00000100, 0x000FFFFF, 0x00100000, 0x7FFFFFFF, 0x80000000,
              0xBFFFFF00, 0xC0000000, 0xFFFFFEFF, 0xFFFFFF00, 0xFFFFFFFF)
N_RANDOM_WORDS = 52

WALK2D = dict(seed=0x77, n=8, steps=37, dt=float(np.float32(1e-3)), D=1.0, p_first=0)
WALK3D = dict(seed=0, n=6, steps=65, K=16, dt=float(np.float32(1e-3)), mu=(0.1, -0.2, 0.05), sigma=0.5,
              p_first=3)


def header(f, lines):
    for ln in lines:
        f.write("# " + ln + "\n")


def write_streams(path):
    with open(path, "w") as f:
        header(f, [
            "First 16 words of the stream (generator, key64, counter): the generators the paper",
            "names (§3; Philox4x32-10 and Threefry4x32-20 after Salmon et al. 2011, Squares after",
            "Widynski 2020, Tyche after Neves & Araujo 2011), a stream being a 64-bit key and a",
            "32-bit counter (§3).  Written by tests/golden/make_golden.py from the oracle.",
            "columns: generator key64 counter w0 .. w15 (hex)",
        ])
        for gen in sorted(GEN_NAMES):
            for key in KEYS:
                for ctr in COUNTERS:
                    w = oracle.stream_words(gen, key, ctr, 0, N_WORDS)
                    f.write("%s %016x %08x %s\n" % (GEN_NAMES[gen], key, ctr, " ".join("%08x" % int(v) for v in w)))


def map_inputs():
    rng = np.random.default_rng(20231030)
    rnd = rng.integers(0, 2**32, N_RANDOM_WORDS, dtype=np.uint64).astype(np.uint32)
    return np.concatenate([np.array(EDGE_WORDS, np.uint32), rnd])


def write_maps(path):
    w = map_inputs()
    pairs = w.reshape(-1, 2)
    f32 = oracle.map_words(oracle.F32_UNIFORM, w)
    f64 = oracle.map_words(oracle.F64_UNIFORM, w)
    z = oracle.box_muller_array(pairs[:, 0], pairs[:, 1])
    with open(path, "w") as f:
        header(f, [
            "Word -> value maps of the fills (§4, Fig. 1 and Fig. 3 draw helpers): FP32 uniform",
            "(w >> 8) 2^-24; FP64 uniform ((hi:lo) >> 11) 2^-53 from a word pair, first word high;",
            "Box-Muller of a word pair (u1 = ((w0 >> 8) + 1) 2^-24, u2 = (w1 >> 8) 2^-24), in FP64.",
            "Written by tests/golden/make_golden.py from the oracle.",
            "f32 lines: word, FP32 bit pattern of the uniform (exact in FP32).",
            "pair lines: w0 w1, FP64 uniform as a hex float, z0 z1 as hex floats (FP64).",
        ])
        for x, u in zip(w, f32):
            f.write("f32 %08x %08x\n" % (int(x), int(np.float32(u).view(np.uint32))))
        for (a, b), d, (z0, z1) in zip(pairs, f64, z):
            f.write("pair %08x %08x %s %s %s\n" % (int(a), int(b), float(d).hex(), float(z0).hex(), float(z1).hex()))


def write_walks(path):
    c2, c3 = WALK2D, WALK3D
    x0, xT = oracle.walk2d(c2["seed"], c2["n"], c2["steps"], c2["dt"], c2["D"], p_first=c2["p_first"])
    yT, _ = oracle.walk3d_forward(c3["seed"], c3["n"], c3["steps"], c3["K"], c3["dt"], c3["mu"], c3["sigma"],
                                  p_first=c3["p_first"])
    with open(path, "w") as f:
        header(f, [
            "Walk end positions in FP64 (§5's Brownian walk; the per-step counter convention of",
            "Fig. 1: start from counter 0, step t from counter t; 3D noise z_t from counter t + 1).",
            "walk2d: seed 0x77, particles 0..7, 37 steps, dt = fl32(1e-3), D = 1.",
            "walk3d: seed 0, particles 3..8, 65 steps, checkpoints every 16, dt = fl32(1e-3),",
            "mu = (0.1, -0.2, 0.05), sigma = 0.5.",
            "Written by tests/golden/make_golden.py from the oracle.",
        ])
        for i in range(c2["n"]):
            f.write("walk2d %d %s %s\n" % (c2["p_first"] + i, float(xT[i, 0]).hex(), float(xT[i, 1]).hex()))
        for i in range(c3["n"]):
            f.write("walk3d %d %s\n" % (c3["p_first"] + i, " ".join(float(v).hex() for v in yT[i])))


def main():
    oracle.build()
    write_streams(os.path.join(HERE, "stream_words.txt"))
    write_maps(os.path.join(HERE, "value_maps.txt"))
    write_walks(os.path.join(HERE, "walk_positions.txt"))


if __name__ == "__main__":
    main()
