"""The paper's host micro-benchmark (§5, Performance Benchmarks).

Single-threaded generation time on the CPU for streams of varying length,
for every generator and for std::mt19937 (the GNU libstdc++ default engine
the paper measures against).  Each stream is a fresh generator (seed r,
counter 0) followed by `length` words, so construction is included: the
paper attributes mt19937's slowness on short streams to its initialisation.
The timing loop runs in C++ (``orand_host_microbench``).

    python -m paper_2310_19925_b300.host_bench
"""
from __future__ import annotations

import argparse
import json

LENGTHS = [1, 4, 16, 64, 256, 1024, 4096, 16384, 65536, 262144, 1048576]


def run(lengths=LENGTHS, words_per_length=1 << 22):
    import paper_2310_19925_b300 as orand
    from paper_2310_19925_b300 import workloads as W

    gens = [(W.GEN_NAMES[g], g) for g in (W.PHILOX, W.THREEFRY, W.SQUARES, W.TYCHE)] + [("mt19937",
                                                                                          orand.HOST_MT19937)]
    res = {"lengths": list(lengths), "ns_per_stream": {}, "ns_per_word": {}, "speedup_vs_mt19937": {}}
    for name, g in gens:
        ns = orand.host_microbench(g, lengths, words_per_length)
        res["ns_per_stream"][name] = [round(float(x), 2) for x in ns]
        res["ns_per_word"][name] = [round(float(x) / n, 3) for x, n in zip(ns, lengths)]
    mt = res["ns_per_stream"]["mt19937"]
    for name, _ in gens[:-1]:
        res["speedup_vs_mt19937"][name] = [round(m / x, 2) for m, x in zip(mt, res["ns_per_stream"][name])]
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--words", type=int, default=1 << 22, help="words drawn per length (stream count = words / length)")
    args = ap.parse_args(argv)
    print(json.dumps(run(words_per_length=args.words)))


if __name__ == "__main__":
    main()
