"""Parallel-stream correlation tests on the GPU (§5, Statistical Evaluation).

The paper checks its generators on parallel streams the way HOOMD-blue does
(Anderson et al. 2020): 16,000 particles each draw a micro-stream of three
numbers per iteration, the micro-streams are concatenated, and the stream
is lengthened over the iterations.  This module builds that stream on the
GPU, chunk by chunk, with ``orand_fill_micro_streams`` and accumulates the
counts of a small battery of classical tests (``orand_stat_*``; Knuth,
TAOCP vol. 2, §3.3.2).  Only the final p-values are computed on the host,
from a few thousand integer counts.

    python -m paper_2310_19925_b300.stream_tests --gen 0 --words 1073741824

Chunks hold a whole number of iterations, a multiple of 32 of them, so
every tuple (stride 1, 2 or 3) and every 4096-word birthday sample falls
where it would in the unchunked stream; the gap test carries its open run
from chunk to chunk.  The counts are therefore those of the whole stream.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

# The battery: (name, kind, parameters).
BATTERY = (
    ("freq_hi8", "tuples", dict(t=1, bits=8, shift=24, stride=1)),
    ("freq_lo8", "tuples", dict(t=1, bits=8, shift=0, stride=1)),
    ("pairs_hi6", "tuples", dict(t=2, bits=6, shift=26, stride=2)),
    ("triples_hi4", "tuples", dict(t=3, bits=4, shift=28, stride=3)),
    ("gaps_1_16", "gaps", dict(lo=0, hi=1 << 28, t_max=64)),
    ("birthday_4096_2p32", "birthday", dict(log2_n=12, bits=32, shift=0, r_max=64)),
)

FAIL_P = 1e-10   # p beyond this on either side is a failure (TestU01's convention)


def _chi2_p(observed, expected):
    """Pearson chi-square with bins of expected count < 5 merged into their neighbour."""
    from scipy import stats

    obs, exp = [], []
    o_acc = e_acc = 0.0
    for o, e in zip(observed, expected):
        o_acc += float(o)
        e_acc += float(e)
        if e_acc >= 5.0:
            obs.append(o_acc)
            exp.append(e_acc)
            o_acc = e_acc = 0.0
    if e_acc > 0 and exp:
        obs[-1] += o_acc
        exp[-1] += e_acc
    if len(exp) < 2:
        return float("nan"), 0, float("nan")
    obs, exp = np.array(obs), np.array(exp)
    stat = float(((obs - exp) ** 2 / exp).sum())
    dof = len(exp) - 1
    return stat, dof, float(stats.chi2.sf(stat, dof))


def expected_probabilities(kind, prm):
    """Cell probabilities of the tuple and gap tests for a perfect generator."""
    if kind == "tuples":
        cells = 1 << (prm["t"] * prm["bits"])
        return np.full(cells, 1.0 / cells)
    if kind == "gaps":
        p = (prm["hi"] - prm["lo"]) / 2.0**32
        t = prm["t_max"]
        return np.array([p * (1 - p) ** r for r in range(t)] + [(1 - p) ** t])
    raise ValueError(kind)


def birthday_mean(log2_n, bits):
    """E[R] per sample for n = 2^log2_n birthdays in m = 2^bits days.

    The n spacings are m times a uniform point of the simplex, so two given
    spacings are equal with probability close to (n - 1) / (2 m) and three
    with probability close to (n - 1)(n - 2) / (3 m^2).  Equal pairs number
    n (n - 1)^2 / (4 m) on average (Knuth's n^3 / (4 m) to first order).  R
    counts equal neighbours after sorting, so a value shared by k spacings
    adds k - 1 to R but k (k - 1) / 2 to the pairs: triples take one off
    each, n (n - 1)^2 (n - 2)^2 / (18 m^2) of them on average.  Larger
    coincidences are smaller by a further factor n^2 / m."""
    n, m = float(1 << log2_n), float(2 ** bits)
    pairs = n * (n - 1) ** 2 / (4 * m)
    triples = n * (n - 1) ** 2 * (n - 2) ** 2 / (18 * m * m)
    return pairs - triples


def evaluate(kind, prm, counts):
    """p-value and verdict from a test's counts.  Tuples and gaps: Pearson
    chi-square against the exact cell probabilities (two-sided: a fit too
    good to be true fails as well).  Birthday spacings: the total Y of R
    over the N samples against Poisson(N E[R]), two-sided (TestU01's form of
    the test; the distribution of R itself is only close to Poisson, not
    close enough for the bin-by-bin test at 10^6 samples)."""
    from scipy import stats

    counts = np.asarray(counts, dtype=np.float64)
    total = counts.sum()
    if kind == "birthday":
        y = float(np.dot(np.arange(counts.size), counts))
        mu = total * birthday_mean(prm["log2_n"], prm["bits"])
        p = float(min(1.0, 2 * min(stats.poisson.cdf(y, mu), stats.poisson.sf(y - 1, mu)))) if total else float("nan")
        return {"samples": int(total), "Y": y, "mean": mu, "p": p,
                "verdict": "fail" if (p < FAIL_P or counts[-1] > 0) else "pass"}
    stat, dof, p = _chi2_p(counts, expected_probabilities(kind, prm) * total)
    return {"samples": int(total), "chi2": stat, "dof": dof, "p": p,
            "verdict": "fail" if (p < FAIL_P or p > 1 - FAIL_P) else "pass"}


class Battery:
    """The battery over one generator's concatenated micro-stream of about
    n_words words (whole iterations), with its buffers allocated once.
    launch() enqueues the whole run on a stream (counts reset first);
    results() waits for it and evaluates the counts."""

    def __init__(self, gen, seed=0, n_particles=16000, draws=3, n_words=1 << 30, chunk_iterations=1024,
                 counter_first=0, battery=BATTERY):
        import torch

        self.gen, self.seed, self.n_particles, self.draws = gen, seed, n_particles, draws
        self.counter_first, self.battery = counter_first, battery
        self.per_iter = n_particles * draws
        self.n_iter = max(1, n_words // self.per_iter)
        self.words = self.n_iter * self.per_iter
        self.chunk = max(32, chunk_iterations - chunk_iterations % 32)
        self.buf = torch.empty(min(self.n_iter, self.chunk) * self.per_iter, dtype=torch.int32, device="cuda")
        self.counts = {}
        for name, kind, prm in battery:
            size = (1 << (prm["t"] * prm["bits"])) if kind == "tuples" else (
                prm["t_max"] + 1 if kind == "gaps" else prm["r_max"] + 1)
            self.counts[name] = torch.zeros(size, dtype=torch.int64, device="cuda")
        self.carry = {name: torch.full((1,), -1, dtype=torch.int64, device="cuda")
                      for name, kind, _ in battery if kind == "gaps"}
        # library kernels per launch(): per chunk one generator launch, one
        # per tuple test, three per gap test, one per birthday test
        per_chunk = 1 + sum({"tuples": 1, "gaps": 3, "birthday": 1}[k] for _, k, _ in battery)
        self.kernels_per_launch = per_chunk * -(-self.n_iter // self.chunk)

    def launch(self, stream=None):
        """Enqueue the run on `stream`: a torch stream, or None / a raw
        handle of the current stream."""
        import torch

        import paper_2310_19925_b300 as orand

        with torch.cuda.stream(stream) if isinstance(stream, torch.cuda.Stream) else _nullcontext():
            for c in self.counts.values():
                c.zero_()
            for c in self.carry.values():
                c.fill_(-1)
        done = 0
        while done < self.n_iter:
            it = min(self.chunk, self.n_iter - done)
            w = self.buf[: it * self.per_iter]
            orand.fill_micro_streams(self.gen, self.seed, self.n_particles, self.draws, self.counter_first + done,
                                     it, out=w, stream=stream)
            for name, kind, prm in self.battery:
                c = self.counts[name]
                if kind == "tuples":
                    orand.stat_tuples(w, prm["t"], prm["bits"], prm["shift"], prm["stride"], c, stream)
                elif kind == "gaps":
                    orand.stat_gaps(w, prm["lo"], prm["hi"], prm["t_max"], c, self.carry[name], stream)
                else:
                    orand.stat_birthday(w, prm["log2_n"], prm["bits"], prm["shift"], prm["r_max"], c, stream)
            done += it

    def results(self):
        import torch

        torch.cuda.synchronize()
        out = {}
        for name, kind, prm in self.battery:
            c = self.counts[name].cpu().numpy().astype(np.uint64)
            out[name] = dict(evaluate(kind, prm, c), kind=kind, **prm)
            out[name]["counts"] = c
        return out


class _nullcontext:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def run(gen, seed=0, n_particles=16000, draws=3, n_words=1 << 30, chunk_iterations=1024, counter_first=0,
        stream=None, battery=BATTERY):
    """Generate and test the concatenated micro-stream of about n_words words
    (whole iterations).  Returns (results per test, timing)."""
    import torch

    b = Battery(gen, seed, n_particles, draws, n_words, chunk_iterations, counter_first, battery)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.launch(stream)
    ev1.record(stream)
    res = b.results()
    gpu_ms = ev0.elapsed_time(ev1)
    timing = {"words": b.words, "iterations": b.n_iter, "gpu_ms": gpu_ms, "wall_s": time.perf_counter() - t0,
              "words_per_s": b.words / (gpu_ms * 1e-3)}
    return res, timing


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gen", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--words", type=int, default=1 << 30)
    ap.add_argument("--particles", type=int, default=16000)
    ap.add_argument("--draws", type=int, default=3)
    args = ap.parse_args(argv)
    res, timing = run(args.gen, args.seed, args.particles, args.draws, args.words)
    out = {"gen": args.gen, "timing": timing}
    out["tests"] = {k: {kk: vv for kk, vv in v.items() if kk != "counts"} for k, v in res.items()}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
