#!/usr/bin/env python
"""Benchmark of the counter-based generation hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl orand|reference]

One JSON line on rank 0.  `value` is the headline metric: Philox4x32-10 u32
bulk-fill throughput (GB/s of output written) on the 2^24-stream x 16-draw
workload (1 GiB per fill; far larger than the 126 MB L2, so no flush is
needed between launches).  A timed step is one pass over every hot-path row
that is built; each row is timed with CUDA events on the stream its kernels
run on, and the row table rides along in `rows`.

--impl reference times the CPU oracle (the plain C restatement of the
method) on the host cores for the same metric, on a bounded sample of the
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6400.0
# The headline kernel and every source file it is built from (its ncu traffic
# figure is used only while these are unchanged).
HEAD_KERNEL_KEY = "fill_tile_kernel<0,0,4>"
HEAD_KERNEL_SOURCES = ["paper_2310_19925_b300/csrc/fill.cu", "paper_2310_19925_b300/csrc/values.cuh",
                       "paper_2310_19925_b300/csrc/common.cuh", "include/orand_device.cuh"]
# The step's dominant kernel (about half of every step), reported as
# `roofline`, and the sources it is built from.
DOMINANT_KERNEL_KEY = "walk2d_kernel"
DOMINANT_KERNEL_SOURCES = ["paper_2310_19925_b300/csrc/walk.cu", "paper_2310_19925_b300/csrc/common.cuh",
                           "include/orand_device.cuh"]
METRIC = "Philox u32 fill GB/s vs HBM peak; walk particle-steps/s; adjoint vs plain walk"

# Issue peak of the integer/FP32 pipes: 148 SMs x 4 schedulers x 32 lanes x
# 2.032 GHz (the B300's unit counts and maximum SM clock), in lane-operations/s.
ALU_PEAK = 148 * 128 * 2.032e9
# Algorithmic work per particle-step, in scalar lane-operations: what one
# step needs when every operation is a scalar instruction (the count ncu
# measured for the scalar form of each kernel).  The kernels now issue the
# FP32 part of the walks' map as packed pairs (one f32x2 instruction does two
# of these operations), so they issue fewer instructions than this count;
# `frac` is the work rate against the issue peak, and `issue_frac` (from the
# committed ncu count of the current kernels) the share of issue slots used.
# 2D, per particle-step: the lane-instructions the scalar kernel needed
# per step, confirmed by ncu (at 2^20 x 1000): Philox4x32-10 with
# the two used words and the constant counter words folded (33), the walks'
# Box-Muller radius (u1 and v, the six-term series with its factor 2 folded
# in, the log2 and square-root estimates, the selection) and angle (the 22
# angle bits masked, converted and scaled, the sin and cos estimates with the
# multiply the compiler puts before them, swap and signs from w1's top bits)
# about 30 together, two FMA sums (2; the block sum is scaled by s once),
# and the Kahan add of each 16-step block sum and the unrolled loop's
# control (2).  This count is kept as the fixed unit of work per step: the
# angle now takes a half-turn split (the sign on the radius, no swap), which
# needs about five operations fewer, so `frac` counts the same work per step
# as before and rises with throughput, while `issue_frac` counts what the
# current kernel issues.
WALK2D_OPS_PER_STEP = 67
# The same per 3D particle-step, forward plus adjoint (ncu-confirmed;
# with the OU drift 112.6 + 123.3 by ncu): Philox with all four words, two radii, a
# cos/sin pair and a cosine, the products and sums (the constant-drift
# forward scales each block sum once; the OU forward scales every step); the
# OU forward adds the drift at the current position, the OU adjoint the
# recompute of x, the lambda decay and the three gradient sums.
WALK3D_OPS_PER_STEP = 102 + 101
WALK3D_OU_OPS_PER_STEP = 113 + 123
# The paper's macro-benchmark (FP64 Brownian dynamics): the fused kernel's
# 14 FP64 multiplies and adds per particle-step (Fig. 1 writes 18; the kicks'
# exact 2r - 1 is built from integer bits), against the FP64 pipe's nominal
# 1.25 TFLOP/s (an FMA counted as two) = 6.25e11 FP64 operations/s.
LANGEVIN_FP64_OPS_PER_STEP = 14
FP64_PEAK = 1.25e12 / 2


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["orand", "reference"], default="orand")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-baselines", action="store_true",
                    help="skip the comparison baselines (plain walk, serial ragged, cuRAND)")
    ap.add_argument("--only", default="", help="keep only rows whose name contains this text (profiling)")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def source_hash(paths):
    h = hashlib.sha1()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


# Issue peak in warp-instructions/s: 148 SMs x 4 schedulers x 2.032 GHz.
ISSUE_PEAK_WARP_INST = 148 * 4 * 2.032e9


def walk_issue_counts():
    """kernel key -> (source hash, lane-instructions per particle-step) from
    the committed ncu summary of the walk kernels."""
    p = os.path.join(ROOT, "profiles", "walk_issue.txt")
    out = {}
    if os.path.exists(p):
        for line in open(p):
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#"):
                out[parts[0]] = (parts[1], float(parts[2]))
    return out


def fill_issue_counts(src_hash):
    """Per (generator, dtype) of the 2^24 x 16 fill: (warp-instructions per
    launch, busiest pipe, its % of peak) from the committed ncu summary, if it
    was taken on the current sources of the fill kernels (else {})."""
    p = os.path.join(ROOT, "profiles", "fill_issue_2p24x16.txt")
    out = {}
    if not os.path.exists(p):
        return out
    for line in open(p):
        parts = line.split()
        if len(parts) >= 6 and not line.startswith("#") and parts[2] == src_hash:
            out[(int(parts[0]), int(parts[1]))] = (float(parts[3]), parts[4], float(parts[5]))
    return out


def ncu_traffic(kernel_key, src_hash):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel_key and parts[1] == src_hash:
            return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid):
        self.uuid = device_uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.uuid, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sms.append(float(f[0]))
                maxs.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxs) if maxs else None, "reasons": sorted(reasons),
                "samples": len(sms)}


# --------------------------------------------------------------------- rows --

class Row:
    """One hot-path row: `run(stream_handle)` launches its kernels on the
    given stream; `units` of `unit` are processed per run."""

    def __init__(self, name, run, units, unit, kernels, bytes_written=None):
        self.name, self.run, self.units, self.unit, self.kernels = name, run, units, unit, kernels
        self.bytes_written = bytes_written
        self.times_ms = []


def fill_rows(torch, orand, W, rank):
    rows = []
    c = W.FILL_LARGE
    n_streams, dps = c["n_streams"], c["dps"]
    first = rank * n_streams                 # rank r fills global streams [r*2^24, (r+1)*2^24)
    bufs = {}
    for dt in (W.U32, W.F32_UNIFORM, W.F64_UNIFORM, W.F32_NORMAL):
        bufs[dt] = torch.empty(n_streams * dps, dtype=orand.torch_dtype(dt), device="cuda")
    for gen in (W.PHILOX, W.THREEFRY, W.SQUARES, W.TYCHE):
        for dt in (W.U32, W.F32_UNIFORM, W.F64_UNIFORM, W.F32_NORMAL):
            out = bufs[dt]
            nbytes = out.numel() * out.element_size()

            def run(sh, gen=gen, dt=dt, out=out):
                orand.orand_fill_streams(gen, dt, c["seed"], c["counter"], first, n_streams, dps, out.data_ptr(), sh)

            row = Row("fill/%s/%s" % (W.GEN_NAMES[gen], W.DTYPE_NAMES[dt]), run, nbytes, "B", 1,
                      bytes_written=nbytes)
            row.gen, row.dtype = gen, dt
            rows.append(row)
    # The small Philox fill (2^16 streams x 64 draws, 16 MiB per dtype): it
    # stays in the 126 MB L2, so the launch's latency is what is measured.
    cs = W.FILL_SMALL
    s_first = rank * cs["n_streams"]
    for dt in (W.U32, W.F32_UNIFORM):
        out = torch.empty(cs["n_streams"] * cs["dps"], dtype=orand.torch_dtype(dt), device="cuda")
        bufs[("small", dt)] = out
        nbytes = out.numel() * out.element_size()

        def run_small(sh, dt=dt, out=out):
            orand.orand_fill_streams(W.PHILOX, dt, cs["seed"], cs["counter"], s_first, cs["n_streams"], cs["dps"],
                                     out.data_ptr(), sh)

        row = Row("fill_small/philox4x32_10/%s" % W.DTYPE_NAMES[dt], run_small, nbytes, "B", 1)
        row.extra = {"note": "16 MiB, L2-resident: launch latency, not HBM"}
        rows.append(row)
    return rows, bufs


def walk_rows(torch, orand, W, rank, world):
    """Fused 2D walk (particle-steps) and fused 3D forward + adjoint.  Rank r
    owns particles [r P, (r+1) P); the 3D loss is normalised by the global
    count, and with more than one rank the loss and scalar gradients are
    summed over ranks (one all-reduce of five or six doubles per row)."""
    from paper_2310_19925_b300 import shard

    rows = []
    keep = {}
    c2 = W.WALK2D
    P2 = c2["n_particles"]
    pos = torch.empty((P2, 2), dtype=torch.float32, device="cuda")
    keep["pos"] = pos
    prm2 = orand.walk2d_params(P2, c2["steps"], c2["dt"], c2["D"], c2["seed"], p_first=rank * P2)

    def run2(sh):
        orand.orand_brownian_walk(prm2, pos.data_ptr(), sh)

    rows.append(Row("walk2d/fused", run2, P2 * c2["steps"], "particle-steps", 1))

    c3 = W.WALK3D
    P3, T = c3["n_particles"], c3["steps"]
    prm3 = orand.walk3d_params(P3, T, c3["dt"], c3["mu"], c3["sigma"], c3["k"], c3["seed"], c3["ckpt_every"],
                               p_first=rank * P3, p_total=world * P3)
    ctx = orand.default_context().handle
    xT = torch.empty((P3, 3), dtype=torch.float32, device="cuda")
    ck = torch.empty((orand.n_checkpoints(T, c3["ckpt_every"]), P3, 3), dtype=torch.float32, device="cuda")
    loss = torch.empty((), dtype=torch.float64, device="cuda")
    dmu = torch.empty(3, dtype=torch.float64, device="cuda")
    dsig = torch.empty((), dtype=torch.float64, device="cuda")
    dx0 = torch.empty_like(xT)
    keep.update(xT=xT, ck=ck, loss=loss, dmu=dmu, dsig=dsig, dx0=dx0)

    def run3(sh):
        orand.orand_walk3d_fwd(ctx, prm3, 0, xT.data_ptr(), ck.data_ptr(), loss.data_ptr(), sh)
        orand.orand_walk3d_bwd(ctx, prm3, xT.data_ptr(), ck.data_ptr(), 0, dmu.data_ptr(), dsig.data_ptr(), 0,
                               dx0.data_ptr(), sh)
        if world > 1:
            shard.allreduce_walk_scalars(loss, dmu, dsig)

    rows.append(Row("walk3d/fused_fwd+adjoint", run3, P3 * T, "particle-steps", 5))

    # The same walk with drift mu - kappa x: the adjoint recomputes positions
    # backwards from the checkpoints and also returns dL/dkappa.
    co = W.WALK3D_OU
    prmo = orand.walk3d_params(P3, T, co["dt"], co["mu"], co["sigma"], co["k"], co["seed"], co["ckpt_every"],
                               p_first=rank * P3, p_total=world * P3, kappa=co["kappa"])
    dkap = torch.empty((), dtype=torch.float64, device="cuda")
    keep["dkap"] = dkap

    def run3ou(sh):
        orand.orand_walk3d_fwd(ctx, prmo, 0, xT.data_ptr(), ck.data_ptr(), loss.data_ptr(), sh)
        orand.orand_walk3d_bwd(ctx, prmo, xT.data_ptr(), ck.data_ptr(), 0, dmu.data_ptr(), dsig.data_ptr(),
                               dkap.data_ptr(), dx0.data_ptr(), sh)
        if world > 1:
            shard.allreduce_walk_scalars(loss, dmu, dsig, dkap)

    rows.append(Row("walk3d/ou_fused_fwd+adjoint", run3ou, P3 * T, "particle-steps", 6))
    return rows, keep


def ragged_rows(torch, orand, W, rank, world):
    """The 100,000-request ragged batch (about 30 GB of output) as one
    graph-launched persistent kernel.  With several ranks the list is split
    by the sharding helper (Tyche chains spread longest first, then bytes
    balanced), each rank serving its share into a buffer of its own."""
    import numpy as np

    from paper_2310_19925_b300 import shard

    recs, total = W.ragged_requests()
    if world > 1:
        recs, total, _ = shard.ragged_shard(recs, rank, world)
    out = torch.empty(total, dtype=torch.uint8, device="cuda")
    ctx = orand.default_context().handle
    values = int(recs["length"].sum())
    nbytes = int((recs["length"] * np.where(recs["dtype"] == 2, 8, 4).astype(np.uint64)).sum())

    def run(sh):
        orand.orand_fill_ragged(ctx, recs.ctypes.data, len(recs), out.data_ptr(), total, sh)

    row = Row("ragged/batched", run, values, "values", 1, bytes_written=nbytes)
    ty = recs["gen"] == W.TYCHE
    row.extra = {"requests": len(recs), "GB_out": round(nbytes / 1e9, 2),
                 "longest_tyche_values": int(recs["length"][ty].max()) if ty.any() else 0}
    return [row], {"ragged_out": out, "recs": recs}


def stream_test_rows(torch, orand, W, rank, n_words=1 << 30):
    """The parallel-stream battery (§5, Statistical Evaluation) per generator:
    16,000 particles x 3-word micro-streams, lengthened to about 2^30 words,
    generated and counted on the GPU.  Rank r tests the iterations after
    those of ranks 0..r-1."""
    from paper_2310_19925_b300 import stream_tests as ST

    rows, keep = [], []
    for gen in (W.PHILOX, W.THREEFRY, W.SQUARES, W.TYCHE):
        b = ST.Battery(gen, seed=0, n_words=n_words)
        b.counter_first = rank * b.n_iter
        keep.append(b)
        row = Row("stream_tests/%s" % W.GEN_NAMES[gen], lambda sh, b=b: b.launch(sh), b.words, "words",
                  b.kernels_per_launch)

        def finish(b=b):
            res = b.results()
            return {"p_values": {k: round(v["p"], 6) for k, v in res.items()},
                    "verdicts": sorted({v["verdict"] for v in res.values()})}

        row.finish = finish
        rows.append(row)
    return rows, keep


def curand_walk2d_baseline(torch, orand, W, reps=1):
    """cuRAND's Philox device API on the 2D walk at full size: the paper's
    Fig. 2 pattern (states and positions in HBM, one launch per step) and a
    fused form with the state in registers."""
    c2 = W.WALK2D
    P2, T = c2["n_particles"], c2["steps"]
    sh = torch.cuda.current_stream().cuda_stream
    prm = orand.walk2d_params(P2, T, c2["dt"], c2["D"], c2["seed"])
    states = torch.empty(P2 * orand.orand_walk2d_curand_state_bytes(), dtype=torch.uint8, device="cuda")
    pos = torch.empty((P2, 2), dtype=torch.float32, device="cuda")

    def timed(fn):
        ts = []
        for r in range(reps + 1):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            if r:
                ts.append(a.elapsed_time(b))
        return statistics.mean(ts)

    per_step = timed(lambda: (orand.orand_walk2d_curand_setup(prm, states.data_ptr(), pos.data_ptr(), 1984, sh),
                              orand.orand_walk2d_curand_run(prm, states.data_ptr(), pos.data_ptr(), sh)))
    fused = timed(lambda: orand.orand_walk2d_curand_fused(prm, pos.data_ptr(), 1984, sh))
    del states
    torch.cuda.empty_cache()
    return {"per_step_ms": round(per_step, 3), "fused_ms": round(fused, 3),
            "state_bytes": orand.orand_walk2d_curand_state_bytes(),
            "pattern": "cuRAND Philox: Fig. 2 (state in HBM, one launch per step) and fused (state in registers)"}


def stored_walk3d_baseline(torch, orand, W, reps=2, chunk=1 << 20):
    """The fused walk with stored noise (one forward launch that also writes
    z_t, one backward launch that reads it back), the other side of the
    regeneration trade-off, over particle chunks of 48 GiB of noise."""
    c3 = W.WALK3D
    P3, T = c3["n_particles"], c3["steps"]
    ctx = orand.default_context().handle
    sh = torch.cuda.current_stream().cuda_stream
    z = torch.empty((T, chunk, 3), dtype=torch.float32, device="cuda")
    xT = torch.empty((chunk, 3), dtype=torch.float32, device="cuda")
    loss = torch.empty((), dtype=torch.float64, device="cuda")
    dmu = torch.empty(3, dtype=torch.float64, device="cuda")
    dsig = torch.empty((), dtype=torch.float64, device="cuda")
    dx0 = torch.empty_like(xT)
    times, fwd_ms = [], []
    for r in range(reps + 1):
        a = torch.cuda.Event(enable_timing=True)
        m = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        f_ms = 0.0
        torch.cuda.synchronize()
        a.record()
        for c0 in range(0, P3, chunk):
            prm = orand.walk3d_params(chunk, T, c3["dt"], c3["mu"], c3["sigma"], c3["k"], c3["seed"], 0,
                                      p_first=c0, p_total=P3)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            orand.orand_walk3d_stored_fwd(ctx, prm, 0, xT.data_ptr(), z.data_ptr(), loss.data_ptr(), sh)
            e1.record()
            orand.orand_walk3d_stored_bwd(ctx, prm, xT.data_ptr(), z.data_ptr(), 0, dmu.data_ptr(), dsig.data_ptr(),
                                          dx0.data_ptr(), sh)
            torch.cuda.synchronize()
            f_ms += e0.elapsed_time(e1)
        b.record()
        torch.cuda.synchronize()
        if r:
            times.append(a.elapsed_time(b))
            fwd_ms.append(f_ms)
    del z
    torch.cuda.empty_cache()
    ms = statistics.mean(times)
    z_bytes = P3 * T * 12
    return {"ms": round(ms, 3), "fwd_ms": round(statistics.mean(fwd_ms), 3),
            "particle_steps_per_s": P3 * T / (ms * 1e-3),
            "pattern": "fused forward writing z (12 B per particle-step), fused backward reading it",
            "noise_bytes": z_bytes, "hbm_needed_GiB": round(z_bytes / 2**30, 1),
            "chunks": P3 // chunk}


def ragged_serial_baseline(torch, orand, W, n_sub=2000, reps=2):
    """One bulk-fill launch per request (in order, one stream) vs the batcher,
    on the first n_sub requests of the list (the full list's serial Tyche
    chains alone take about a minute one after another)."""
    import numpy as np

    recs, _ = W.ragged_requests()
    sub = recs[:n_sub].copy()
    end = int(sub["out_offset_bytes"][-1] + sub["length"][-1] * 8)
    out = torch.empty(end, dtype=torch.uint8, device="cuda")
    ctx = orand.default_context().handle
    sh = torch.cuda.current_stream().cuda_stream
    res = {}
    for name, fn in [("serial", lambda: orand.orand_fill_ragged_serial(sub.ctypes.data, len(sub), out.data_ptr(),
                                                                        end, sh)),
                     ("batched", lambda: orand.orand_fill_ragged(ctx, sub.ctypes.data, len(sub), out.data_ptr(),
                                                                 end, sh))]:
        ts = []
        for r in range(reps + 1):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            if r:
                ts.append(a.elapsed_time(b))
        res[name + "_ms"] = round(statistics.mean(ts), 3)
    res["requests"] = n_sub
    res["values"] = int(sub["length"].sum())
    res["batched_speedup"] = round(res["serial_ms"] / res["batched_ms"], 2)
    return res


def curand_reference(torch, n=1 << 28, reps=5):
    """cuRAND's Philox4_32_10 generator on the same GPU, through its public
    host API (device generation), for the bulk-fill sizes: GB/s per dtype."""
    import ctypes

    try:
        lib = ctypes.CDLL("libcurand.so")
    except OSError:
        try:
            lib = ctypes.CDLL("/usr/local/cuda/lib64/libcurand.so")
        except OSError as e:
            return {"unavailable": str(e)}
    gen = ctypes.c_void_p()
    if lib.curandCreateGenerator(ctypes.byref(gen), 161) != 0:
        return {"unavailable": "curandCreateGenerator failed"}
    lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(0x5EED))
    lib.curandSetStream(gen, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    res = {}
    cases = [("u32", torch.int32, lambda p: lib.curandGenerate(gen, p, ctypes.c_size_t(n))),
             ("f32_uniform", torch.float32, lambda p: lib.curandGenerateUniform(gen, p, ctypes.c_size_t(n))),
             ("f64_uniform", torch.float64, lambda p: lib.curandGenerateUniformDouble(gen, p, ctypes.c_size_t(n))),
             ("f32_normal", torch.float32, lambda p: lib.curandGenerateNormal(gen, p, ctypes.c_size_t(n),
                                                                             ctypes.c_float(0.0),
                                                                             ctypes.c_float(1.0)))]
    for name, dt, fn in cases:
        buf = torch.empty(n, dtype=dt, device="cuda")
        ptr = ctypes.c_void_p(buf.data_ptr())
        ts = []
        for r in range(reps + 1):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            st = fn(ptr)
            b.record()
            torch.cuda.synchronize()
            if st != 0:
                res[name] = {"error": int(st)}
                break
            if r:
                ts.append(a.elapsed_time(b))
        if ts:
            ms = statistics.mean(ts)
            res[name] = {"ms": round(ms, 4), "GB/s": round(n * buf.element_size() / (ms * 1e-3) / 1e9, 1)}
        del buf
    lib.curandDestroyGenerator(gen)
    torch.cuda.empty_cache()
    return res


def paper_brownian_benchmark(torch, orand, n=1_000_000, steps=10_000, reps=2):
    """The paper's §5 macro-benchmark on this GPU: 10^6 particles x 10^4
    steps of 2D Brownian dynamics with drag and FP64 uniform kicks, in the
    paper's OpenRAND pattern (Fig. 1: one launch per step, generator built
    in-thread), its cuRAND pattern (Fig. 2: per-particle state set up once,
    loaded and stored every step), and this library's fused kernel."""
    prm = orand.langevin2d_params(n)
    sh = torch.cuda.current_stream().cuda_stream
    ps = orand.particles_tensor(n)
    states = torch.empty(n * orand.orand_langevin2d_curand_state_bytes(), dtype=torch.uint8, device="cuda")
    runs = {
        "openrand_pattern_per_step": lambda: (orand.orand_langevin2d_init(prm, ps.data_ptr(), sh),
                                              orand.orand_langevin2d_run_per_step(prm, ps.data_ptr(), 1, steps, sh)),
        "curand_pattern_per_step": lambda: (orand.orand_langevin2d_curand_setup(prm, ps.data_ptr(), states.data_ptr(),
                                                                                1984, sh),
                                            orand.orand_langevin2d_curand_run(prm, ps.data_ptr(), states.data_ptr(),
                                                                              steps, sh)),
        "fused": lambda: (orand.orand_langevin2d_init(prm, ps.data_ptr(), sh),
                          orand.orand_langevin2d_fused(prm, ps.data_ptr(), 1, steps, sh)),
    }
    res = {"particles": n, "steps": steps, "precision": "fp64"}
    for name, fn in runs.items():
        ts = []
        for r in range(reps + 1):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            if r:
                ts.append(a.elapsed_time(b))
        res[name + "_ms"] = round(statistics.mean(ts), 3)
    res["curand_over_openrand_pattern"] = round(res["curand_pattern_per_step_ms"] /
                                                res["openrand_pattern_per_step_ms"], 3)
    res["curand_over_fused"] = round(res["curand_pattern_per_step_ms"] / res["fused_ms"], 3)
    res["paper_reports"] = "OpenRAND 1.8x faster than cuRAND on V100/A100 (paper §5)"
    del states, ps
    torch.cuda.empty_cache()
    return res


def plain_walk3d_baseline(torch, orand, W, reps=2, chunk=1 << 20):
    """The plain noise-storing walk (one launch per step, z stored in forward
    and read back in backward), run over particle chunks so that the stored
    noise of one chunk (steps x chunk x 3 floats = 48 GiB) fits in HBM."""
    c3 = W.WALK3D
    P3, T = c3["n_particles"], c3["steps"]
    ctx = orand.default_context().handle
    sh = torch.cuda.current_stream().cuda_stream
    z = torch.empty((T, chunk, 3), dtype=torch.float32, device="cuda")
    x = torch.empty((chunk, 3), dtype=torch.float32, device="cuda")
    loss = torch.empty((), dtype=torch.float64, device="cuda")
    dmu = torch.empty(3, dtype=torch.float64, device="cuda")
    dsig = torch.empty((), dtype=torch.float64, device="cuda")
    dx0 = torch.empty_like(x)
    times = []
    launches = 0
    for r in range(reps + 1):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for c0 in range(0, P3, chunk):
            prm = orand.walk3d_params(chunk, T, c3["dt"], c3["mu"], c3["sigma"], c3["k"], c3["seed"], 0,
                                      p_first=c0, p_total=P3)
            orand.orand_walk3d_plain_fwd(ctx, prm, 0, x.data_ptr(), z.data_ptr(), loss.data_ptr(), sh)
            orand.orand_walk3d_plain_bwd(ctx, prm, x.data_ptr(), z.data_ptr(), 0, dmu.data_ptr(), dsig.data_ptr(),
                                         dx0.data_ptr(), sh)
            launches += (1 + T + 2) + (T + 3)
        b.record()
        torch.cuda.synchronize()
        if r:
            times.append(a.elapsed_time(b))
    del z
    torch.cuda.empty_cache()
    ms = statistics.mean(times)
    return {"ms": round(ms, 3), "particle_steps_per_s": P3 * T / (ms * 1e-3),
            "pattern": "one launch per step, noise stored (%d GiB per %d-particle chunk)" % (
                T * chunk * 12 >> 30, chunk),
            "launches_per_run": launches // (reps + 1)}


# ---------------------------------------------------------------- reference --

def cpu_oracle_fill_rate(threads, n_streams=1 << 24, dps=16):
    """Oracle Philox u32 fill on `threads` host threads: returns (GB/s, seconds, sample)."""
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    out = oracle.fill(0, 0, 0x5EED, 0, n_streams, dps, threads=threads)
    dt = time.perf_counter() - t0
    return out.nbytes / dt / 1e9, dt, ("philox4x32_10 u32, %d streams x %d draws (%d MiB), seed 0x5EED, "
                                       "counter 0, on %d host threads" % (n_streams, dps, out.nbytes >> 20, threads))


def cpu_oracle_row_rates(threads):
    """The oracle on bounded samples of the other rows' workloads, for context
    beside their GPU rates (a few seconds in all).  Walks step in FP64."""
    import oracle
    from paper_2310_19925_b300 import workloads as W

    oracle.build()
    rates = {}
    n2, t2 = 1 << 14, W.WALK2D["steps"]
    t0 = time.perf_counter()
    oracle.walk2d(0, n2, t2, W.WALK2D["dt"], W.WALK2D["D"], threads=threads)
    dt = time.perf_counter() - t0
    rates["walk2d/fused"] = {"particle-steps_per_s": n2 * t2 / dt, "cores": threads,
                             "sample": "%d particles x %d steps (FP64)" % (n2, t2)}
    c3 = W.WALK3D
    n3, t3 = 1 << 12, c3["steps"]
    t0 = time.perf_counter()
    xT, _ = oracle.walk3d_forward(0, n3, t3, c3["ckpt_every"], c3["dt"], c3["mu"], c3["sigma"], want_ckpt=True,
                                  threads=threads)
    oracle.walk3d_adjoint(0, n3, t3, c3["dt"], xT, c3["k"], float(n3), threads=threads)
    dt = time.perf_counter() - t0
    rates["walk3d/fused_fwd+adjoint"] = {"particle-steps_per_s": n3 * t3 / dt, "cores": threads,
                                         "sample": "%d particles x %d steps, forward + adjoint (FP64)" % (n3, t3)}
    recs, _ = W.ragged_requests()
    sub = recs[:200]
    t0 = time.perf_counter()
    oracle.ragged(sub)
    dt = time.perf_counter() - t0
    rates["ragged/batched"] = {"values_per_s": int(sub["length"].sum()) / dt, "cores": 1,
                               "sample": "the first 200 requests (%d values), one thread" % int(sub["length"].sum())}
    return rates


def run_reference(args, rank, world):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    vals = []
    for _ in range(max(args.warmup, 0)):
        cpu_oracle_fill_rate(threads, n_streams=1 << 18)
    t_total = 0.0
    sample = None
    for _ in range(args.steps):
        v, dt, sample = cpu_oracle_fill_rate(threads, n_streams=1 << 22)
        vals.append(v)
        t_total += dt
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "philox4x32_10 u32 bulk fill, seed 0x5EED, counter 0, 16 draws per stream; "
                               "CPU oracle on a 2^22-stream sample (the first quarter) of the 2^24-stream "
                               "workload per step"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# -------------------------------------------------------------------- main --

def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    import paper_2310_19925_b300 as orand
    from paper_2310_19925_b300 import workloads as W

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    orand._lib()
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    frows, _keep = fill_rows(torch, orand, W, rank)
    head = frows[0]  # fill/philox4x32_10/u32: the headline kernel
    wrows, _wkeep = walk_rows(torch, orand, W, rank, world)
    rrows, _rkeep = ragged_rows(torch, orand, W, rank, world)
    srows, _skeep = stream_test_rows(torch, orand, W, rank)
    # Step order: walks, ragged batch, stream tests, then the fills with the
    # headline Philox u32 fill last, right after the Philox f32 fill, so that
    # it runs behind a kernel of its own kind rather than behind the 30 GB batch.
    rows = wrows + rrows + srows + frows[::-1]
    if args.only:
        rows = [r for r in rows if args.only in r.name]
        if head not in rows:
            rows.insert(0, head)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        for r in rows:
            r.run(sh)
    barrier()

    props = torch.cuda.get_device_properties(local_rank)
    sampler = ClockSampler("GPU-" + str(props.uuid)) if hasattr(props, "uuid") else ClockSampler("0")
    sampler.start()
    time.sleep(0.3)
    ev = []
    step_start = torch.cuda.Event(enable_timing=True)
    step_end = torch.cuda.Event(enable_timing=True)
    barrier()
    step_start.record()
    for _ in range(args.steps):
        for r in rows:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            r.run(sh)
            b.record()
            ev.append((r, a, b))
    step_end.record()
    barrier()
    clocks = sampler.stop()
    for r, a, b in ev:
        r.times_ms.append(a.elapsed_time(b))
    total_ms = step_start.elapsed_time(step_end)

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    head_ms = max_over_ranks(statistics.mean(head.times_ms))
    ms_per_step = max_over_ranks(total_ms / args.steps)
    value = world * head.units / (head_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    achieved = head.bytes_written / (statistics.mean(head.times_ms) * 1e-3) / 1e9
    src = source_hash(HEAD_KERNEL_SOURCES)
    traffic = ncu_traffic(HEAD_KERNEL_KEY, src)

    row_table = {}
    step_ms = total_ms / args.steps
    for r in rows:
        t = max_over_ranks(statistics.mean(r.times_ms))
        e = {"ms": round(t, 4), r.unit + "_per_s": world * r.units / (t * 1e-3),
             "share_of_step": round(statistics.mean(r.times_ms) / step_ms, 4)}
        if r.bytes_written:
            e["GB/s"] = round(world * r.bytes_written / (t * 1e-3) / 1e9, 1)
            e["frac_hbm"] = round(r.bytes_written / (t * 1e-3) / 1e9 / peak, 4)
        e.update(getattr(r, "extra", {}))
        if hasattr(r, "finish"):
            e.update(r.finish())
        row_table[r.name] = e

    # Per-kernel rooflines beside the headline: the step's dominant kernels
    # (the 2D walk, and the 3D walks' forward + adjoint pairs; issue-bound)
    # against the issue peak.
    rooflines = {}
    walk_src = source_hash(DOMINANT_KERNEL_SOURCES)
    walk_issue = walk_issue_counts()

    def issued(key, rate):
        h, per_step = walk_issue.get(key, (None, None))
        if h != walk_src or per_step is None:
            return None, None
        return per_step, per_step * rate / ALU_PEAK

    for row, key, opc in [("walk2d/fused", "walk2d_kernel", WALK2D_OPS_PER_STEP),
                          ("walk3d/fused_fwd+adjoint", "walk3d_fwd_kernel<0>+walk3d_bwd_kernel<0>", WALK3D_OPS_PER_STEP),
                          ("walk3d/ou_fused_fwd+adjoint", "walk3d_fwd_kernel<1>+walk3d_bwd_kernel<1>",
                           WALK3D_OU_OPS_PER_STEP)]:
        w = row_table.get(row)
        if w:
            rate = w["particle-steps_per_s"] / world
            ops = rate * opc
            per_step, ifrac = issued(key, rate)
            rooflines[key] = {"bound": "alu", "achieved": ops, "peak": ALU_PEAK, "unit": "lane-ops/s",
                              "frac": ops / ALU_PEAK, "ops_per_particle_step": opc,
                              "ops_kind": "fixed unit of work per particle-step (the scalar kernel's instruction "
                                          "count for one Philox block, the Box-Muller map and the sums); "
                                          "issue_frac counts the instructions the current kernel issues",
                              "issued_lane_instructions_per_particle_step": per_step, "issue_frac": ifrac,
                              "share_of_step": w["share_of_step"],
                              "peak_kind": "derived: 148 SMs x 128 lanes x 2.032 GHz"}
    # The headline metric's kernel: the Philox u32 fill against the measured
    # copy bandwidth, with its ncu DRAM traffic.
    rooflines["fill_tile_kernel<philox,u32>"] = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
        "traffic": traffic, "share_of_step": row_table[head.name]["share_of_step"],
        "kernel": "fill_tile_kernel<philox4x32_10, u32, R=4, whole rows> (swizzled tile, TMA tensor store)",
        "peak_kind": peak_kind + " (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)"}
    # Every fill of the 2^24 x 16 workload against both of its bounds: the
    # measured copy bandwidth (bytes written) and the issue peak (its ncu
    # warp-instruction count per launch over the event-timed duration), with
    # the busiest pipe from the same capture.  The larger fraction names the
    # bound.
    issue = fill_issue_counts(source_hash(HEAD_KERNEL_SOURCES))
    for r in rows:
        if not hasattr(r, "gen"):
            continue
        t_s = statistics.mean(r.times_ms) * 1e-3
        gbs = r.bytes_written / t_s / 1e9
        e = {"kernel": "fill_tile_kernel<%s,%s>" % (W.GEN_NAMES[r.gen], W.DTYPE_NAMES[r.dtype]),
             "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak},
             "share_of_step": row_table[r.name]["share_of_step"]}
        if (r.gen, r.dtype) in issue:
            inst, pipe, pct = issue[(r.gen, r.dtype)]
            e["issue"] = {"achieved": inst / t_s, "peak": ISSUE_PEAK_WARP_INST, "unit": "warp-instructions/s",
                          "frac": inst / t_s / ISSUE_PEAK_WARP_INST, "warp_instructions_per_launch": inst,
                          "busiest_pipe": pipe, "busiest_pipe_pct_of_peak": pct,
                          "peak_kind": "derived: 148 SMs x 4 schedulers x 2.032 GHz"}
            e["bound"] = "hbm" if e["hbm"]["frac"] >= e["issue"]["frac"] else "issue"
        else:
            e["issue"] = None
            e["bound"] = "hbm"
        rooflines["fill/%s/%s" % (W.GEN_NAMES[r.gen], W.DTYPE_NAMES[r.dtype])] = e
    # `roofline`: the dominant kernel of the step, the 2D walk (issue-bound),
    # with the DRAM bytes of one launch from ncu (the 2^24 positions; the
    # steps move no memory).
    dominant = None
    if "walk2d_kernel" in rooflines:
        dominant = dict(rooflines["walk2d_kernel"])
        dominant.update(traffic=ncu_traffic(DOMINANT_KERNEL_KEY, source_hash(DOMINANT_KERNEL_SOURCES)),
                        kernel="walk2d_kernel (fused 2D Brownian walk, 2^24 particles x 10^4 steps per launch)",
                        algorithmic_bytes=8 * W.WALK2D["n_particles"])

    # End to end through the C ABI: the same fill, then the 1 GiB result read
    # back into pinned host memory, both inside the timed region.
    host = torch.empty(head.bytes_written // 4, dtype=torch.int32, pin_memory=True)
    dev_out = _keep[W.U32]
    e2e_ms = []
    for i in range(max(2, min(args.steps, 5)) + 1):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        head.run(sh)
        host.copy_(dev_out, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        if i:
            e2e_ms.append(a.elapsed_time(b))
    e2e_t = max_over_ranks(statistics.mean(e2e_ms))
    e2e = {"value": world * head.bytes_written / (e2e_t * 1e-3) / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": head.bytes_written}

    baselines = {}
    if not args.only and not args.no_baselines and world == 1:
        fused = row_table.get("walk3d/fused_fwd+adjoint")
        plain = plain_walk3d_baseline(torch, orand, W)
        if fused:
            plain["fused_speedup"] = round(plain["ms"] / fused["ms"], 3)
        baselines["walk3d/plain_noise_storing_fwd+bwd"] = plain
        stored = stored_walk3d_baseline(torch, orand, W)
        if fused:
            stored["regenerating_ms"] = fused["ms"]
            stored["regenerating_over_stored"] = round(fused["ms"] / stored["ms"], 3)
        baselines["walk3d/fused_noise_storing_fwd+bwd"] = stored
        baselines["ragged/one_launch_per_request_first2000"] = ragged_serial_baseline(torch, orand, W)
        baselines["curand_philox4_32_10_2^28_values"] = curand_reference(torch)
        cw = curand_walk2d_baseline(torch, orand, W)
        w2 = row_table.get("walk2d/fused")
        if w2:
            cw["orand_fused_ms"] = w2["ms"]
            cw["curand_fused_over_orand"] = round(cw["fused_ms"] / w2["ms"], 3)
            cw["curand_per_step_over_orand"] = round(cw["per_step_ms"] / w2["ms"], 3)
        baselines["walk2d/curand_2^24x10^4"] = cw
        baselines["paper_brownian_dynamics_1e6x1e4"] = mb = paper_brownian_benchmark(torch, orand)
        # The macro-benchmark's fused kernel against the FP64 pipe that bounds it.
        ops = mb["particles"] * mb["steps"] * LANGEVIN_FP64_OPS_PER_STEP / (mb["fused_ms"] * 1e-3)
        rooflines["langevin_fused_kernel"] = {"bound": "fp64", "achieved": ops, "peak": FP64_PEAK,
                                              "unit": "FP64 ops/s", "frac": ops / FP64_PEAK,
                                              "ops_per_particle_step": LANGEVIN_FP64_OPS_PER_STEP,
                                              "peak_kind": "nominal: 1.25 TFLOP/s FP64 with FMA as two"}
        from paper_2310_19925_b300 import host_bench

        hb = host_bench.run()
        hb["note"] = "paper §5 host micro-benchmark: one host thread, fresh generator per stream, vs std::mt19937"
        baselines["host_microbench_ns_per_word"] = {"lengths": hb["lengths"], **hb["ns_per_word"],
                                                    "speedup_vs_mt19937": hb["speedup_vs_mt19937"],
                                                    "note": hb["note"]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        v, dt, sample = cpu_oracle_fill_rate(threads)
        cpu = {"value": v, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": sample}
        # The same oracle on samples of the walk and ragged rows, with the
        # GPU row's rate over it (context: the oracle is deliberately plain).
        cpu["rows"] = cpu_oracle_row_rates(threads)
        for name, r in cpu["rows"].items():
            unit = "particle-steps_per_s" if "particle-steps_per_s" in r else "values_per_s"
            if name in row_table and unit in row_table[name]:
                r["gpu_over_oracle"] = row_table[name][unit] / world / r[unit]

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "philox4x32_10 u32 bulk fill, 2^24 streams x 16 draws per rank (1 GiB), "
                                   "key = stream id ^ 0x5EED, counter 0",
                       "step": "one pass over every built hot-path row (%d rows)" % len(rows),
                       "l2": "every output >= 1 GiB, larger than the 126 MB L2: no flush between launches",
                       "parallelism": "dp%d (disjoint stream ranges per rank)" % world},
            "roofline": dominant if dominant is not None else rooflines["fill_tile_kernel<philox,u32>"],
            "rooflines": rooflines,
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": sum(r.kernels for r in rows) * args.steps,
            "rows": row_table,
            "baselines": baselines,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
