"""Run one hot-path case a few times at a chosen size (profiling and timing).

    python -m paper_2310_19925_b300.cases fill --gen 0 --dtype 0 --streams 16777216 --dps 16
    python -m paper_2310_19925_b300.cases fill --gen -1 --dtype -1     (every generator x dtype)
    python -m paper_2310_19925_b300.cases walk2d --particles 1048576 --steps 1000
    python -m paper_2310_19925_b300.cases walk3d --particles 1048576 --steps 512
    python -m paper_2310_19925_b300.cases ragged --requests 2000 --max-log2 20
    python -m paper_2310_19925_b300.cases tyche-chain --dtype 3 --length 1048576
    python -m paper_2310_19925_b300.cases langevin --form fused --particles 1000000 --steps 100

Each case launches its kernels `--reps` times on the current stream.  Every
launch is timed with CUDA events, and one line per case is printed with the
mean time and the case's own throughput unit.  The ragged cases queue 100 ms
of GPU work before each timed call, so the host's planning of the batch
overlaps it and the events measure GPU time.  The sizes are free, so an ncu
capture can target one kernel at a small size (`-k`, `-c`).
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np


def timed(torch, fn, reps, busy_ms=0.0):
    """Event-timed launches.  busy_ms > 0 first queues that much GPU work
    (torch.cuda._sleep), so host-side preparation inside fn (the ragged
    batch's planning) overlaps it, as it does in a step with work queued
    ahead, and the events measure GPU time only."""
    ts = []
    for _ in range(reps):
        if busy_ms > 0:
            torch.cuda._sleep(int(busy_ms * 1e-3 * 2.0e9))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return ts


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["fill", "walk2d", "walk3d", "ragged", "tyche-chain", "langevin"])
    ap.add_argument("--gen", type=int, default=0, help="fill: generator, -1 for all four in turn")
    ap.add_argument("--dtype", type=int, default=0, help="fill: dtype, -1 for all four in turn")
    ap.add_argument("--streams", type=int, default=1 << 24)
    ap.add_argument("--dps", type=int, default=16)
    ap.add_argument("--particles", type=int, default=1 << 20)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--max-log2", type=int, default=20)
    ap.add_argument("--length", type=int, default=1 << 20)
    ap.add_argument("--kappa", type=float, default=0.0, help="walk3d: OU drift mu - kappa x")
    ap.add_argument("--form", choices=["fused", "per-step", "curand"], default="fused",
                    help="langevin: the fused kernel, Fig. 1's launch per step, or Fig. 2's cuRAND pattern")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)

    import torch

    import paper_2310_19925_b300 as orand
    from paper_2310_19925_b300 import workloads as W

    sh = torch.cuda.current_stream().cuda_stream
    res = {"case": args.case}
    if args.case == "fill" and (args.gen < 0 or args.dtype < 0):
        # Every requested (generator, dtype) in turn, one line each; the
        # launches run in this order, so an ncu capture of `-c 16` sees one
        # launch per combination at --reps 1.
        gens = range(4) if args.gen < 0 else [args.gen]
        dts = range(4) if args.dtype < 0 else [args.dtype]
        for g in gens:
            for d in dts:
                main(["fill", "--gen", str(g), "--dtype", str(d), "--streams", str(args.streams),
                      "--dps", str(args.dps), "--reps", str(args.reps)])
        return
    if args.case == "fill":
        out = torch.empty(args.streams * args.dps, dtype=orand.torch_dtype(args.dtype), device="cuda")
        fn = lambda: orand.orand_fill(args.gen, args.dtype, 0x5EED, 0, args.streams, args.dps, out.data_ptr(), sh)
        ts = timed(torch, fn, args.reps)
        nbytes = out.numel() * out.element_size()
        res.update(gen=args.gen, dtype=args.dtype, streams=args.streams, dps=args.dps,
                   ms=statistics.mean(ts), GBps=nbytes / (statistics.mean(ts) * 1e-3) / 1e9)
        del out
    elif args.case == "walk2d":
        pos = torch.empty((args.particles, 2), dtype=torch.float32, device="cuda")
        prm = orand.walk2d_params(args.particles, args.steps)
        ts = timed(torch, lambda: orand.orand_brownian_walk(prm, pos.data_ptr(), sh), args.reps)
        res.update(particles=args.particles, steps=args.steps, ms=statistics.mean(ts),
                   particle_steps_per_s=args.particles * args.steps / (statistics.mean(ts) * 1e-3))
    elif args.case == "walk3d":
        prm = orand.walk3d_params(args.particles, args.steps, kappa=args.kappa)
        ctx = orand.default_context().handle
        dk = torch.empty((), dtype=torch.float64, device="cuda")
        xT = torch.empty((args.particles, 3), dtype=torch.float32, device="cuda")
        ck = torch.empty((orand.n_checkpoints(args.steps, 64), args.particles, 3), dtype=torch.float32,
                         device="cuda")
        loss = torch.empty((), dtype=torch.float64, device="cuda")
        g = torch.empty(4, dtype=torch.float64, device="cuda")
        dx0 = torch.empty_like(xT)

        def fn():
            orand.orand_walk3d_fwd(ctx, prm, 0, xT.data_ptr(), ck.data_ptr(), loss.data_ptr(), sh)
            orand.orand_walk3d_bwd(ctx, prm, xT.data_ptr(), ck.data_ptr(), 0, g.data_ptr(), g.data_ptr() + 24,
                                   dk.data_ptr() if args.kappa else 0, dx0.data_ptr(), sh)

        ts = timed(torch, fn, args.reps)
        res.update(particles=args.particles, steps=args.steps, kappa=args.kappa, ms=statistics.mean(ts),
                   particle_steps_per_s=args.particles * args.steps / (statistics.mean(ts) * 1e-3))
    elif args.case == "langevin":
        # The paper's macro-benchmark (FP64 Brownian dynamics); setup is untimed.
        prm = orand.langevin2d_params(args.particles)
        ps = orand.particles_tensor(args.particles)
        st = torch.empty(args.particles * orand.orand_langevin2d_curand_state_bytes(), dtype=torch.uint8,
                         device="cuda")
        if args.form == "curand":
            orand.orand_langevin2d_curand_setup(prm, ps.data_ptr(), st.data_ptr(), 1984, sh)
            fn = lambda: orand.orand_langevin2d_curand_run(prm, ps.data_ptr(), st.data_ptr(), args.steps, sh)
        else:
            orand.orand_langevin2d_init(prm, ps.data_ptr(), sh)
            run = orand.orand_langevin2d_fused if args.form == "fused" else orand.orand_langevin2d_run_per_step
            fn = lambda: run(prm, ps.data_ptr(), 1, args.steps, sh)
        ts = timed(torch, fn, args.reps)
        res.update(form=args.form, particles=args.particles, steps=args.steps, ms=statistics.mean(ts),
                   particle_steps_per_s=args.particles * args.steps / (statistics.mean(ts) * 1e-3))
    elif args.case in ("ragged", "tyche-chain"):
        if args.case == "ragged":
            recs, total = W.ragged_requests(args.requests, args.max_log2)
        else:
            recs = np.zeros(1, W.REQUEST_DTYPE)
            recs[0] = (W.TYCHE, args.dtype, 1, 7, 0, args.length, 0)
            total = args.length * W.ELEM_BYTES[args.dtype]
        out = torch.empty(max(total, 16), dtype=torch.uint8, device="cuda")
        ctx = orand.default_context().handle
        fn = lambda: orand.orand_fill_ragged(ctx, recs.ctypes.data, len(recs), out.data_ptr(), total, sh)
        fn()  # first call tunes its size class
        torch.cuda.synchronize()
        ts = timed(torch, fn, args.reps, busy_ms=100.0)
        values = int(recs["length"].sum())
        res.update(requests=len(recs), values=values, ms=statistics.mean(ts),
                   values_per_s=values / (statistics.mean(ts) * 1e-3),
                   config=orand.orand_ragged_get_config(ctx).__class__.__name__)
        c = orand.orand_ragged_get_config(ctx)
        res["config"] = dict(block=c.block, chunk_values=c.chunk_values, store_bytes=c.store_bytes)
        if args.case == "tyche-chain":
            res["ns_per_value"] = statistics.mean(ts) * 1e6 / max(values, 1)
    res["times_ms"] = [round(t, 4) for t in ts]
    print(json.dumps(res))


if __name__ == "__main__":
    main()
