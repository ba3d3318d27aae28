"""Host-side failure injection and the persistent ragged tuning table, on the
GPU (a context needs a device).

* ORAND_FAIL_ALLOC=1 refuses every library allocation before the allocator
  runs: a context's first scratch growth (the walk adjoint's partials) and
  the ragged batcher's state and tables come back as ORAND_ERR_ALLOC, and the
  same context works once the switch is off.  Nothing is launched, so no
  device state is involved.
* The ragged autotuner's choices go to a file (ORAND_TUNE_CACHE) keyed by
  the GPU's name and the batch's size class: a second process reads it and
  does not tune, and writes the same bits.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2310_19925_b300 as orand
from paper_2310_19925_b300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_scratch_and_batch_allocation_failures(torch_cuda, monkeypatch, orc):
    torch = torch_cuda
    ctx = orand.Context()
    try:
        p = orand.walk3d_params(3000, 40, ckpt_every=8)
        xT, _, _ = orand.walk3d_forward(p, want_ckpt=False)
        dmu = torch.empty(3, dtype=torch.float64, device="cuda")
        dsig = torch.empty((), dtype=torch.float64, device="cuda")
        dx0 = torch.empty_like(xT)
        sh = torch.cuda.current_stream().cuda_stream
        args = (ctx.handle, p, xT.data_ptr(), 0, 0, dmu.data_ptr(), dsig.data_ptr(), 0, dx0.data_ptr(), sh)
        recs, total = W.ragged_requests(50, 10, list_seed=9)
        out = torch.zeros(total, dtype=torch.uint8, device="cuda")
        monkeypatch.setenv("ORAND_FAIL_ALLOC", "1")
        with pytest.raises(orand.OrandError) as e:
            orand.orand_walk3d_bwd(*args)                       # first scratch growth
        assert e.value.status == -4
        with pytest.raises(orand.OrandError) as e:
            orand.fill_ragged(recs, out=out, out_bytes=total, ctx=ctx)   # batcher state and tables
        assert e.value.status == -4
        monkeypatch.delenv("ORAND_FAIL_ALLOC")
        orand.orand_walk3d_bwd(*args)
        ref_dmu, ref_dsig, _ = orand.walk3d_backward(p, xT)
        orand.fill_ragged(recs, out=out, out_bytes=total, ctx=ctx)
        torch.cuda.synchronize()
        assert torch.equal(dmu, ref_dmu) and torch.equal(dsig, ref_dsig)
        host = out.cpu().numpy()
        r = recs[7]
        o, n = int(r["out_offset_bytes"]), int(r["length"])
        if int(r["dtype"]) == W.U32:
            assert np.array_equal(host[o:o + 4 * n].view(np.uint32),
                                  orc.fill(int(r["gen"]), 0, int(r["seed"]), int(r["counter"]), 1, n))
    finally:
        ctx.close()


_TUNE_CHILD = """
import json, sys, hashlib
import torch
import paper_2310_19925_b300 as orand
from paper_2310_19925_b300 import workloads as W
recs, total = W.ragged_requests(3000, 16, list_seed=21)
ctx = orand.Context()
out = torch.zeros(total, dtype=torch.uint8, device="cuda")
orand.fill_ragged(recs, out=out, out_bytes=total, ctx=ctx)
torch.cuda.synchronize()
st = orand.orand_ragged_stats(ctx.handle)
print(json.dumps({"tune_runs": st.tune_runs, "digest": hashlib.sha1(out.cpu().numpy().tobytes()).hexdigest()}))
"""


def test_tuning_table_persists_across_processes(torch_cuda, tmp_path):
    import json

    path = tmp_path / "sub" / "ragged_tune.txt"
    env = dict(os.environ, ORAND_TUNE_CACHE=str(path))
    env.pop("ORAND_AUTOTUNE", None)
    runs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", _TUNE_CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        runs.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert runs[0]["tune_runs"] > 0 and runs[1]["tune_runs"] == 0
    assert runs[0]["digest"] == runs[1]["digest"]
    lines = path.read_text().split("\n")
    assert len([ln for ln in lines if ln.strip()]) == 1
    name, lv, ln_, ty, bl, ch, sw, cps = lines[0].split()
    assert "B300" in name or name != "unknown"
    assert int(bl) in (128, 256, 512) and int(sw) in (8, 16)
