"""The allocation-free adjoint, orand_walk3d_bwd_noalloc.

Some callers must not allocate device memory.  A host framework may own the
whole device-memory budget, a memory cap may make a new allocation fail
mid-run, or the code may be too latency-sensitive for the device-wide
synchronisation of cudaMalloc/cudaFree.  For them the library offers the
walk adjoint with its reduction scratch in a fixed device array.  These
tests call it through the C ABI and hold its gradients to those of the
context-based adjoint (orand_walk3d_bwd).  Both run the same kernels and the
same fixed-order reduction, so the header promises the same bits and the
tests ask for exact equality (well inside the 1e-3 gradient tolerance of the
other walk tests).  The calls come back to back, so each reuses the
shared array right after the previous call left its contents there, and a
request past the array's fixed limit is refused before anything runs.
"""
import ctypes

import pytest

import paper_2310_19925_b300 as orand

MAX_PARTICLES = 1 << 22


def test_size_limit_is_refused_on_the_host():
    lib = orand._lib()
    p = orand.walk3d_params(MAX_PARTICLES + 1, 8)
    assert lib.orand_walk3d_bwd_noalloc(ctypes.byref(p), 16, None, None, 16, 16, None, None, None) == -8
    assert "ORAND_ERR_SCRATCH_LIMIT" in lib.orand_status_string(-8).decode()


@pytest.mark.gpu
def test_noalloc_adjoint_matches_context_adjoint_on_consecutive_calls():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sh = torch.cuda.current_stream().cuda_stream
    # Largest first, then smaller: a later call must not pick up partials a
    # larger earlier call left behind in the shared array.
    calls = [(MAX_PARTICLES, 16, 1.0, 0), (1 << 16, 64, 0.75, 12345), (4096 + 77, 96, -2.0, 999)]
    for n, steps, g, p_first in calls:
        p = orand.walk3d_params(n, steps, p_first=p_first, p_total=3 * n)
        xT, _, _ = orand.walk3d_forward(p, want_ckpt=False)
        gl = torch.tensor(g, dtype=torch.float64, device="cuda")
        ref_dmu, ref_dsig, ref_dx0 = orand.walk3d_backward(p, xT, gl)
        dmu = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        dsig = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        dx0 = torch.full_like(xT, float("nan"))
        orand.orand_walk3d_bwd_noalloc(p, xT.data_ptr(), 0, gl.data_ptr(), dmu.data_ptr(), dsig.data_ptr(), 0,
                                       dx0.data_ptr(), sh)
        torch.cuda.synchronize()
        assert torch.equal(dmu, ref_dmu), (n, dmu, ref_dmu)
        assert torch.equal(dsig, ref_dsig), (n, dsig, ref_dsig)
        assert torch.equal(dx0, ref_dx0), n


@pytest.mark.gpu
def test_noalloc_adjoint_with_ou_drift_and_dkappa():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sh = torch.cuda.current_stream().cuda_stream
    p = orand.walk3d_params(5000, 100, ckpt_every=16, kappa=3.0)
    xT, ck, _ = orand.walk3d_forward(p)
    ref_dmu, ref_dsig, ref_dk, ref_dx0 = orand.walk3d_backward_full(p, xT, ck)
    dmu = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    dsig = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    dk = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    dx0 = torch.full_like(xT, float("nan"))
    orand.orand_walk3d_bwd_noalloc(p, xT.data_ptr(), ck.data_ptr(), 0, dmu.data_ptr(), dsig.data_ptr(),
                                   dk.data_ptr(), dx0.data_ptr(), sh)
    torch.cuda.synchronize()
    assert torch.equal(dmu, ref_dmu) and torch.equal(dsig, ref_dsig) and torch.equal(dk, ref_dk)
    assert torch.equal(dx0, ref_dx0)
