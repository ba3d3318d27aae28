"""GPU parity of the walk kernels against the FP64 CPU oracle.

Bars: walk positions |gpu - oracle| <= 1e-5 * max(|oracle|, 1) (FP32 with
compensated summation vs FP64); initial positions bit-exact; loss and
gradients within 1e-3 relative (they come out near 1e-6).  Full-size
workloads (2^24 x 10^4 2D, 2^22 x 4096 3D) run in the benchmark's launch
configuration and are checked on sampled particles, on particle-range
subsets, and by properties that hold at any size.
"""
import math

import numpy as np
import pytest

from helpers import to_numpy

import paper_2310_19925_b300 as orand
from paper_2310_19925_b300 import workloads as W

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5
GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def pos_close(gpu, ref, scale=1.0):
    """|gpu - ref| <= POS_TOL * max(|ref|, scale): relative, with the floor at
    the walk's own length scale (1 for the benchmark walks, whose steps are
    below it; s sqrt(steps) for walks of larger steps, where positions that
    end near 0 are sums that cancelled)."""
    err = np.abs(gpu.astype(np.float64) - ref)
    bound = POS_TOL * np.maximum(np.abs(ref), scale)
    assert np.all(err <= bound), "worst %.3g (bound %.3g)" % ((err / bound).max(), POS_TOL)


# ------------------------------------------------------------------- 2D ----

@pytest.mark.parametrize("steps", [0, 1, 31, 32, 37, 64, 1000])
@pytest.mark.parametrize("p_first", [0, 2**40 + 5])
def test_walk2d_small(torch_cuda, orc, steps, p_first):
    n = 1000
    f32 = lambda v: float(np.float32(v))
    got = to_numpy(orand.brownian_walk(n, steps, dt=1e-3, D=1.0, seed=0x77, p_first=p_first))
    x0, xT = orc.walk2d(0x77, n, steps, f32(1e-3), 1.0, p_first=p_first, threads=8)
    if steps == 0:
        assert np.array_equal(got.astype(np.float64), x0)
    pos_close(got, xT)


@pytest.mark.parametrize("D,dt", [(1e30, 1.0), (1e-32, 1.0)])
def test_walk2d_extreme_step_scales(torch_cuda, orc, D, dt):
    # Step scales s = sqrt(2 D dt) of about 1.4e15 and 1.4e-16.
    n, steps = 1000, 37
    got = to_numpy(orand.brownian_walk(n, steps, dt=dt, D=D, seed=0x77))
    x0, xT = orc.walk2d(0x77, n, steps, _f32(dt), _f32(D), threads=8)
    s = float(np.float32(np.sqrt(2.0 * _f32(D) * _f32(dt))))
    pos_close(got, xT, scale=max(1.0, s * np.sqrt(steps)))


def test_walk2d_full_workload_sampled(torch_cuda, orc):
    c = W.WALK2D
    got = orand.brownian_walk(c["n_particles"], c["steps"], c["dt"], c["D"], c["seed"])
    torch_cuda.cuda.synchronize()
    rng = np.random.default_rng(7)
    ids = np.unique(np.concatenate([[0, c["n_particles"] - 1], rng.integers(0, c["n_particles"], 62)]))
    g = to_numpy(got)
    for p in ids:
        _, xT = orc.walk2d(c["seed"], 1, c["steps"], float(np.float32(c["dt"])), c["D"], p_first=int(p))
        pos_close(g[p:p + 1], xT)
    # Einstein relation over all 2^24 particles: Var(x_T - x_0) = 2 D T dt.
    d = got.double() - 0.5
    var = (d.var(dim=0) - 1.0 / 12.0).cpu().numpy()
    expect = 2 * c["D"] * c["steps"] * float(np.float32(c["dt"]))
    assert np.all(np.abs(var / expect - 1) < 5 * math.sqrt(2 / c["n_particles"]) * 1.2)


# ------------------------------------------------------------------- 3D ----

MU = (0.1, -0.2, 0.05)


def _p(n, steps, K=16, p_first=0, p_total=0, seed=0, mu=MU, sigma=0.5):
    return orand.walk3d_params(n, steps, dt=1e-3, mu=mu, sigma=sigma, k=2.0, seed=seed, ckpt_every=K,
                               p_first=p_first, p_total=p_total)


def _f32(v):
    return float(np.float32(v))


def test_walk3d_forward_extreme_noise_scale(torch_cuda, orc):
    # sigma sqrt(dt) of about 3.2e14.
    n, steps, K, sigma = 300, 65, 16, 1e16
    p = _p(n, steps, K, sigma=sigma)
    xT, ck, loss = orand.walk3d_forward(p)
    torch_cuda.cuda.synchronize()
    oxT, ock = orc.walk3d_forward(0, n, steps, K, _f32(1e-3), MU, _f32(sigma), want_ckpt=True)
    scale = _f32(sigma) * np.sqrt(_f32(1e-3) * steps)
    pos_close(to_numpy(xT), oxT, scale=scale)
    pos_close(to_numpy(ck), ock, scale=scale)


@pytest.mark.parametrize("n,steps,K", [(1, 1, 1), (777, 200, 16), (300, 65, 64), (513, 0, 8), (400, 130, 24)])
def test_walk3d_forward_small(torch_cuda, orc, n, steps, K):
    p = _p(n, steps, K, p_first=3)
    x0 = orand.walk3d_init(p)
    xT, ck, loss = orand.walk3d_forward(p)
    xT2, ck2, loss2 = orand.walk3d_forward(p, x0=x0)
    torch_cuda.cuda.synchronize()
    ox0 = orc.walk3d_init(0, n, p_first=3)
    oxT, ock = orc.walk3d_forward(0, n, steps, K, _f32(1e-3), MU, 0.5, p_first=3, want_ckpt=True)
    assert np.array_equal(to_numpy(x0).astype(np.float64), ox0)
    pos_close(to_numpy(xT), oxT)
    assert torch_cuda.equal(xT, xT2) and loss.item() == loss2.item()
    if ock.shape[0]:
        pos_close(to_numpy(ck), ock)
        assert torch_cuda.equal(ck, ck2)
    else:
        assert ck is None
    oloss = orc.walk3d_loss(oxT, 2.0, n)
    assert loss.item() == pytest.approx(oloss, rel=GRAD_TOL, abs=1e-12)


@pytest.mark.parametrize("seed,p_first", [(0x1234, 2**40 + 3), (2**64 - 1, 2**63 - 700)])
def test_walk3d_far_keys(torch_cuda, orc, seed, p_first):
    """Forward and adjoint with a nonzero seed and particle ids far from 0
    (keys seed ^ (p_first + i) use all 64 bits)."""
    n, steps, K = 513, 80, 16
    p = _p(n, steps, K, p_first=p_first, p_total=n, seed=seed)
    xT, ck, _ = orand.walk3d_forward(p)
    g = torch_cuda.tensor(1.0, dtype=torch_cuda.float64, device="cuda")
    dmu, dsig, dx0 = orand.walk3d_backward(p, xT, g)
    torch_cuda.cuda.synchronize()
    oxT, ock = orc.walk3d_forward(seed, n, steps, K, _f32(1e-3), MU, 0.5, p_first=p_first, want_ckpt=True)
    pos_close(to_numpy(xT), oxT)
    pos_close(to_numpy(ck), ock)
    odmu, odsig, odx0 = orc.walk3d_adjoint(seed, n, steps, _f32(1e-3), oxT, 2.0, n, p_first=p_first)
    assert np.allclose(to_numpy(dmu), odmu, rtol=GRAD_TOL, atol=0)
    assert dsig.item() == pytest.approx(odsig, rel=GRAD_TOL)
    np.testing.assert_allclose(to_numpy(dx0), odx0, rtol=GRAD_TOL, atol=2.0 / n * POS_TOL)


@pytest.mark.parametrize("n,steps", [(1, 3), (777, 200), (1024, 64)])
def test_walk3d_adjoint_small(torch_cuda, orc, n, steps):
    p = _p(n, steps, p_first=11, p_total=5 * n)
    xT, _, _ = orand.walk3d_forward(p, want_ckpt=False)
    g = torch_cuda.tensor(0.75, dtype=torch_cuda.float64, device="cuda")
    dmu, dsig, dx0 = orand.walk3d_backward(p, xT, g)
    torch_cuda.cuda.synchronize()
    oxT, _ = orc.walk3d_forward(0, n, steps, 16, _f32(1e-3), MU, 0.5, p_first=11)
    odmu, odsig, odx0 = orc.walk3d_adjoint(0, n, steps, _f32(1e-3), oxT, 2.0, 5 * n, p_first=11)
    assert np.allclose(to_numpy(dmu), 0.75 * odmu, rtol=GRAD_TOL, atol=0)
    assert dsig.item() == pytest.approx(0.75 * odsig, rel=GRAD_TOL)
    # dx0 = g k x_T / P inherits the position error absolutely (near x_T = 0
    # the relative bar does not apply; the propagated one does).
    np.testing.assert_allclose(to_numpy(dx0), 0.75 * odx0, rtol=GRAD_TOL, atol=0.75 * 2.0 / (5 * n) * POS_TOL)


def test_walk3d_autograd_function(torch_cuda, orc):
    torch = torch_cuda
    n, steps = 2048, 128
    BW = orand.BrownianWalk3D()
    p = _p(n, steps, K=32)
    x0 = orand.walk3d_init(p).requires_grad_(True)
    mu = torch.tensor(MU, dtype=torch.float32, requires_grad=True)
    sigma = torch.tensor(0.5, dtype=torch.float32, requires_grad=True)
    loss = BW.apply(mu, sigma, x0, steps, 1e-3, 2.0, 0, 32)
    loss.backward()
    oxT, _ = orc.walk3d_forward(0, n, steps, 32, _f32(1e-3), MU, 0.5)
    odmu, odsig, odx0 = orc.walk3d_adjoint(0, n, steps, _f32(1e-3), oxT, 2.0, n)
    assert loss.item() == pytest.approx(orc.walk3d_loss(oxT, 2.0, n), rel=1e-6)
    assert np.allclose(mu.grad.numpy(), odmu, rtol=GRAD_TOL)
    assert sigma.grad.item() == pytest.approx(odsig, rel=GRAD_TOL)
    np.testing.assert_allclose(to_numpy(x0.grad), odx0, rtol=GRAD_TOL, atol=2.0 / n * POS_TOL)
    # Central differences through the GPU forward agree with the adjoint.
    h = 1e-3
    with torch.no_grad():
        lp = BW.apply(mu, sigma + h, x0, steps, 1e-3, 2.0, 0, 32).item()
        lm = BW.apply(mu, sigma - h, x0, steps, 1e-3, 2.0, 0, 32).item()
    sp, sm = _f32(_f32(0.5) + h), _f32(_f32(0.5) - h)
    assert (lp - lm) / (sp - sm) == pytest.approx(sigma.grad.item(), rel=GRAD_TOL)


def test_walk3d_autograd_frees_checkpoints_after_backward(torch_cuda):
    """The forward's checkpoints live on the call's autograd context only:
    held between forward and backward, freed once backward has run (what is
    left is x0's gradient).  mu and sigma stay on the CPU, so no device read
    is needed to set up the kernels."""
    torch = torch_cuda
    n, steps, K = 1 << 18, 256, 32                 # 8 checkpoints of 3 MiB each
    BW = orand.BrownianWalk3D()
    p = _p(n, steps, K=K)
    x0 = orand.walk3d_init(p).requires_grad_(True)
    mu = torch.tensor(MU, dtype=torch.float32, requires_grad=True)
    sigma = torch.tensor(0.5, dtype=torch.float32, requires_grad=True)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    loss = BW.apply(mu, sigma, x0, steps, 1e-3, 2.0, 0, K)
    held = torch.cuda.memory_allocated() - base
    assert held >= (steps // K) * n * 3 * 4         # checkpoints (and x_T) kept for backward
    loss.backward()
    del loss
    torch.cuda.synchronize()
    left = torch.cuda.memory_allocated() - base
    assert left <= n * 3 * 4 + (1 << 16), (held, left)   # x0.grad and small scalars only
    assert x0.grad is not None and mu.grad.device.type == "cpu"


def test_walk3d_plain_baseline_matches_fused(torch_cuda):
    torch = torch_cuda
    n, steps = 4096, 100
    p = _p(n, steps)
    ctx = orand.default_context().handle
    sh = torch.cuda.current_stream().cuda_stream
    xT, _, loss = orand.walk3d_forward(p, want_ckpt=False)
    dmu, dsig, dx0 = orand.walk3d_backward(p, xT)
    x = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    z = torch.empty((steps, n, 3), dtype=torch.float32, device="cuda")
    ploss = torch.empty((), dtype=torch.float64, device="cuda")
    orand.orand_walk3d_plain_fwd(ctx, p, 0, x.data_ptr(), z.data_ptr(), ploss.data_ptr(), sh)
    pdmu = torch.empty(3, dtype=torch.float64, device="cuda")
    pdsig = torch.empty((), dtype=torch.float64, device="cuda")
    pdx0 = torch.empty_like(x)
    orand.orand_walk3d_plain_bwd(ctx, p, x.data_ptr(), z.data_ptr(), 0, pdmu.data_ptr(), pdsig.data_ptr(),
                                 pdx0.data_ptr(), sh)
    torch.cuda.synchronize()
    assert torch.allclose(x, xT, rtol=POS_TOL, atol=POS_TOL)
    assert ploss.item() == pytest.approx(loss.item(), rel=GRAD_TOL)
    assert torch.allclose(pdmu, dmu, rtol=GRAD_TOL) and pdsig.item() == pytest.approx(dsig.item(), rel=GRAD_TOL)
    assert torch.allclose(pdx0, dx0, rtol=GRAD_TOL)
    # The stored noise is exactly what the fused kernels regenerate: z_0 drives x_1.
    p1 = _p(n, 1)
    x1, _, _ = orand.walk3d_forward(p1, want_ckpt=False)
    x0 = orand.walk3d_init(p1)
    inc = (x1 - x0).double()
    mu_dt = torch.tensor([_f32(m * _f32(1e-3)) for m in MU], dtype=torch.float64, device="cuda")
    zz = (inc - mu_dt) / _f32(0.5 * math.sqrt(_f32(1e-3)))
    assert torch.allclose(zz, z[0].double(), atol=1e-4)


def test_walk3d_full_workload(torch_cuda, orc):
    """2^22 x 4096 forward + adjoint: sampled particles against the oracle,
    a particle-range subset of the reductions against the oracle adjoint,
    and loss/dmu/dsigma by properties of the full run."""
    torch = torch_cuda
    c = W.WALK3D
    P, T = c["n_particles"], c["steps"]
    p = orand.walk3d_params(P, T, c["dt"], c["mu"], c["sigma"], c["k"], c["seed"], c["ckpt_every"])
    xT, ck, loss = orand.walk3d_forward(p)
    dmu, dsig, dx0 = orand.walk3d_backward(p, xT)
    torch.cuda.synchronize()
    assert ck.shape == (T // c["ckpt_every"], P, 3)
    rng = np.random.default_rng(9)
    ids = np.unique(np.concatenate([[0, P - 1], rng.integers(0, P, 30)]))
    dt32 = _f32(c["dt"])
    gx, gdx = to_numpy(xT), to_numpy(dx0)
    for q in ids:
        oxT, ock = orc.walk3d_forward(c["seed"], 1, T, c["ckpt_every"], dt32, c["mu"], c["sigma"], p_first=int(q),
                                      want_ckpt=True)
        pos_close(gx[q:q + 1], oxT)
        pos_close(to_numpy(ck[:, q]), ock[:, 0])
        np.testing.assert_allclose(gdx[q], c["k"] * oxT[0] / P, rtol=GRAD_TOL, atol=c["k"] / P * POS_TOL)
    # Properties of the full run (exact identities of the linear walk).
    x64 = xT.double()
    assert loss.item() == pytest.approx(0.5 * c["k"] * (x64 ** 2).sum().item() / P, rel=1e-9)
    assert np.allclose(to_numpy(dmu), c["k"] * T * dt32 * x64.mean(dim=0).cpu().numpy(), rtol=1e-6)
    assert np.allclose(to_numpy(dmu), [3.35, -6.7, 1.68], rtol=0.05)
    assert dsig.item() == pytest.approx(12.3, rel=0.05)
    # A particle-range subset of the reductions against the FP64 oracle adjoint.
    sub = orand.walk3d_params(1024, T, c["dt"], c["mu"], c["sigma"], c["k"], c["seed"], c["ckpt_every"],
                              p_first=123456, p_total=P)
    sxT, _, _ = orand.walk3d_forward(sub, want_ckpt=False)
    sdmu, sdsig, _ = orand.walk3d_backward(sub, sxT)
    oxT, _ = orc.walk3d_forward(c["seed"], 1024, T, 64, dt32, c["mu"], c["sigma"], p_first=123456, threads=8)
    odmu, odsig, _ = orc.walk3d_adjoint(c["seed"], 1024, T, dt32, oxT, c["k"], P, p_first=123456, threads=8)
    assert np.allclose(to_numpy(sdmu), odmu, rtol=GRAD_TOL)
    assert sdsig.item() == pytest.approx(odsig, rel=GRAD_TOL)
    # Central differences (h = 1e-3) on the GPU forward: exact for the quadratic loss.
    h = 1e-3
    lp = orand.walk3d_forward(orand.walk3d_params(P, T, c["dt"], c["mu"], c["sigma"] + h, c["k"], c["seed"], 0),
                              want_ckpt=False)[2].item()
    lm = orand.walk3d_forward(orand.walk3d_params(P, T, c["dt"], c["mu"], c["sigma"] - h, c["k"], c["seed"], 0),
                              want_ckpt=False)[2].item()
    sp, sm = _f32(_f32(c["sigma"]) + h), _f32(_f32(c["sigma"]) - h)
    assert (lp - lm) / (sp - sm) == pytest.approx(dsig.item(), rel=GRAD_TOL)
    del xT, ck, dx0
    torch.cuda.empty_cache()


# ------------------------------------------------- 3D, OU drift mu - kappa x ----

def _pou(n, steps, K, kappa, p_first=0, p_total=0, seed=0):
    return orand.walk3d_params(n, steps, dt=1e-3, mu=MU, sigma=0.5, k=2.0, seed=seed, ckpt_every=K,
                               p_first=p_first, p_total=p_total, kappa=kappa)


@pytest.mark.parametrize("n,steps,K,kappa", [(777, 200, 16, 1.5), (300, 203, 16, 1.5), (513, 97, 8, 20.0),
                                             (129, 64, 64, -3.0), (1, 1, 1, 0.5), (256, 150, 32, 0.0),
                                             (400, 130, 24, 1.5)])
def test_walk3d_ou_forward_and_adjoint(torch_cuda, orc, n, steps, K, kappa):
    """Fused OU forward and the checkpointed reverse-time adjoint against the
    FP64 oracle: positions, checkpoints, loss, dmu, dsigma, dkappa and dx0.
    Covers a short last segment (203 = 12 x 16 + 11), a strongly contracting
    drift (kappa dt = 0.02), an expanding one (kappa < 0), one segment, one
    step, and kappa = 0 with dL/dkappa requested."""
    torch = torch_cuda
    p = _pou(n, steps, K, kappa, p_first=5, p_total=3 * n)
    xT, ck, loss = orand.walk3d_forward(p)
    g = torch.tensor(-1.25, dtype=torch.float64, device="cuda")
    dmu, dsig, dkap, dx0 = orand.walk3d_backward_full(p, xT, ck, g)
    torch.cuda.synchronize()
    dt32 = _f32(1e-3)
    oxT, ock, xs = orc.walk3d_ou_forward(0, n, steps, K, dt32, MU, 0.5, _f32(kappa), p_first=5, want_ckpt=True)
    pos_close(to_numpy(xT), oxT)
    pos_close(to_numpy(ck), ock)
    assert loss.item() == pytest.approx(orc.walk3d_loss(oxT, 2.0, 3 * n), rel=GRAD_TOL)
    odmu, odsig, odk, odx0 = orc.walk3d_ou_adjoint(0, n, steps, dt32, _f32(kappa), xs, 2.0, 3 * n, p_first=5)
    assert np.allclose(to_numpy(dmu), -1.25 * odmu, rtol=GRAD_TOL, atol=0)
    assert dsig.item() == pytest.approx(-1.25 * odsig, rel=GRAD_TOL)
    assert dkap.item() == pytest.approx(-1.25 * odk, rel=GRAD_TOL)
    # dx0 = g k x_T (1 - kappa dt)^T / P inherits the position error absolutely:
    # where x_T is near 0 the relative bar does not apply, the propagated one does.
    np.testing.assert_allclose(to_numpy(dx0), -1.25 * odx0, rtol=GRAD_TOL, atol=1.25 * 2.0 / (3 * n) * POS_TOL)
    # Without dkappa the same entry point gives the same dmu, dsigma, dx0.
    if kappa != 0.0:
        dmu2, dsig2, dx02 = orand.walk3d_backward(p, xT, g, ckpt=ck)
        assert torch.equal(dmu2, dmu) and dsig2.item() == dsig.item() and torch.equal(dx02, dx0)


def test_walk3d_ou_argument_checks(torch_cuda):
    """The kappa != 0 adjoint needs checkpoints; 1 - kappa dt must stay positive."""
    torch = torch_cuda
    p = _pou(64, 40, 8, 2.0)
    xT, ck, _ = orand.walk3d_forward(p)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        orand.walk3d_backward(p, xT)  # no checkpoints
    p0 = _pou(64, 40, 0, 2.0)
    xT0, ck0, _ = orand.walk3d_forward(p0)  # the forward alone needs no checkpoint interval
    assert ck0 is None
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        orand.walk3d_backward(p0, xT0)  # the adjoint does
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        orand.walk3d_forward(_pou(64, 40, 8, 1000.0))  # kappa dt = 1
    torch.cuda.synchronize()


def test_walk3d_ou_autograd_and_central_differences(torch_cuda, orc):
    """kappa through BrownianWalk3D: its gradient matches the oracle adjoint
    and central differences of the GPU forward in kappa."""
    torch = torch_cuda
    n, steps, K = 4096, 256, 32
    BW = orand.BrownianWalk3D()
    p = _pou(n, steps, K, 2.5)
    x0 = orand.walk3d_init(p).requires_grad_(True)
    mu = torch.tensor(MU, dtype=torch.float32, requires_grad=True)
    sigma = torch.tensor(0.5, dtype=torch.float32, requires_grad=True)
    kappa = torch.tensor(2.5, dtype=torch.float32, requires_grad=True)
    loss = BW.apply(mu, sigma, x0, steps, 1e-3, 2.0, 0, K, kappa)
    loss.backward()
    dt32 = _f32(1e-3)
    oxT, _, xs = orc.walk3d_ou_forward(0, n, steps, K, dt32, MU, 0.5, 2.5)
    odmu, odsig, odk, odx0 = orc.walk3d_ou_adjoint(0, n, steps, dt32, 2.5, xs, 2.0, n)
    assert loss.item() == pytest.approx(orc.walk3d_loss(oxT, 2.0, n), rel=1e-6)
    assert np.allclose(mu.grad.numpy(), odmu, rtol=GRAD_TOL)
    assert sigma.grad.item() == pytest.approx(odsig, rel=GRAD_TOL)
    assert kappa.grad.item() == pytest.approx(odk, rel=GRAD_TOL)
    np.testing.assert_allclose(to_numpy(x0.grad), odx0, rtol=GRAD_TOL, atol=2.0 / n * POS_TOL)
    h = 1e-2
    with torch.no_grad():
        lp = BW.apply(mu, sigma, x0, steps, 1e-3, 2.0, 0, K, kappa + h).item()
        lm = BW.apply(mu, sigma, x0, steps, 1e-3, 2.0, 0, K, kappa - h).item()
    kp, km = _f32(_f32(2.5) + h), _f32(_f32(2.5) - h)
    assert (lp - lm) / (kp - km) == pytest.approx(kappa.grad.item(), rel=GRAD_TOL)


# ------------------------------------------- fused noise-storing variant ----

def _stored_run(torch, p, n, steps):
    ctx = orand.default_context().handle
    sh = torch.cuda.current_stream().cuda_stream
    xT = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    z = torch.empty((steps, n, 3), dtype=torch.float32, device="cuda")
    loss = torch.empty((), dtype=torch.float64, device="cuda")
    orand.orand_walk3d_stored_fwd(ctx, p, 0, xT.data_ptr(), z.data_ptr(), loss.data_ptr(), sh)
    dmu = torch.empty(3, dtype=torch.float64, device="cuda")
    dsig = torch.empty((), dtype=torch.float64, device="cuda")
    dx0 = torch.empty_like(xT)
    g = torch.tensor(0.5, dtype=torch.float64, device="cuda")
    orand.orand_walk3d_stored_bwd(ctx, p, xT.data_ptr(), z.data_ptr(), g.data_ptr(), dmu.data_ptr(),
                                  dsig.data_ptr(), dx0.data_ptr(), sh)
    torch.cuda.synchronize()
    return xT, z, loss, dmu, dsig, dx0


@pytest.mark.parametrize("n,steps", [(4096 + 33, 100), (1, 17), (300, 0)])
def test_walk3d_stored_matches_regenerating_and_plain(torch_cuda, orc, n, steps):
    """Stored noise equals the plain baseline's bit for bit; positions,
    loss and gradients equal the regenerating walk's and the oracle's."""
    torch = torch_cuda
    p = _p(n, steps, K=16, p_first=9, p_total=2 * n)
    xT, z, loss, dmu, dsig, dx0 = _stored_run(torch, p, n, steps)
    rxT, _, rloss = orand.walk3d_forward(p, want_ckpt=False)
    g = torch.tensor(0.5, dtype=torch.float64, device="cuda")
    rdmu, rdsig, rdx0 = orand.walk3d_backward(p, rxT, g)
    torch.cuda.synchronize()
    oxT, _ = orc.walk3d_forward(0, n, steps, 16, _f32(1e-3), MU, 0.5, p_first=9)
    pos_close(to_numpy(xT), oxT)
    assert loss.item() == pytest.approx(rloss.item(), rel=GRAD_TOL)
    assert np.allclose(to_numpy(dmu), to_numpy(rdmu), rtol=GRAD_TOL)
    assert dsig.item() == pytest.approx(rdsig.item(), rel=GRAD_TOL, abs=1e-12)
    np.testing.assert_allclose(to_numpy(dx0), to_numpy(rdx0), rtol=GRAD_TOL, atol=1e-12)
    if steps:
        ctx = orand.default_context().handle
        x = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        zp = torch.empty((steps, n, 3), dtype=torch.float32, device="cuda")
        orand.orand_walk3d_plain_fwd(ctx, p, 0, x.data_ptr(), zp.data_ptr(), 0, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert torch.equal(z, zp)


def test_walk3d_stored_full_steps_subset(torch_cuda, orc):
    """4096 steps on a 2^18-particle range of the 2^22-particle workload
    (12.9 GB of stored noise): gradients against the regenerating adjoint,
    and a particle-range subset against the FP64 oracle adjoint."""
    torch = torch_cuda
    c = W.WALK3D
    n, T = 1 << 18, c["steps"]
    p = orand.walk3d_params(n, T, c["dt"], c["mu"], c["sigma"], c["k"], c["seed"], 0, p_first=777, p_total=c["n_particles"])
    xT, z, loss, dmu, dsig, dx0 = _stored_run(torch, p, n, T)
    del z
    rxT, _, _ = orand.walk3d_forward(p, want_ckpt=False)
    g = torch.tensor(0.5, dtype=torch.float64, device="cuda")
    rdmu, rdsig, _ = orand.walk3d_backward(p, rxT, g)
    torch.cuda.synchronize()
    assert torch.allclose(xT, rxT, rtol=POS_TOL, atol=POS_TOL)
    assert np.allclose(to_numpy(dmu), to_numpy(rdmu), rtol=GRAD_TOL)
    assert dsig.item() == pytest.approx(rdsig.item(), rel=GRAD_TOL)
    sub = orand.walk3d_params(512, T, c["dt"], c["mu"], c["sigma"], c["k"], c["seed"], 0, p_first=777,
                              p_total=c["n_particles"])
    sxT, _, _, sdmu, sdsig, _ = _stored_run(torch, sub, 512, T)
    dt32 = _f32(c["dt"])
    oxT, _ = orc.walk3d_forward(c["seed"], 512, T, 64, dt32, c["mu"], c["sigma"], p_first=777, threads=8)
    odmu, odsig, _ = orc.walk3d_adjoint(c["seed"], 512, T, dt32, oxT, c["k"], c["n_particles"], p_first=777, threads=8)
    assert np.allclose(to_numpy(sdmu), 0.5 * odmu, rtol=GRAD_TOL)
    assert sdsig.item() == pytest.approx(0.5 * odsig, rel=GRAD_TOL)


# --------------------------------------------------- cuRAND comparison ----

def test_walk2d_curand_forms_agree_and_diffuse(torch_cuda):
    """cuRAND's Philox walk, per-step (Fig. 2) and fused: the same cuRAND
    draws, so the same positions up to summation order; at 0 steps the
    start positions match exactly; the fused walk obeys Einstein's relation."""
    torch = torch_cuda
    sh = torch.cuda.current_stream().cuda_stream
    n, steps = 5000 + 17, 300
    p = orand.walk2d_params(n, steps, dt=1e-3, D=1.0, p_first=123)
    states = torch.empty(n * orand.orand_walk2d_curand_state_bytes(), dtype=torch.uint8, device="cuda")
    pos_a = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    pos_b = torch.empty_like(pos_a)
    orand.orand_walk2d_curand_setup(p, states.data_ptr(), pos_a.data_ptr(), 1984, sh)
    p0 = orand.walk2d_params(n, 0, dt=1e-3, D=1.0, p_first=123)
    orand.orand_walk2d_curand_fused(p0, pos_b.data_ptr(), 1984, sh)
    torch.cuda.synchronize()
    assert torch.equal(pos_a, pos_b)
    orand.orand_walk2d_curand_run(p, states.data_ptr(), pos_a.data_ptr(), sh)
    orand.orand_walk2d_curand_fused(p, pos_b.data_ptr(), 1984, sh)
    torch.cuda.synchronize()
    assert torch.allclose(pos_a, pos_b, rtol=POS_TOL, atol=POS_TOL)
    m, T = 1 << 20, 1000
    big = orand.walk2d_params(m, T, dt=1e-3, D=1.0)
    start = torch.empty((m, 2), dtype=torch.float32, device="cuda")
    end = torch.empty_like(start)
    orand.orand_walk2d_curand_fused(orand.walk2d_params(m, 0), start.data_ptr(), 7, sh)
    orand.orand_walk2d_curand_fused(big, end.data_ptr(), 7, sh)
    torch.cuda.synchronize()
    var = (end.double() - start.double()).var(dim=0).cpu().numpy()
    expect = 2 * 1.0 * T * _f32(1e-3)
    assert np.all(np.abs(var / expect - 1) < 5 * math.sqrt(2 / m))


def test_walk3d_ou_full_workload(torch_cuda, orc):
    """The OU walk in the bench's configuration (2^22 x 4096, kappa = 1):
    sampled particles (positions, checkpoints, dx0) against the FP64 oracle,
    the loss identity over all particles, and a particle-range subset of the
    reductions (dmu, dsigma, dkappa) against the oracle adjoint."""
    torch = torch_cuda
    c = W.WALK3D_OU
    P, T, K = c["n_particles"], c["steps"], c["ckpt_every"]
    p = orand.walk3d_params(P, T, c["dt"], c["mu"], c["sigma"], c["k"], c["seed"], K, kappa=c["kappa"])
    xT, ck, loss = orand.walk3d_forward(p)
    dmu, dsig, dkap, dx0 = orand.walk3d_backward_full(p, xT, ck)
    torch.cuda.synchronize()
    dt32 = _f32(c["dt"])
    rng = np.random.default_rng(21)
    ids = np.unique(np.concatenate([[0, P - 1], rng.integers(0, P, 14)]))
    gx, gdx = to_numpy(xT), to_numpy(dx0)
    for q in ids:
        oxT, ock, xs = orc.walk3d_ou_forward(c["seed"], 1, T, K, dt32, c["mu"], c["sigma"], c["kappa"],
                                             p_first=int(q), want_ckpt=True)
        pos_close(gx[q:q + 1], oxT)
        pos_close(to_numpy(ck[:, q]), ock[:, 0])
        _, _, _, odx0 = orc.walk3d_ou_adjoint(c["seed"], 1, T, dt32, c["kappa"], xs, c["k"], P, p_first=int(q))
        np.testing.assert_allclose(gdx[q], odx0[0], rtol=GRAD_TOL, atol=c["k"] / P * POS_TOL)
    x64 = xT.double()
    assert loss.item() == pytest.approx(0.5 * c["k"] * (x64 ** 2).sum().item() / P, rel=1e-9)
    assert np.all(np.isfinite(to_numpy(dmu))) and np.isfinite(dsig.item()) and np.isfinite(dkap.item())
    sub = orand.walk3d_params(1024, T, c["dt"], c["mu"], c["sigma"], c["k"], c["seed"], K, p_first=654321,
                              p_total=P, kappa=c["kappa"])
    sxT, sck, _ = orand.walk3d_forward(sub)
    sdmu, sdsig, sdk, _ = orand.walk3d_backward_full(sub, sxT, sck)
    torch.cuda.synchronize()
    _, _, xs = orc.walk3d_ou_forward(c["seed"], 1024, T, K, dt32, c["mu"], c["sigma"], c["kappa"], p_first=654321)
    odmu, odsig, odk, _ = orc.walk3d_ou_adjoint(c["seed"], 1024, T, dt32, c["kappa"], xs, c["k"], P, p_first=654321)
    assert np.allclose(to_numpy(sdmu), odmu, rtol=GRAD_TOL)
    assert sdsig.item() == pytest.approx(odsig, rel=GRAD_TOL)
    assert sdk.item() == pytest.approx(odk, rel=GRAD_TOL)
