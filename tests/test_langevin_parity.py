"""The paper's Brownian-dynamics macro-benchmark (Fig. 1, §5) on the GPU.

The per-step kernel (one launch per step, the Fig. 1 host loop) and the
fused kernel (all steps in registers) are held bit-exact to the FP64 oracle.
All three use explicit round-to-nearest FP64 operations in the paper's order.
The cuRAND-state pattern (Fig. 2, the paper's comparison system) draws other
numbers, so it is checked by the stationary velocity variance
(dt/3)/(1 - c^2) with c = 1 - gamma dt / m.
"""
import math

import numpy as np
import pytest

import paper_2310_19925_b300 as orand

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _state(torch, ps):
    torch.cuda.synchronize()
    return orand.particle_state(ps).cpu().numpy()


def test_per_step_and_fused_match_oracle_bit_exact(torch_cuda, orc):
    torch = torch_cuda
    n, steps, p_first = 5000, 60, 123456
    prm = orand.langevin2d_params(n, dt=1e-3, gamma=1.0, mass=1.0, seed=7, p_first=p_first)
    sh = torch.cuda.current_stream().cuda_stream
    a = orand.particles_tensor(n)
    b = orand.particles_tensor(n)
    orand.orand_langevin2d_init(prm, a.data_ptr(), sh)
    orand.orand_langevin2d_init(prm, b.data_ptr(), sh)
    init = _state(torch, a).copy()
    for it in range(1, steps + 1):
        orand.orand_langevin2d_step(prm, a.data_ptr(), it, sh)
    orand.orand_langevin2d_fused(prm, b.data_ptr(), 1, steps // 2, sh)
    orand.orand_langevin2d_fused(prm, b.data_ptr(), 1 + steps // 2, steps - steps // 2, sh)
    sa, sb = _state(torch, a), _state(torch, b)
    ref = orc.langevin2d(7, n, steps, dt=1e-3, gamma=1.0, mass=1.0, p_first=p_first, threads=8)
    ref0 = orc.langevin2d(7, n, 0, p_first=p_first)
    assert np.array_equal(init, ref0)
    assert np.array_equal(sa, ref) and np.array_equal(sb, ref)
    pids = a[:, 4].contiguous().view(torch.int64).cpu().numpy()
    assert np.array_equal(pids, np.arange(p_first, p_first + n))


def test_paper_size_fused_sampled(torch_cuda, orc):
    """10^6 particles x 10^4 steps (the paper's §5 size) in one fused launch."""
    torch = torch_cuda
    n, steps = 1_000_000, 10_000
    prm = orand.langevin2d_params(n)
    sh = torch.cuda.current_stream().cuda_stream
    ps = orand.particles_tensor(n)
    orand.orand_langevin2d_init(prm, ps.data_ptr(), sh)
    orand.orand_langevin2d_fused(prm, ps.data_ptr(), 1, steps, sh)
    st = _state(torch, ps)
    rng = np.random.default_rng(3)
    for i in np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 24)])):
        ref = orc.langevin2d(0, 1, steps, p_first=int(i))
        assert np.array_equal(st[i:i + 1], ref), i
    v = st[:, 2:].ravel()
    c = 1 - 1e-3
    var = (1e-3 / 3) / (1 - c * c)
    assert abs(v.var() / var - 1) < 5 * math.sqrt(2 / v.size)


def test_curand_pattern_statistics(torch_cuda):
    torch = torch_cuda
    n, steps = 1 << 16, 4000
    prm = orand.langevin2d_params(n)
    sh = torch.cuda.current_stream().cuda_stream
    ps = orand.particles_tensor(n)
    states = torch.empty(n * orand.orand_langevin2d_curand_state_bytes(), dtype=torch.uint8, device="cuda")
    orand.orand_langevin2d_curand_setup(prm, ps.data_ptr(), states.data_ptr(), 1984, sh)
    x0 = _state(torch, ps)[:, :2].copy()
    assert np.all((x0 > 0) & (x0 <= 1))
    for _ in range(steps):
        orand.orand_langevin2d_curand_step(prm, ps.data_ptr(), states.data_ptr(), sh)
    v = _state(torch, ps)[:, 2:].ravel()
    c = 1 - 1e-3
    var = (1e-3 / 3) / (1 - c * c)
    assert abs(v.var() / var - 1) < 5 * math.sqrt(2 / v.size)
    assert abs(v.mean()) < 5 * math.sqrt(var / v.size)
