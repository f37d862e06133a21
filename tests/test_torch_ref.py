"""The differentiable torch restatement (oracle/torch_ref.py) against the C
oracle: residual, one forced step, and its autograd gradient of the surface
functional against central differences of the C oracle's own window."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import torch_ref  # noqa: E402
from paper_2301_00817_gb300 import synth  # noqa: E402


def _case(orc, shape, noise=3e-2, pnoise=1e-2, seed=5, **kw):
    xyz = synth.jet_grid(*shape)
    M = orc.metrics(xyz, (0, 0, 1))
    P = orc.params(**kw)
    Q = orc.init_jet(P, xyz, seed=seed, noise=noise)
    rng = np.random.default_rng(seed)
    Q[4] += pnoise / (P.gamma - 1.0) * rng.standard_normal(Q[4].shape)
    return xyz, M, P, Q


def _rel(a, b):
    scale = np.abs(b).reshape(5, -1).max(axis=1)[:, None, None, None]
    return float(np.max(np.abs(a - b) / np.maximum(scale, 1e-300)))


def test_residual_matches_oracle(orc):
    xyz, M, P, Q = _case(orc, (12, 10, 8), Re=300.0)
    MK = orc.mu_eff(P, Q, M)
    R_orc = orc.rhs(P, Q, M, MK)
    case = torch_ref.Case(M, xyz, Re=300.0)
    R_t = case.rhs(torch.from_numpy(Q), tuple(torch.from_numpy(MK)))
    assert _rel(R_t.numpy(), R_orc) <= 1e-12
    # the viscosity restatement too
    mu, kap = case.viscosity(torch.from_numpy(Q))
    assert np.allclose(mu.numpy(), MK[0], rtol=1e-14, atol=0)
    assert np.allclose(kap.numpy(), MK[1], rtol=1e-14, atol=0)


def test_forced_step_matches_oracle(orc):
    amps = synth.forcing_amplitudes(3, scale=2e-2)
    xyz, M, P, Q = _case(orc, (12, 10, 8), Re=500.0, dt_mode=1, dt_fixed=1e-3,
                         amp=tuple(amps))
    t = 0.0137
    Q1, dt = orc.rk_step(P, Q, M, xyz, t)
    case = torch_ref.Case(M, xyz, Re=500.0)
    Q1t = case.step(torch.from_numpy(Q), torch.from_numpy(amps), t, dt)
    assert _rel(Q1t.numpy(), Q1) <= 1e-12


def test_axis_grid_residual_and_step_match_oracle(orc):
    """True centerline grid (reading A27): the torch restatement's residual
    and forced step against the C oracle's axis mode, viscous, with the
    dissipation on."""
    shape = (12, 10, 8)
    amps = synth.forcing_amplitudes(3, scale=2e-2)
    xyz = synth.jet_grid(*shape, r0=0.0)
    M = orc.metrics(xyz, (0, 0, 1))
    P = orc.params(Re=300.0, dt_mode=1, dt_fixed=1e-3, amp=tuple(amps), axis=1)
    Q = orc.init_jet(P, xyz, seed=6, noise=3e-2)
    rng = np.random.default_rng(6)
    Q[4] += 1e-2 / (P.gamma - 1.0) * rng.standard_normal(Q[4].shape)
    MK = orc.mu_eff(P, Q, M)
    R_orc = orc.rhs(P, Q, M, MK)
    assert np.isfinite(R_orc).all() and np.abs(R_orc[:, :, 1]).max() > 0.0
    case = torch_ref.Case(M, xyz, Re=300.0, axis=True)
    R_t = case.rhs(torch.from_numpy(Q), tuple(torch.from_numpy(MK)))
    assert _rel(R_t.numpy(), R_orc) <= 1e-12
    t = 0.021
    Q1, dt = orc.rk_step(P, Q, M, xyz, t)
    Q1t = case.step(torch.from_numpy(Q), torch.from_numpy(amps), t, dt)
    assert np.isfinite(Q1).all()
    assert _rel(Q1t.numpy(), Q1) <= 1e-12


def _functional_orc(orc, P, Q0, M, xyz, nsteps, j5):
    """The surface functional over a window of oracle steps (the C oracle's
    own window: dt times the functional term after every step)."""
    return orc.window_functional(P, Q0, M, xyz, nsteps, 0.0, j5)


def test_autograd_gradient_matches_oracle_differences(orc):
    shape = (16, 8, 8)
    amps = synth.forcing_amplitudes(9, scale=2e-2)
    xyz, M, P, Q = _case(orc, shape, noise=1e-3, pnoise=0.0, seed=1, Re=500.0, dt_mode=1,
                         dt_fixed=1e-3, amp=tuple(amps))
    j5 = int(np.argmin(np.abs(synth.jet_radial(shape[1]) - 0.5)))
    nsteps, dt = 2, 1e-3
    case = torch_ref.Case(M, xyz, Re=500.0)
    a = torch.tensor(amps, dtype=torch.float64, requires_grad=True)
    J, _ = case.window(torch.from_numpy(Q), a, 0.0, dt, nsteps, j5)
    J.backward()
    g = a.grad.numpy()
    assert np.isclose(float(J.detach()), _functional_orc(orc, P, Q, M, xyz, nsteps, j5),
                      rtol=1e-12, atol=0)
    h = 1e-6
    for m in (0, 5, 10, 15):
        ap, am = amps.copy(), amps.copy()
        ap[m] += h
        am[m] -= h
        Pp = orc.params(Re=500.0, dt_mode=1, dt_fixed=dt, amp=tuple(ap))
        Pm = orc.params(Re=500.0, dt_mode=1, dt_fixed=dt, amp=tuple(am))
        fd = (_functional_orc(orc, Pp, Q, M, xyz, nsteps, j5) -
              _functional_orc(orc, Pm, Q, M, xyz, nsteps, j5)) / (2 * h)
        assert abs(fd - g[m]) <= 1e-6 * np.abs(g).max(), (m, fd, g[m])


@pytest.mark.parametrize("shape", [(16, 8, 8), (6, 5, 4)])
def test_brute_force_tiny_grids(orc, shape):
    """Two independent FP64 implementations (C loops, torch array shifts) on
    tiny jet grids: residual and three forced steps with the CFL time step,
    <= 1e-14 of each component's scale."""
    xyz = synth.jet_grid(*shape)
    M = orc.metrics(xyz, (0, 0, 1))
    amps = synth.forcing_amplitudes(4, scale=2e-2)
    P = orc.params(Re=300.0, amp=tuple(amps))
    Q = orc.init_jet(P, xyz, seed=3, noise=3e-2)
    Q[4] += 1e-2 / (P.gamma - 1.0) * np.random.default_rng(3).standard_normal(Q[4].shape)
    MK = orc.mu_eff(P, Q, M)
    case = torch_ref.Case(M, xyz, Re=300.0)
    R = orc.rhs(P, Q, M, MK)
    Rt = case.rhs(torch.from_numpy(Q), tuple(torch.from_numpy(MK))).numpy()
    assert _rel(Rt, R) <= 1e-14
    Qo, Qt, t = Q.copy(), torch.from_numpy(Q.copy()), 0.0
    for _ in range(3):
        Qo, dt = orc.rk_step(P, Qo, M, xyz, t)
        Qt = case.step(Qt, torch.from_numpy(amps), t, dt)
        t += dt
        assert _rel(Qt.numpy(), Qo) <= 1e-14
