"""Discrete adjoint of the FP64 step (vector-Jacobian products) on the GPU.

* Residual: the hand-written adjoint against the exact tangent obtained by
  running the FP64 residual kernels on dual numbers: <lamR, J dQ> must equal
  <J^T lamR, dQ> to round-off (dot-product test).
* One time step (stages + boundary conditions + frozen viscosity): adjoint
  against central finite differences of the GPU step, in a random state
  direction and in every forcing-amplitude direction.
* Window: the checkpointed adjoint gradient of the surface functional against
  central finite differences (step 1e-6) of the whole window, the same result
  for several checkpoint spacings, and the torch.autograd wrapper against the
  direct call.
* The same window against torch.autograd through the independent FP64 torch
  restatement of the step (oracle/torch_ref.py), on a 16 x 8 x 8 grid.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lj():
    from paper_2301_00817_gb300 import _build
    _build.build()
    import paper_2301_00817_gb300 as lj
    lj.load_library()
    return lj


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _jet(lj, torch, shape, **kw):
    ctx = lj.Context(lj.make_params(**kw), shape, "cuda:0")
    xyz = torch.from_numpy(lj.synth.jet_grid(*shape)).cuda()
    ctx.les_set_grid(xyz)
    return ctx, xyz


def _vdot(a, b):
    return float((a * b).sum())


@pytest.mark.parametrize("case", ["jet", "box", "box_conservative"])
def test_residual_adjoint_dot_product(lj, torch, case):
    if case == "jet":
        shape = (13, 11, 8)
        ctx, xyz = _jet(lj, torch, shape, Re=300.0)
        Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
        ctx.les_init_jet(xyz, 3, 3e-2, Q)
    else:
        shape = (9, 11, 10)
        xyz_np, shift = lj.synth.box_grid(shape, (1.0, 1.3, 0.8), wave=0.25)
        form = lj.METRIC_CONSERVATIVE if case == "box_conservative" else lj.METRIC_CROSS
        ctx = lj.Context(lj.make_params(periodic=(1, 1, 1), bc=0, Re=300.0, metric_form=form),
                         shape, "cuda:0")
        ctx.les_set_grid(torch.from_numpy(xyz_np).cuda(), shift)
        import oracle
        P = oracle.params(periodic=(1, 1, 1), bc=0)
        prim = lj.synth.smooth_periodic_prim(xyz_np, (1.0, 1.3, 0.8), amp=0.2, seed=4)
        Q = torch.from_numpy(oracle.prim_to_cons(P, prim)).cuda()
    gen = torch.Generator(device="cuda").manual_seed(11)
    dQ = 1e-2 * torch.randn(Q.shape, dtype=torch.float64, device="cuda", generator=gen)
    dMK = 1e-4 * torch.randn((2,) + shape, dtype=torch.float64, device="cuda", generator=gen)
    lamR = torch.randn(Q.shape, dtype=torch.float64, device="cuda", generator=gen)
    aw = ctx.adjoint_workspace()
    R = torch.empty_like(Q)
    dR = torch.empty_like(Q)
    ctx.les_rhs_jvp(Q, dQ, dMK, R, dR, aw)
    R_ref = torch.empty_like(Q)
    ctx.les_rhs(Q, R_ref)
    assert torch.equal(R, R_ref)  # the dual-number run reproduces the residual
    lamQ = torch.empty_like(Q)
    lamMK = torch.empty_like(dMK)
    ctx.les_rhs_vjp(Q, lamR, lamQ, lamMK, aw)
    lhs = _vdot(lamR, dR)
    rhs = _vdot(lamQ, dQ) + _vdot(lamMK, dMK)
    scale = _vdot(lamR.abs(), dR.abs())
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)
    # the viscosity direction alone, too
    ctx.les_rhs_jvp(Q, torch.zeros_like(Q), dMK, None, dR, aw)
    assert abs(_vdot(lamR, dR) - _vdot(lamMK, dMK)) <= 1e-12 * _vdot(lamR.abs(), dR.abs())


def _step_ctx(lj, torch, shape, amps):
    ctx, xyz = _jet(lj, torch, shape, Re=500.0, dt_mode=lj.DT_FIXED, dt_fixed=1.0e-3,
                    amp=tuple(amps))
    return ctx, xyz


def test_step_adjoint_against_finite_differences(lj, torch):
    shape = (14, 12, 8)
    amps = lj.synth.forcing_amplitudes(5, scale=2e-2)
    ctx, xyz = _step_ctx(lj, torch, shape, amps)
    Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
    ctx.les_init_jet(xyz, 7, 1e-2, Q)
    t_n = 0.0137
    gen = torch.Generator(device="cuda").manual_seed(2)
    # The initial pressure is uniform, so every pressure sensor |d2p| sits on
    # its kink and a central difference straddles it.  Pressure fluctuations of
    # 1e-2 (energy only) move the state to a generic point, far from the kinks
    # at the finite-difference step used below.
    Q[4] += 1e-2 / (lj.make_params().gamma - 1.0) * torch.randn(
        shape, dtype=torch.float64, device="cuda", generator=gen)
    lam = torch.randn(Q.shape, dtype=torch.float64, device="cuda", generator=gen)
    u = torch.randn(Q.shape, dtype=torch.float64, device="cuda", generator=gen) * Q.abs().amax(
        dim=(1, 2, 3), keepdim=True)
    aw = ctx.adjoint_workspace()
    lam_out = torch.empty_like(Q)
    grad = ctx.les_adjoint_step(Q, t_n, lam, lam_out, aw)

    def step(Qs, p=None):
        if p is not None:
            ctx.les_set_params(p)
        Qw = Qs.clone()
        ctx.les_set_time(t_n)
        ctx.les_rk_step(Qw)
        return Qw

    eps = 1e-6
    dq = (step(Q + eps * u) - step(Q - eps * u)) / (2 * eps)
    lhs, rhs = _vdot(lam, dq), _vdot(lam_out, u)
    assert abs(lhs - rhs) <= 1e-6 * abs(rhs), (lhs, rhs)
    base = lj.LesParams.from_buffer_copy(ctx.params)
    for m in range(16):
        pp = lj.LesParams.from_buffer_copy(base)
        pm = lj.LesParams.from_buffer_copy(base)
        pp.amp[m] += eps
        pm.amp[m] -= eps
        fd = _vdot(lam, (step(Q, pp) - step(Q, pm)) / (2 * eps))
        assert abs(fd - grad[m]) <= 1e-6 * max(abs(g) for g in grad), (m, fd, grad[m])
    ctx.les_set_params(base)


def _j_surface(lj, shape, radius):
    r = lj.synth.jet_radial(shape[1])
    return int(np.argmin(np.abs(r - radius)))


def test_window_gradient_against_finite_differences(lj, torch):
    """Well-conditioned companion of the far-field functional (pressure
    fluctuation on the shear-layer surface r = 0.5 D), 6 steps with a
    checkpoint every 2 steps."""
    shape = (16, 14, 16)
    amps = lj.synth.forcing_amplitudes(9, scale=2e-2)
    ctx, xyz = _step_ctx(lj, torch, shape, amps)
    Q0 = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
    ctx.les_init_jet(xyz, 1, 1e-3, Q0)
    j5 = _j_surface(lj, shape, 0.5)
    nsteps, K = 6, 2
    aw = ctx.adjoint_workspace(nsteps, K)
    J, grad = ctx.les_adjoint_window(Q0, 0.0, nsteps, K, j5, aw)
    assert J > 0 and max(abs(g) for g in grad) > 0
    base = lj.LesParams.from_buffer_copy(ctx.params)
    h = 1e-6
    fd = []
    for m in range(16):
        pp = lj.LesParams.from_buffer_copy(base)
        pm = lj.LesParams.from_buffer_copy(base)
        pp.amp[m] += h
        pm.amp[m] -= h
        ctx.les_set_params(pp)
        Jp, _ = ctx.les_adjoint_window(Q0, 0.0, nsteps, K, j5, aw)
        ctx.les_set_params(pm)
        Jm, _ = ctx.les_adjoint_window(Q0, 0.0, nsteps, K, j5, aw)
        fd.append((Jp - Jm) / (2 * h))
    ctx.les_set_params(base)
    gmax = max(abs(g) for g in grad)
    for m in range(16):
        assert abs(fd[m] - grad[m]) <= 1e-6 * gmax, (m, fd[m], grad[m])
    # other checkpoint spacings (every step, a ragged last segment, the whole
    # window kept by the forward sweep) give the same functional and gradient
    for K2 in (1, 4, nsteps):
        aw2 = ctx.adjoint_workspace(nsteps, K2)
        J2, g2 = ctx.les_adjoint_window(Q0, 0.0, nsteps, K2, j5, aw2)
        assert math.isclose(J2, J, rel_tol=1e-12), (K2, J2, J)
        assert np.allclose(g2, grad, rtol=0, atol=1e-10 * gmax), K2
    # same J and gradient through torch.autograd
    a = torch.tensor(list(base.amp), dtype=torch.float64, requires_grad=True)
    Jt = lj.window_functional(ctx, a, Q0, 0.0, nsteps, K, j5, aw)
    Jt.backward()
    assert math.isclose(float(Jt.detach()), J, rel_tol=1e-12)
    assert np.allclose(a.grad.numpy(), np.array(grad), rtol=1e-12, atol=0)


def test_adjoint_is_bitwise_reproducible(lj, torch):
    """Every interface writes its cotangent record and each node sums the
    records that concern it in a fixed order (no atomics): two window
    gradients and two residual VJPs of the same inputs agree bit for bit,
    on a grid with many blocks per direction (48 x 40 x 32)."""
    shape = (48, 40, 32)
    amps = lj.synth.forcing_amplitudes(3, scale=2e-2)
    ctx, xyz = _step_ctx(lj, torch, shape, amps)
    Q0 = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
    ctx.les_init_jet(xyz, 2, 1e-2, Q0)
    j5 = _j_surface(lj, shape, 0.5)
    aw = ctx.adjoint_workspace(4, 2)
    J1, g1 = ctx.les_adjoint_window(Q0, 0.0, 4, 2, j5, aw)
    J2, g2 = ctx.les_adjoint_window(Q0, 0.0, 4, 2, j5, aw)
    assert J1 == J2 and list(g1) == list(g2)
    assert max(abs(g) for g in g1) > 0
    lamR = torch.randn(Q0.shape, dtype=torch.float64, device="cuda",
                       generator=torch.Generator(device="cuda").manual_seed(5))
    outs = []
    aw0 = ctx.adjoint_workspace(0, 1)
    for _ in range(2):
        lamQ = torch.empty_like(Q0)
        lamMK = torch.empty((2,) + shape, dtype=torch.float64, device="cuda")
        ctx.les_rhs_vjp(Q0, lamR, lamQ, lamMK, aw0)
        outs.append((lamQ.clone(), lamMK.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_adjoint_rejects_unsupported_settings(lj, torch):
    shape = (8, 8, 8)
    ctx, xyz = _jet(lj, torch, shape)  # CFL time step: not supported
    Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
    ctx.les_init_jet(xyz, 1, 1e-3, Q)
    aw = ctx.adjoint_workspace(2, 1)
    with pytest.raises(lj.LesError) as e:
        ctx.les_adjoint_window(Q, 0.0, 2, 1, 3, aw)
    assert e.value.code == lj.LES_ERR_UNSUPPORTED


@pytest.mark.parametrize("radius", [0.5, 5.0])
def test_window_gradient_against_torch_autograd(lj, torch, radius):
    """The hand-written adjoint against torch.autograd through the independent
    FP64 torch restatement of the step (16 x 8 x 8 jet, 6 steps, checkpoint
    every 2), on the shear-layer surface and on the stated r = 5 surface; the
    window's J also against the C oracle's window."""
    import oracle
    from oracle import torch_ref
    shape = (16, 8, 8)
    amps = lj.synth.forcing_amplitudes(9, scale=2e-2)
    xyz = lj.synth.jet_grid(*shape)
    P = oracle.params(Re=500.0)
    M = oracle.metrics(xyz, (0, 0, 1))
    Q0 = oracle.init_jet(P, xyz, seed=1, noise=1e-3)
    dt, nsteps, K = 1e-3, 6, 2
    js = _j_surface(lj, shape, radius)
    case = torch_ref.Case(M, xyz, Re=500.0)
    a = torch.tensor(amps, dtype=torch.float64, requires_grad=True)
    Jt, _ = case.window(torch.from_numpy(Q0), a, 0.0, dt, nsteps, js)
    Jt.backward()
    g_ref = a.grad.numpy()

    ctx = lj.Context(lj.make_params(Re=500.0, dt_mode=lj.DT_FIXED, dt_fixed=dt,
                                    amp=tuple(amps)), shape, "cuda:0")
    ctx.les_set_grid(torch.from_numpy(xyz).cuda())
    aw = ctx.adjoint_workspace(nsteps, K)
    J, g = ctx.les_adjoint_window(torch.from_numpy(Q0).cuda(), 0.0, nsteps, K, js, aw)
    assert math.isclose(J, float(Jt.detach()), rel_tol=1e-11), (J, float(Jt.detach()))
    # and the C oracle's window (its steps, then its functional term)
    Po = oracle.params(Re=500.0, dt_mode=1, dt_fixed=dt, amp=tuple(amps))
    J_orc = oracle.window_functional(Po, Q0, M, xyz, nsteps, 0.0, js)
    assert math.isclose(J, J_orc, rel_tol=2e-11), (J, J_orc)
    gmax = np.abs(g_ref).max()
    assert gmax > 0
    # the r = 5 gradient reaches the surface only through the numerical domain
    # of dependence (about 1e-17 here), so it carries more relative round-off
    tol = 1e-9 if radius < 1.0 else 1e-6
    assert np.allclose(np.array(g), g_ref, rtol=0, atol=tol * gmax), (g, g_ref)


def test_functional_along_fp64_and_mixed_forward_runs(lj, torch):
    """les_surface_functional summed over a forward run: equal to the adjoint
    window's J in FP64, and within 1e-5 of it with the FP32-mixed forward
    (default and compact forms)."""
    shape = (16, 14, 16)
    amps = lj.synth.forcing_amplitudes(9, scale=2e-2)
    xyz = torch.from_numpy(lj.synth.jet_grid(*shape)).cuda()
    j5 = _j_surface(lj, shape, 0.5)
    nsteps, dt = 6, 1e-3
    out = {}
    for prec in (lj.PREC_FP64, lj.PREC_MIXED, lj.PREC_MIXED_COMPACT):
        ctx = lj.Context(lj.make_params(Re=500.0, dt_mode=lj.DT_FIXED, dt_fixed=dt, amp=tuple(amps),
                                        precision=prec), shape, "cuda:0")
        ctx.les_set_grid(xyz)
        Q = torch.empty((5,) + shape, dtype=torch.float64, device="cuda")
        ctx.les_init_jet(xyz, 1, 1e-3, Q)
        if prec == lj.PREC_FP64:
            aw = ctx.adjoint_workspace(nsteps, 2)
            out["window"], _ = ctx.les_adjoint_window(Q, 0.0, nsteps, 2, j5, aw)
        ctx.les_set_time(0.0)
        J = 0.0
        for _ in range(nsteps):
            ctx.les_run_n_steps(1, Q)
            J += ctx.les_surface_functional(Q, j5, dt)
        out[prec] = J
    assert out["window"] > 0
    assert math.isclose(out[lj.PREC_FP64], out["window"], rel_tol=1e-12)
    for prec in (lj.PREC_MIXED, lj.PREC_MIXED_COMPACT):
        assert math.isclose(out[prec], out["window"], rel_tol=1e-5), (prec, out)
