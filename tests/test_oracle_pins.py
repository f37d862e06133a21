"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms of linearised/1-D special cases, discrete
invariants (metric identity, free-stream preservation, telescoping
conservation), the RK amplification polynomial, locality of the stencil, and
the boundary-condition invariants.  A dropped term, a wrong sign or a
transposed index anywhere in the residual breaks at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_2301_00817_gb300 import synth

GAMMA = 1.4
HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------------ Philox

def test_philox_known_answers(orc):
    """Philox4x32-10 against the published known-answer vectors."""
    path = os.path.join(HERE, "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        assert orc.philox4x32_10(vals[0:4], vals[4:6]) == tuple(vals[6:10])


def test_box_muller_normals_are_standard(orc):
    """Box-Muller over Philox gives N(0,1): moments and a KS test."""
    stats = pytest.importorskip("scipy.stats")
    z = np.array([orc.normals3(7, n) for n in range(40000)]).reshape(-1)
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1.0) < 0.03
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # distinct nodes and distinct seeds decorrelate
    a = np.array([orc.normals3(1, n) for n in range(4000)])
    b = np.array([orc.normals3(2, n) for n in range(4000)])
    assert abs(np.corrcoef(a[:, 0], b[:, 0])[0, 1]) < 0.06
    assert abs(np.corrcoef(a[:, 0], a[:, 2])[0, 1]) < 0.06


# ------------------------------------------------ constants the paper prints

def _paper_constants():
    """tests/golden/paper_constants.txt as {name: value}."""
    from fractions import Fraction
    out = {}
    with open(os.path.join(HERE, "golden", "paper_constants.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            name, value = line.split()[:2]
            if value.startswith("sqrt("):
                out[name] = math.sqrt(float(value[5:-1]))
            else:
                out[name] = float(Fraction(value))
    return out


def test_paper_constants_are_the_defaults(orc):
    """The oracle's and the library binding's default parameters are the
    constants the paper prints (Pr, Pr_sgs, C_s, k2, k4), and the oracle's
    laminar viscosity uses the printed Sutherland constant."""
    c = _paper_constants()
    import paper_2301_00817_gb300 as lj
    for P in (orc.params(), lj.make_params()):
        for name in ("Pr", "Pr_sgs", "Cs", "k2", "k4"):
            assert getattr(P, name) == c[name], name
    # mu_lam at a node of temperature T: (M_j/Re) T^1.5 (1 + S)/(T + S), S = S1/T_ref
    P = orc.params(Re=1000.0)
    prim = np.empty((5, 8, 8, 8))
    prim[0], prim[1], prim[2], prim[3] = 1.3, 0.0, 0.0, 0.0
    prim[4] = 1.3 * 1.7 / GAMMA  # T = gamma p / rho = 1.7
    Q = orc.prim_to_cons(P, prim)
    M = orc.metrics(synth.jet_grid(8, 8, 8))
    S = c["S1_K"] / P.T_ref
    mu = (P.Mj / 1000.0) * 1.7 ** 1.5 * (1.0 + S) / (1.7 + S)
    assert np.allclose(orc.mu_eff(P, Q, M)[0], mu, rtol=1e-14, atol=0)


def test_runge_kutta_coefficients_and_stability_statement(orc):
    """The oracle's five-stage driver has the amplification factor of the
    printed coefficients, G(z) = 1 + a5 z (1 + a4 z (1 + a3 z (1 + a2 z (1 +
    a1 z)))) for dQ/dt = lambda Q, z = lambda dt; and |G(i y)| <= 1 for
    |y| <= 2 sqrt 2, the paper's linear stability statement."""
    c = _paper_constants()
    alpha = [c[f"alpha{m}"] for m in range(1, 6)]

    def G(z):
        g = 1.0
        for a in alpha:
            g = 1.0 + a * z * g
        return g

    for lam_dt in (-0.3, -1.1, -2.5, 0.7):
        Q = np.ones((1, 1))
        out = orc.rk5(Q, lambda q: -lam_dt * q, 1.0)  # RHS = -lambda Q, dt = 1
        assert out[0, 0] == pytest.approx(G(lam_dt), rel=1e-15, abs=1e-15)
    y = np.linspace(0.0, c["cfl_max"], 2001)
    assert np.abs(G(1j * y)).max() <= 1.0 + 1e-15


# ----------------------------------------------------------------- metrics

def _coord_jacobian(xyz, periodic, shift):
    """X[c, d] = d x_c / d xi_d by numpy finite differences (central; one-sided
    second order at non-periodic faces; periodic wrap with the period shift)."""
    X = np.empty((3, 3) + xyz.shape[1:])
    sh = np.asarray(shift).reshape(3, 3)
    for c in range(3):
        for d in range(3):
            f = xyz[c]
            if periodic[d]:
                fp = np.roll(f, -1, axis=d)
                fm = np.roll(f, 1, axis=d)
                idx_last = [slice(None)] * 3
                idx_last[d] = -1
                idx_first = [slice(None)] * 3
                idx_first[d] = 0
                fp[tuple(idx_last)] += sh[d, c]
                fm[tuple(idx_first)] -= sh[d, c]
                X[c, d] = 0.5 * (fp - fm)
            else:
                X[c, d] = np.gradient(f, axis=d, edge_order=2)
    return X


@pytest.mark.parametrize("case", ["jet", "wavy_box"])
def test_metric_identity(orc, case):
    """Reading A1: the nine metrics are the inverse of d(x,y,z)/d(xi,eta,zeta)
    at every node and J^-1 is its determinant (a wrong eta row fails)."""
    if case == "jet":
        xyz, per, shift = synth.jet_grid(20, 12, 16), (0, 0, 1), np.zeros(9)
    else:
        xyz, shift = synth.box_grid((10, 9, 8), (1.0, 1.3, 0.7), wave=0.3)
        per = (1, 1, 1)
    M = orc.metrics(xyz, per, shift)
    X = _coord_jacobian(xyz, per, shift)
    Mm = M[:9].reshape((3, 3) + xyz.shape[1:])  # Mm[d, c] = d xi_d / d x_c
    ident = np.einsum("dc...,ce...->de...", Mm, X)
    assert np.abs(ident - np.eye(3)[:, :, None, None, None]).max() < 1e-12
    det = np.linalg.det(np.moveaxis(X, (0, 1), (-2, -1)))
    assert np.allclose(det, M[9], rtol=1e-13, atol=0)
    assert (M[9] > 0).all()


def _central(f, d, periodic):
    """Central difference along axis d at interior nodes (NaN elsewhere for a
    non-periodic axis)."""
    out = 0.5 * (np.roll(f, -1, axis=d) - np.roll(f, 1, axis=d))
    if not periodic:
        idx = [slice(None)] * 3
        idx[d] = 0
        out[tuple(idx)] = np.nan
        idx[d] = -1
        out[tuple(idx)] = np.nan
    return out


def _wavy_open_grid(n=(11, 10, 9), wave=0.3):
    """The wavy box's coordinates taken as a grid with no periodic direction."""
    xyz, _ = synth.box_grid(n, (1.0, 1.3, 0.7), wave=wave)
    return xyz


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1), (0, 0, 1)])
def test_conservative_metrics_geometric_conservation(orc, periodic):
    """The conservative metric form satisfies the discrete geometric
    conservation law sum_r delta_r (J^-1 r_c) = 0 at every interior node of a
    non-separable grid, to round-off; the cross-product form does not (its
    error is O(h^2), far above round-off here)."""
    xyz, shift = synth.box_grid((11, 10, 9), (1.0, 1.3, 0.7), wave=0.3)
    if not any(periodic):
        shift = np.zeros(9)
    gcl = {}
    for form in (0, 1):
        M = orc.metrics(xyz, periodic, shift, form=form)
        cof = M[:9] * M[9]  # J^-1 r_c, row r = 3r + c
        worst = 0.0
        for c in range(3):
            total = sum(_central(cof[3 * r + c], r, periodic[r]) for r in range(3))
            inner = total[~np.isnan(total)]
            worst = max(worst, np.abs(inner).max())
        gcl[form] = worst / np.abs(cof).max()
    assert gcl[1] < 1e-14, gcl
    assert gcl[0] > 1e-5, gcl


def test_conservative_metrics_exact_on_affine_grid(orc):
    """On an affine grid x = A xi + b every second-order difference is exact:
    both forms give A^-1 and det A at every node, faces included."""
    rng = np.random.default_rng(4)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    n = (7, 6, 5)
    I = np.stack(np.meshgrid(*[np.arange(m, dtype=np.float64) for m in n], indexing="ij"))
    xyz = np.einsum("cd,d...->c...", A, I) + np.array([0.3, -1.0, 2.0])[:, None, None, None]
    Ainv = np.linalg.inv(A)
    for form in (0, 1):
        M = orc.metrics(xyz, (0, 0, 0), None, form=form)
        for r in range(3):
            for c in range(3):
                assert np.abs(M[3 * r + c] - Ainv[r, c]).max() < 1e-13, (form, r, c)
        assert np.abs(M[9] - np.linalg.det(A)).max() < 1e-13


def test_conservative_metrics_converge_to_the_mapping(orc):
    """On a smooth non-separable mapping both forms approach the analytic
    metrics at second order (the error falls about 4x per halving of h)."""
    def grid(m):
        s = np.arange(m, dtype=np.float64) / (m - 1)
        S0, S1, S2 = np.meshgrid(s, s, s, indexing="ij")
        x = S0 + 0.1 * np.sin(2.0 * S1) * np.cos(1.5 * S2)
        y = S1 + 0.1 * np.sin(1.7 * S0) * np.sin(1.3 * S2)
        z = S2 + 0.1 * np.cos(1.1 * S0) * np.sin(1.9 * S1)
        h = 1.0 / (m - 1)
        X = np.empty((3, 3) + S0.shape)  # analytic d x_c / d xi_d (xi = s/h)
        X[0, 0], X[0, 1], X[0, 2] = 1.0, 0.2 * np.cos(2.0 * S1) * np.cos(1.5 * S2), \
            -0.15 * np.sin(2.0 * S1) * np.sin(1.5 * S2)
        X[1, 0], X[1, 1], X[1, 2] = 0.17 * np.cos(1.7 * S0) * np.sin(1.3 * S2), 1.0, \
            0.13 * np.sin(1.7 * S0) * np.cos(1.3 * S2)
        X[2, 0], X[2, 1], X[2, 2] = -0.11 * np.sin(1.1 * S0) * np.sin(1.9 * S1), \
            0.19 * np.cos(1.1 * S0) * np.cos(1.9 * S1), 1.0
        X *= h
        Minv = np.linalg.inv(np.moveaxis(X, (0, 1), (-2, -1)))  # [..., d, c]
        return np.stack([x, y, z]), np.moveaxis(Minv, (-2, -1), (0, 1))
    for form in (0, 1):
        errs = []
        for m in (9, 17, 33):
            xyz, exact = grid(m)
            M = orc.metrics(xyz, (0, 0, 0), None, form=form)
            h = 1.0 / (m - 1)
            errs.append(max(np.abs(M[3 * r + c] - exact[r, c]).max() * h
                            for r in range(3) for c in range(3)))
        rates = [errs[i] / errs[i + 1] for i in range(2)]
        assert all(3.3 < q < 4.8 for q in rates), (form, errs, rates)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 1)])
def test_conservative_metrics_converge_on_the_periodic_box(orc, periodic):
    """The wavy box (coordinates jump by one period across each periodic
    wrap): the conservative metrics approach the analytic inverse Jacobian at
    second order at every node, wrapped neighbours included."""
    L, wave, tp = (1.0, 1.3, 0.7), 0.2, 2.0 * math.pi
    errs = []
    for m in (8, 16, 32):
        xyz, shift = synth.box_grid((m, m, m), L, wave=wave)
        S = np.stack(np.meshgrid(*[np.arange(m) / m] * 3, indexing="ij"))
        X = np.zeros((3, 3) + S.shape[1:])  # d x_c / d i_d of box_grid's mapping
        X[0, 0] = L[0] / m
        X[0, 1] = wave * L[0] * np.cos(tp * S[1]) * np.sin(tp * S[2]) / m
        X[0, 2] = wave * L[0] * np.sin(tp * S[1]) * np.cos(tp * S[2]) / m
        X[1, 0] = wave * L[1] * np.cos(tp * S[0]) * np.cos(tp * S[2]) / m
        X[1, 1] = L[1] / m
        X[1, 2] = -wave * L[1] * np.sin(tp * S[0]) * np.sin(tp * S[2]) / m
        X[2, 0] = -wave * L[2] * np.sin(tp * S[0]) * np.sin(tp * S[1]) / m
        X[2, 1] = wave * L[2] * np.cos(tp * S[0]) * np.cos(tp * S[1]) / m
        X[2, 2] = L[2] / m
        exact = np.moveaxis(np.linalg.inv(np.moveaxis(X, (0, 1), (-2, -1))), (-2, -1), (0, 1))
        M = orc.metrics(xyz, periodic, shift, form=1)
        errs.append(max(np.abs(M[3 * r + c] - exact[r, c]).max() / m
                        for r in range(3) for c in range(3)))
    rates = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.3 < q < 4.8 for q in rates), (errs, rates)


@pytest.mark.parametrize("sgs", [0, 1])
def test_free_stream_preservation_conservative_metrics(orc, sgs):
    """With conservative metrics a uniform state on a non-separable grid has
    zero residual to round-off, at all interior nodes (open faces, frozen);
    with the cross-product form it does not."""
    xyz = _wavy_open_grid()
    P = orc.params(periodic=(0, 0, 0), bc=0, sgs_model=sgs, Re=300.0)
    Q = orc.prim_to_cons(P, synth.uniform_prim(xyz.shape[1:], u=0.9, v=-0.3, w=0.2))
    res = {}
    for form in (0, 1):
        M = orc.metrics(xyz, (0, 0, 0), None, form=form)
        R = orc.rhs(P, Q, M)
        res[form] = np.abs(R).max() / (np.abs(M[9]).max() * 10.0)
    assert res[1] < 1e-14, res
    assert res[0] > 1e-5, res


# --------------------------------------------------------- jet grid and IC

def test_jet_grid_recipe():
    x, r, th = synth.jet_lines(48, 24, 32)
    assert x[0] == 0.0 and abs(x[-1] - 20.0) < 1e-12
    assert np.allclose(np.diff(x)[1:] / np.diff(x)[:-1], 1.01, rtol=1e-12)
    assert abs(r[0] - 0.02) < 1e-14 and abs(r[-1] - 10.0) < 1e-12
    dr = np.diff(r)
    assert (dr > 0).all()
    rmid = 0.5 * (r[1:] + r[:-1])
    assert abs(rmid[np.argmin(dr)] - 0.5) < 0.1
    assert np.allclose(np.diff(th), 2 * math.pi / 32)


def test_jet_initial_condition_profile(orc):
    """Noise-free IC is the tanh profile with rho = 1, p = 1/gamma; the noise
    is noise*U_j times the node's three normals."""
    P = orc.params()
    xyz = synth.jet_grid(8, 10, 8)
    Q = orc.init_jet(P, xyz, seed=3, noise=0.0)
    r = np.sqrt(xyz[1] ** 2 + xyz[2] ** 2)
    u = 0.7 * (1.0 + np.tanh((0.5 - r) / 0.1))
    assert np.allclose(Q[0], 1.0, rtol=0, atol=0)
    assert np.allclose(Q[1], u, rtol=1e-15, atol=1e-15)
    assert np.abs(Q[2:4]).max() == 0.0
    assert np.allclose(Q[4], 1.0 / (GAMMA * 0.4) + 0.5 * u * u, rtol=1e-15)
    Qn = orc.init_jet(P, xyz, seed=3, noise=1e-3)
    z = np.array([orc.normals3(3, n) for n in range(xyz[0].size)]).T.reshape((3,) + xyz.shape[1:])
    assert np.allclose(Qn[2], 1e-3 * 1.4 * z[1], rtol=1e-14, atol=1e-15)
    assert np.allclose(Qn[1], u + 1e-3 * 1.4 * z[0], rtol=1e-14, atol=1e-15)


# ------------------------------------------------- free stream / conservation

@pytest.mark.parametrize("sgs", [0, 1, 2])
def test_free_stream_preservation_jet_grid(orc, sgs):
    """A uniform state on the curvilinear jet grid has zero residual to
    round-off (Reading A9 makes the dissipation vanish exactly)."""
    P = orc.params(sgs_model=sgs)
    xyz = synth.jet_grid(24, 16, 16)
    M = orc.metrics(xyz, (0, 0, 1))
    Q = orc.prim_to_cons(P, synth.uniform_prim(xyz.shape[1:], u=0.9, v=-0.3, w=0.2))
    R = orc.rhs(P, Q, M)
    # flux scale: J^-1 |grad xi| (rho|u|^2 + p)
    scale = np.abs(M[9]).max() * 10.0
    assert np.abs(R).max() / scale < 1e-13


@pytest.mark.parametrize("wave", [0.0, 0.25])
@pytest.mark.parametrize("sgs", [1, 2, 3])
def test_discrete_conservation_periodic_box(orc, wave, sgs):
    """Interface fluxes telescope: sum J^-1 Q is constant in a periodic box."""
    P = orc.params(periodic=(1, 1, 1), bc=0, sgs_model=sgs, Re=200.0, cfl=0.8)
    L = (1.0, 1.2, 0.9)
    xyz, shift = synth.box_grid((12, 10, 9), L, wave=wave)
    M = orc.metrics(xyz, (1, 1, 1), shift)
    Q = orc.prim_to_cons(P, synth.smooth_periodic_prim(xyz, L, amp=0.2, seed=4))
    tot0 = orc.totals(Q, M)
    Qn, t = orc.run(P, Q, M, xyz, 20)
    tot1 = orc.totals(Qn, M)
    assert t > 0 and np.isfinite(Qn).all()
    assert np.abs(Qn - Q).max() > 1e-3  # the state really evolved
    scale = np.abs(orc.totals(np.abs(Q), M)).max()
    assert np.abs(tot1 - tot0).max() / scale < 1e-13


# ------------------------------------------------- manufactured solution

def _mms_exact_divergence(Re, Mj=1.4, Pr=0.72, Tref=288.15):
    """Exact d/dx_j (F_inviscid_j - F_viscous_j) of the continuous System I
    equations (Eq. modified_system_I with sigma = 0) for analytic periodic
    fields, by symbolic differentiation."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    tp = 2 * sp.pi
    rho = 1 + sp.Rational(1, 10) * sp.sin(tp * x) * sp.cos(tp * y) + sp.Rational(1, 20) * sp.sin(tp * z)
    u = sp.Rational(3, 10) + sp.Rational(1, 10) * sp.cos(tp * (x + z))
    v = -sp.Rational(1, 5) + sp.Rational(1, 10) * sp.sin(tp * y) * sp.cos(tp * z)
    w = sp.Rational(1, 10) + sp.Rational(1, 10) * sp.sin(tp * (x - y))
    p = sp.Rational(5, 7) * (1 + sp.Rational(1, 10) * sp.cos(tp * x) * sp.sin(tp * y + tp * z))
    g = sp.Rational(7, 5)
    X = (x, y, z)
    U = (u, v, w)
    e = p / (g - 1) + rho * (u * u + v * v + w * w) / 2
    T = g * p / rho
    S = sp.Float(110.4) / sp.Float(Tref)
    mu = (sp.Float(Mj) / sp.Float(Re)) * T ** sp.Rational(3, 2) * (1 + S) / (T + S)
    kap = mu / ((g - 1) * sp.Float(Pr))
    grad = [[sp.diff(U[i], X[j]) for j in range(3)] for i in range(3)]
    div = grad[0][0] + grad[1][1] + grad[2][2]
    tau = [[mu * (grad[i][j] + grad[j][i]) - (2 * mu / 3) * div * (1 if i == j else 0)
            for j in range(3)] for i in range(3)]
    q = [-kap * sp.diff(T, X[j]) for j in range(3)]
    res = []
    res.append(sum(sp.diff(rho * U[j], X[j]) for j in range(3)))
    for i in range(3):
        res.append(sum(sp.diff(rho * U[i] * U[j] + (p if i == j else 0) - tau[i][j], X[j])
                       for j in range(3)))
    res.append(sum(sp.diff((e + p) * U[j] - sum(tau[i][j] * U[i] for i in range(3)) + q[j], X[j])
                   for j in range(3)))
    visc = []
    for i in range(3):
        visc.append(sum(sp.diff(-tau[i][j], X[j]) for j in range(3)))
    visc.append(sum(sp.diff(-sum(tau[i][j] * U[i] for i in range(3)) + q[j], X[j]) for j in range(3)))
    f_prim = sp.lambdify((x, y, z), [rho, u, v, w, p], "numpy")
    f_res = sp.lambdify((x, y, z), res, "numpy")
    f_visc = sp.lambdify((x, y, z), visc, "numpy")
    return f_prim, f_res, f_visc


def test_manufactured_solution_second_order(orc):
    """J * RHS converges at second order to the exact flux divergence of the
    paper's continuous equations on a non-separable periodic curvilinear grid
    (viscous terms made O(1) with a low Reynolds number)."""
    Re = 20.0
    f_prim, f_res, f_visc = _mms_exact_divergence(Re)
    P = orc.params(periodic=(1, 1, 1), bc=0, Re=Re, sgs_model=0)
    errs, vmag = [], None
    for n in (12, 24, 48):
        xyz, shift = synth.box_grid((n, n, n), (1.0, 1.0, 1.0), wave=0.2)
        M = orc.metrics(xyz, (1, 1, 1), shift)
        prim = np.array([np.broadcast_to(f, xyz.shape[1:]) for f in f_prim(*xyz)])
        Q = orc.prim_to_cons(P, prim)
        R = orc.rhs(P, Q, M)
        JR = R / M[9]
        exact = np.array([np.broadcast_to(f, xyz.shape[1:]) for f in f_res(*xyz)])
        errs.append(np.abs(JR - exact).max())
        vmag = np.abs(np.array([np.broadcast_to(f, xyz.shape[1:]) for f in f_visc(*xyz)])).max()
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.4 < r1 < 4.8 and 3.6 < r2 < 4.5, errs
    # the finest error is far below the viscous contribution itself, so a sign
    # or factor error in the viscous fluxes could not hide in the tolerance
    assert errs[2] < 0.05 * vmag, (errs, vmag)


# ------------------------------------------------------- 1-D special cases

def _cartesian_box(n, h):
    L = tuple(m * h for m in n)
    return synth.box_grid(n, L, wave=0.0)


@pytest.mark.parametrize("periodic_x", [1, 0])
def test_one_dimensional_jst_reduction(orc, periodic_x):
    """Uniform Cartesian grid, inviscid, variation along x only: the residual
    equals the textbook 1-D central flux plus JST/Turkel-Vatsa dissipation
    with the sensor normalised by the pressure sum.  On a non-periodic line
    the faces use the paper's closure (DW)_{1/2} = -(DW)_{1+1/2} and the face
    sensor copies its neighbour."""
    n, h = (10, 5, 5), 0.1
    xyz, shift = _cartesian_box(n, h)
    per = (periodic_x, 1, 1)
    P = orc.params(periodic=per, bc=0, Re=0.0, sgs_model=0, k2=0.25, k4=0.016)
    M = orc.metrics(xyz, per, shift)
    xs = xyz[0][:, 0, 0]
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * xs / 0.8)
    u = 0.5 + 0.3 * np.cos(2 * np.pi * xs / 0.8)
    p = (1.0 / GAMMA) * (1.0 + 0.4 * (xs > 0.35) + 0.3 * (xs < 0.15))
    prim = np.zeros((5,) + n)
    prim[0] = rho[:, None, None]
    prim[1] = u[:, None, None]
    prim[4] = p[:, None, None]
    Q = orc.prim_to_cons(P, prim)
    R = orc.rhs(P, Q, M)
    # textbook 1-D JST on the line, fluxes per unit area h^2
    E = p / (GAMMA - 1) + 0.5 * rho * u * u
    f = np.array([rho * u, rho * u * u + p, 0 * u, 0 * u, (E + p) * u])
    Wv = np.array([rho, rho * u, 0 * u, 0 * u, E + p])
    a = np.sqrt(GAMMA * p / rho)
    lx, ly = (np.abs(u) + a) / h, a / h
    lbar = lx * (1 + 2 * np.sqrt(ly / lx))
    m = n[0]
    nu = np.empty(m)
    for i in range(m):
        c = i
        if not periodic_x:
            c = min(max(i, 1), m - 2)  # face sensor = neighbour's sensor
        pp, p0, pm = p[(c + 1) % m], p[c], p[(c - 1) % m]
        nu[i] = abs(pp - 2 * p0 + pm) / (pp + 2 * p0 + pm)
    nint = m if periodic_x else m - 1
    Fh = np.zeros((5, nint))
    for i in range(nint):
        b = (i + 1) % m
        D1 = Wv[:, b] - Wv[:, i]
        if periodic_x or i > 0:
            Dm = Wv[:, i] - Wv[:, (i - 1) % m]
        else:
            Dm = -D1
        if periodic_x or i < m - 2:
            Dp = Wv[:, (i + 2) % m] - Wv[:, b]
        else:
            Dp = -D1
        e2 = 0.25 * max(nu[i], nu[b])
        e4 = max(0.0, 0.016 - e2)
        lam = 0.5 * (lbar[i] + lbar[b])
        Fh[:, i] = h * h * 0.5 * (f[:, i] + f[:, b]) - h ** 3 * lam * (e2 * D1 - e4 * (Dp - 2 * D1 + Dm))
    expect = np.zeros((5, m))
    for i in range(m):
        if periodic_x:
            expect[:, i] = Fh[:, i] - Fh[:, (i - 1) % m]
        elif 0 < i < m - 1:
            expect[:, i] = Fh[:, i] - Fh[:, i - 1]
    for c in range(5):
        assert np.allclose(R[c], expect[c][:, None, None], rtol=0, atol=1e-14 * np.abs(Fh).max())


@pytest.mark.parametrize("d", [0, 1, 2])
def test_fourth_difference_mode_decays(orc, d):
    """Reading A8/A10: at rest with uniform p (eps2 = 0) a density wave along
    direction d on anisotropic cells is damped by the fourth difference:
    J RHS_rho = 16 lbar_d k4 sin^4(k h_d/2) rho', with
    lbar_d = (a/h_d)[1 + sum over the other two e of (h_d/h_e)^0.5]."""
    n = [5, 5, 5]
    n[d] = 16
    n = tuple(n)
    hs = (0.05, 0.08, 0.03)
    eps = 1e-8
    xyz, shift = synth.box_grid(n, tuple(m * h for m, h in zip(n, hs)))
    P = orc.params(periodic=(1, 1, 1), bc=0, Re=0.0, sgs_model=0)
    M = orc.metrics(xyz, (1, 1, 1), shift)
    xs = xyz[d]
    kw = 2 * np.pi * 3 / (n[d] * hs[d])
    prim = synth.uniform_prim(n)
    prim[0] = 1.0 + eps * np.sin(kw * xs)
    Q = orc.prim_to_cons(P, prim)
    JR = orc.rhs(P, Q, M)[0] / M[9]
    h = hs[d]
    lbar = (1.0 / h) * (1.0 + sum(math.sqrt(h / hs[e]) for e in range(3) if e != d))
    expect = 16 * lbar * 0.016 * np.sin(kw * h / 2) ** 4 * (eps * np.sin(kw * xs))
    assert np.allclose(JR, expect, rtol=0, atol=1e-5 * np.abs(expect).max())
    assert np.sum(JR * (prim[0] - 1.0)) > 0  # d rho/dt = -J RHS opposes the mode


def test_fourth_difference_boundary_closure(orc):
    """Sec. "Centerline Boundary Condition": with (DW)_{1/2} = -(DW)_{1+1/2}
    the first interface's fourth difference is DW_{3/2} - 3 DW_{1/2}.  A
    linear density ramp (slope c per node) at rest is annihilated by the
    interior fourth difference; the closure leaves J RHS_rho = +2 lbar k4 c
    at the node next to the low face and -2 lbar k4 c next to the high face."""
    n, h, c = (10, 5, 5), 0.05, 1e-9
    L = (n[0] * h, n[1] * h, n[2] * h)
    xyz, shift = synth.box_grid(n, L)
    P = orc.params(periodic=(0, 1, 1), bc=0, Re=0.0, sgs_model=0)
    M = orc.metrics(xyz, (0, 1, 1), shift)
    prim = synth.uniform_prim(n)
    prim[0] = 1.0 + c * np.arange(n[0])[:, None, None]
    Q = orc.prim_to_cons(P, prim)
    JR = orc.rhs(P, Q, M)[0] / M[9]
    lbar = 3.0 / h
    expect = np.zeros(n)
    expect[1] = 2 * lbar * 0.016 * c
    expect[-2] = -2 * lbar * 0.016 * c
    expect[0] = expect[-1] = 0.0
    assert np.allclose(JR, expect, rtol=0, atol=1e-6 * 2 * lbar * 0.016 * c)


def test_viscous_shear_wave_rate(orc):
    """Reading A4/A11: a shear wave u(y) at uniform rho, p decays by the
    compact viscous second difference with mu = M_j/Re (T = 1)."""
    n, h, eps = (5, 16, 5), 0.05, 1e-6
    xyz, shift = _cartesian_box(n, h)
    Re = 100.0
    P = orc.params(periodic=(1, 1, 1), bc=0, Re=Re, sgs_model=0, k2=0.0, k4=0.0)
    M = orc.metrics(xyz, (1, 1, 1), shift)
    ys = xyz[1]
    kw = 2 * np.pi * 2 / (n[1] * h)
    prim = synth.uniform_prim(n)
    prim[1] = eps * np.sin(kw * ys)
    Q = orc.prim_to_cons(P, prim)
    JR = orc.rhs(P, Q, M) / M[9]
    mu = 1.4 / Re
    expect = mu * 4 * np.sin(kw * h / 2) ** 2 / h ** 2 * eps * np.sin(kw * ys)
    assert np.allclose(JR[1], expect, rtol=0, atol=1e-8 * np.abs(expect).max())
    assert np.abs(JR[0]).max() < 1e-14 and np.abs(JR[2:4]).max() < 1e-14


def test_heat_conduction_sign_and_rate(orc):
    """Reading A2: at rest with uniform p, a temperature wave in the energy
    equation obeys J RHS_e = kappa 4 sin^2(kh/2)/h^2 T' (heat flows from hot
    to cold), kappa = (M_j/Re)/((gamma-1) Pr)."""
    n, h, eps = (16, 5, 5), 0.05, 1e-7
    xyz, shift = _cartesian_box(n, h)
    Re = 100.0
    P = orc.params(periodic=(1, 1, 1), bc=0, Re=Re, sgs_model=0, k2=0.0, k4=0.0)
    M = orc.metrics(xyz, (1, 1, 1), shift)
    xs = xyz[0]
    kw = 2 * np.pi * 3 / (n[0] * h)
    Tp = eps * np.cos(kw * xs)
    prim = synth.uniform_prim(n)
    prim[0] = 1.0 / (1.0 + Tp)  # T = gamma p / rho = 1 + T'
    Q = orc.prim_to_cons(P, prim)
    JR = orc.rhs(P, Q, M) / M[9]
    kap = (1.4 / Re) / (0.4 * 0.72)
    expect = kap * 4 * np.sin(kw * h / 2) ** 2 / h ** 2 * Tp
    assert np.allclose(JR[4], expect, rtol=0, atol=1e-5 * np.abs(expect).max())


# -------------------------------------------------------------- SGS / mu

def _linear_velocity_box(orc, grad, sgs, n=(7, 7, 7), h=0.1):
    xyz = _cartesian_box(n, h)[0]
    P = orc.params(periodic=(0, 0, 0), bc=0, sgs_model=sgs, Re=1e4)
    M = orc.metrics(xyz, (0, 0, 0), np.zeros(9))
    prim = synth.uniform_prim(n)
    for i in range(3):
        prim[1 + i] = sum(grad[i][j] * xyz[j] for j in range(3))
    Q = orc.prim_to_cons(P, prim)
    MK = orc.mu_eff(P, Q, M)
    mu_l = (1.4 / 1e4) * 1.0
    return MK, mu_l, h


def test_sgs_closed_forms(orc):
    """Smagorinsky and Vreman on linear velocity fields (exact gradients)."""
    Cs = 0.148
    s = 0.7
    shear = [[0, s, 0], [0, 0, 0], [0, 0, 0]]  # u = s y
    MK, mu_l, h = _linear_velocity_box(orc, shear, 1)
    T = np.ones_like(MK[0])
    assert np.allclose(MK[0], mu_l * T + (Cs * h) ** 2 * s, rtol=1e-12)
    MK, mu_l, h = _linear_velocity_box(orc, shear, 2)
    assert np.allclose(MK[0], mu_l, rtol=1e-12)  # Vreman vanishes for pure shear
    rot = [[0, -0.5, 0], [0.5, 0, 0], [0, 0, 0]]
    MK, mu_l, h = _linear_velocity_box(orc, rot, 1)
    assert np.allclose(MK[0], mu_l, rtol=1e-12)  # no strain in solid rotation
    rng = np.random.default_rng(5)
    G = rng.normal(size=(3, 3))
    MK, mu_l, h = _linear_velocity_box(orc, G, 2)
    alpha = G.T  # alpha_ij = d u_j / d x_i
    beta = h * h * alpha.T @ alpha
    Bb = 0.5 * (np.trace(beta) ** 2 - np.trace(beta @ beta))  # 2nd invariant
    mu_v = 2.5 * Cs * Cs * np.sqrt(Bb / np.sum(alpha * alpha))
    assert np.allclose(MK[0], mu_l + mu_v, rtol=1e-12)
    # kappa split with the two Prandtl numbers
    assert np.allclose(MK[1], mu_l / (0.4 * 0.72) + mu_v / (0.4 * 0.9), rtol=1e-12)


# ------------------------------------------------------- dynamic model

def _linear_state(orc, n, h, G, g, U0=(0.2, -0.1, 0.05), rho0=1.1, T0=1.0):
    xyz, _ = synth.box_grid(n, tuple(m * hh for m, hh in zip(n, h)))
    X = xyz.reshape(3, -1)
    prim = np.empty((5,) + n)
    prim[0] = rho0
    prim[1:4] = (G @ X).reshape((3,) + n) + np.asarray(U0)[:, None, None, None]
    prim[4] = rho0 * (T0 + (g @ X).reshape(n)) / GAMMA
    return xyz, prim


def test_dynamic_procedure_linear_fields_closed_form(orc):
    """Constant velocity gradient G and temperature gradient g, uniform
    density, on a Cartesian grid of spacings h: every difference and filter
    is exact, the test filter's variance along d is h_d^2/2, so with
    Sigma = diag(h_d^2/2), D = (h_x h_y h_z)^(1/3) and Delta^ = 2 Delta:
    L = rho G Sigma G^T, K = rho G Sigma g, S^ = S, and
      <num C_ds> = rho [L:S/rho - tr(L/rho) tr S/3],
      <den C_ds> = -6 D^2 rho |S| (S:S - (tr S)^2/3),
      C_I = tr(G Sigma G^T)/(6 D^2 |S|^2),
      Pr_sgs = C_ds (-3 D^2 |S| |g|^2)/(g . G Sigma g)
    (an asymmetric G: a transposed index or a dropped trace term fails)."""
    n, h = (9, 8, 7), (0.1, 0.13, 0.07)
    G = 0.5 * np.array([[1.0, 0.3, -0.2], [0.1, 0.8, 0.4], [-0.3, 0.2, -2.1]])
    g = np.array([0.3, -0.5, 0.8])
    xyz, prim = _linear_state(orc, n, h, G, g)
    P = orc.params(periodic=(0, 0, 0), bc=0, sgs_model=3)
    M = orc.metrics(xyz, (0, 0, 0), None)
    out = orc.dynamic_coefficients(P, orc.prim_to_cons(P, prim), M)
    rho0 = 1.1
    Sig = np.diag([hh * hh / 2 for hh in h])
    S = 0.5 * (G + G.T)
    Smag = math.sqrt(2 * (S * S).sum())
    D2 = (h[0] * h[1] * h[2]) ** (2.0 / 3.0)
    GSG, trS = G @ Sig @ G.T, np.trace(S)
    expect = dict(numC=rho0 * ((GSG * S).sum() - np.trace(GSG) * trS / 3),
                  denC=-6 * D2 * rho0 * Smag * ((S * S).sum() - trS ** 2 / 3),
                  numI=rho0 * np.trace(GSG), denI=6 * D2 * rho0 * Smag ** 2,
                  numP=-3 * D2 * rho0 * Smag * (g @ g), denP=rho0 * g @ (G @ Sig @ g))
    expect["Cd"] = expect["numC"] / expect["denC"]
    expect["CI"] = expect["numI"] / expect["denI"]
    expect["Prt"] = expect["Cd"] * expect["numP"] / expect["denP"]
    assert expect["Cd"] > 0 and expect["CI"] > 0 and expect["Prt"] > 0
    for k, v in expect.items():
        assert abs(out[k] - v) <= 1e-12 * abs(v), (k, out[k], v)


def test_dynamic_procedure_pure_shear_and_dilatation(orc):
    """A unidirectional linear shear has L:S = 0 (C_ds = 0); a pure
    dilatation has no deviatoric part, so numerator and denominator of C_ds
    both vanish: the model acts on the deviatoric strain only."""
    n, h = (8, 9, 7), (0.1, 0.1, 0.1)
    P = orc.params(periodic=(0, 0, 0), bc=0, sgs_model=3)
    for G, both_zero in ((np.array([[0.0, 0.7, 0.0], [0, 0, 0], [0, 0, 0]]), False),
                         (0.4 * np.eye(3), True)):
        xyz, prim = _linear_state(orc, n, h, G, np.zeros(3))
        out = orc.dynamic_coefficients(P, orc.prim_to_cons(P, prim), orc.metrics(xyz, (0, 0, 0)))
        assert abs(out["numC"]) < 1e-15
        assert out["Cd"] == 0.0
        if both_zero:
            assert abs(out["denC"]) < 1e-14
        else:
            assert out["denC"] < -1e-4


def test_test_filter_transfer_function_and_faces(orc):
    """Periodic: a Fourier mode is multiplied by prod_d cos^2(pi m_d/n_d).
    Open directions: linear fields pass unchanged (the face nodes filter only
    along their own face)."""
    n = (12, 10, 8)
    I = np.meshgrid(*[np.arange(m, dtype=float) for m in n], indexing="ij")
    m = (2, 3, 1)
    f = np.cos(2 * np.pi * m[0] * I[0] / n[0] + 0.3) * np.cos(2 * np.pi * m[1] * I[1] / n[1]) \
        * np.sin(2 * np.pi * m[2] * I[2] / n[2] + 1.1)
    gain = np.prod([math.cos(math.pi * m[d] / n[d]) ** 2 for d in range(3)])
    assert np.abs(orc.test_filter(f, (1, 1, 1)) - gain * f).max() < 1e-14
    lin = 0.3 + 1.7 * I[0] - 0.4 * I[1] + 0.9 * I[2]
    assert np.abs(orc.test_filter(lin, (0, 0, 0)) - lin).max() < 1e-13
    q = I[1] ** 2  # curvature along eta: + h^2/2 inside, unchanged on the eta faces
    fq = orc.test_filter(q, (0, 0, 0))
    assert np.abs(fq[:, 1:-1] - (q[:, 1:-1] + 0.5)).max() < 1e-13
    assert np.abs(fq[:, [0, -1]] - q[:, [0, -1]]).max() < 1e-13


def test_dynamic_procedure_invariances(orc):
    """On a non-separable periodic grid with a smooth 3-D state: adding a
    uniform velocity changes nothing (Galilean invariance of L, K and the
    strains); scaling the velocity by s scales the C_ds terms by s^3, the C_I
    terms by s^2 and the Pr_sgs terms by s, leaving the coefficients; a
    uniform temperature shift changes nothing."""
    Lb = (1.0, 1.2, 0.9)
    xyz, shift = synth.box_grid((12, 10, 9), Lb, wave=0.25)
    P = orc.params(periodic=(1, 1, 1), bc=0, sgs_model=3)
    M = orc.metrics(xyz, (1, 1, 1), shift)
    prim = synth.smooth_periodic_prim(xyz, Lb, amp=0.3, seed=4)
    base = orc.dynamic_coefficients(P, orc.prim_to_cons(P, prim), M)
    assert base["Cd"] > 0 and base["denP"] != 0
    moved = prim.copy()
    moved[1:4] += np.array([0.7, -0.4, 0.25])[:, None, None, None]
    gal = orc.dynamic_coefficients(P, orc.prim_to_cons(P, moved), M)
    for k in base:
        assert abs(gal[k] - base[k]) <= 1e-11 * max(abs(base[k]), 1e-300), k
    s = 1.7
    scaled = prim.copy()
    scaled[1:4] *= s
    sc = orc.dynamic_coefficients(P, orc.prim_to_cons(P, scaled), M)
    for k, e in (("numC", 3), ("denC", 3), ("numI", 2), ("denI", 2), ("numP", 1), ("denP", 1)):
        assert abs(sc[k] - s ** e * base[k]) <= 1e-12 * abs(s ** e * base[k]), k
    for k in ("Cd", "CI", "Prt"):
        assert abs(sc[k] - base[k]) <= 1e-12 * abs(base[k]), k
    hot = prim.copy()
    hot[4] = prim[4] + 0.3 * prim[0] / GAMMA  # T + 0.3 at the same rho
    ht = orc.dynamic_coefficients(P, orc.prim_to_cons(P, hot), M)
    for k in base:
        assert abs(ht[k] - base[k]) <= 1e-11 * max(abs(base[k]), 1e-300), k


def test_yoshizawa_isotropic_stress_in_the_residual(orc):
    """The isotropic SGS stress sigma_ll/3 enters the interface flux like a
    pressure: on a uniform Cartesian periodic grid the residual changes by
    A_d (s_{+1/2} - s_{-1/2}) in momentum d and by sum_d A_d ((s u_d)_{+1/2} -
    (s u_d)_{-1/2}) in energy, s = sigma/3 and u_d at the interface means,
    A_d = J^-1/h_d."""
    n, h = (10, 9, 8), (0.1, 0.15, 0.2)
    Lb = tuple(m * hh for m, hh in zip(n, h))
    xyz, shift = synth.box_grid(n, Lb)
    P = orc.params(periodic=(1, 1, 1), bc=0, sgs_model=3, k2=0.0, k4=0.0)
    M = orc.metrics(xyz, (1, 1, 1), shift)
    prim = synth.smooth_periodic_prim(xyz, Lb, amp=0.2, seed=1)
    Q = orc.prim_to_cons(P, prim)
    rng = np.random.default_rng(3)
    MK0 = np.concatenate([orc.mu_eff(orc.params(periodic=(1, 1, 1), bc=0), Q, M),
                          np.zeros((1,) + n)])
    MK1 = MK0.copy()
    MK1[2] = 0.05 * rng.random(n)
    dR = orc.rhs(P, Q, M, MK1) - orc.rhs(P, Q, M, MK0)
    s = MK1[2] / 3.0
    Jinv = h[0] * h[1] * h[2]
    vel = prim[1:4]
    expect = np.zeros((5,) + n)
    for d in range(3):
        A = Jinv / h[d]
        sp = 0.5 * (s + np.roll(s, -1, axis=d))  # interface (n, n + e_d)
        up = 0.5 * (vel[d] + np.roll(vel[d], -1, axis=d))
        expect[1 + d] += A * (sp - np.roll(sp, 1, axis=d))
        fe = sp * up
        expect[4] += A * (fe - np.roll(fe, 1, axis=d))
    assert np.abs(dR - expect).max() < 1e-15 * 50


def test_sutherland_law(orc):
    n = (5, 5, 5)
    xyz = _cartesian_box(n, 0.1)[0]
    P = orc.params(periodic=(1, 1, 1), bc=0, Re=1e5, sgs_model=0)
    xyz, shift = _cartesian_box(n, 0.1)
    M = orc.metrics(xyz, (1, 1, 1), shift)
    prim = synth.uniform_prim(n, rho=0.5)  # T = gamma p / rho = 2
    MK = orc.mu_eff(P, orc.prim_to_cons(P, prim), M)
    S = 110.4 / 288.15
    assert np.allclose(MK[0], 1.4e-5 * 2 ** 1.5 * (1 + S) / (2 + S), rtol=1e-14)


# --------------------------------------------------------------- locality

def test_stencil_locality(orc):
    """Perturbing one node changes the residual exactly on the stencil:
    +-1, +-2 along each axis, +-1 in two axes (cross derivatives), itself."""
    n = (9, 9, 9)
    xyz, shift = synth.box_grid(n, (1.0, 1.0, 1.0), wave=0.2)
    P = orc.params(periodic=(1, 1, 1), bc=0, Re=50.0, sgs_model=2)
    M = orc.metrics(xyz, (1, 1, 1), shift)
    Q = orc.prim_to_cons(P, synth.smooth_periodic_prim(xyz, amp=0.2, seed=1))
    MK = orc.mu_eff(P, Q, M)
    R0 = orc.rhs(P, Q, M, MK)
    Qp = Q.copy()
    Qp[1, 4, 4, 4] += 1e-3  # changes u, T (viscous) and W, p (inviscid)
    Qp[4, 4, 4, 4] += 1e-3
    R1 = orc.rhs(P, Qp, M, MK)  # viscosity frozen, as within the stages
    changed = set(map(tuple, np.argwhere(np.abs(R1 - R0).max(axis=0) > 0)))
    expect = set()
    for di in range(-2, 3):
        for dj in range(-2, 3):
            for dk in range(-2, 3):
                nz = [abs(x) for x in (di, dj, dk) if x != 0]
                if len(nz) <= 1 or (len(nz) == 2 and max(nz) == 1):
                    expect.add((4 + di, 4 + dj, 4 + dk))
    assert changed == expect


# ----------------------------------------------------------------- RK5

def test_rk5_amplification_polynomial(orc):
    """Eq. localdt with alpha = 1/4,1/6,3/8,1/2,1 on y' = z y gives
    G(z) = 1 + z + z^2/2 + 3 z^3/16 + z^4/32 + z^5/128 (second order)."""
    zs = np.array([-0.3, -1.7, 0.5, -2.5])
    y0 = np.ones((1, zs.size))

    def rhs_fn(q):
        return -zs[None, :] * q  # RHS = -dQ/dt

    y1 = orc.rk5(y0, rhs_fn, 1.0)[0]
    G = 1 + zs + zs ** 2 / 2 + 3 * zs ** 3 / 16 + zs ** 4 / 32 + zs ** 5 / 128
    assert np.allclose(y1, G, rtol=1e-15, atol=1e-15)
    # temporal order two: error of y' = -y ratio ~ 4 when dt halves
    errs = []
    for nstep in (10, 20, 40):
        y = np.ones((1, 1))
        for _ in range(nstep):
            y = orc.rk5(y, lambda q: q, 1.0 / nstep)
        errs.append(abs(y[0, 0] - math.exp(-1.0)))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_rk5_local_steps_per_node(orc):
    """Local steps (Eq. localdt with a node-dependent dt): decoupled
    y_n' = -lam_n y_n advanced with dt_n gives G(-lam_n dt_n) at every node,
    so each node sees its own step (a transposed or shared index fails)."""
    lam = np.array([0.3, 1.7, 0.5, 2.5, 0.9, 1.1])
    dtn = np.array([1.0, 0.4, 2.0, 0.7, 1.3, 0.25])
    y0 = np.ones((2, lam.size))

    def rhs_fn(q):
        return lam[None, :] * q

    y1 = orc.rk5(y0, rhs_fn, 123.0, dtn=dtn)
    z = -lam * dtn
    G = 1 + z + z ** 2 / 2 + 3 * z ** 3 / 16 + z ** 4 / 32 + z ** 5 / 128
    assert np.allclose(y1, G[None, :], rtol=1e-15, atol=1e-15)


def test_rk5_linear_stability_bound():
    """The paper states linear stability up to CFL 2 sqrt(2): |G(iy)| <= 1 on
    the imaginary axis for |y| <= 2 sqrt(2) (and up to ~4)."""
    y = np.linspace(0.0, 2.0 * math.sqrt(2.0), 400)
    z = 1j * y
    G = 1 + z + z ** 2 / 2 + 3 * z ** 3 / 16 + z ** 4 / 32 + z ** 5 / 128
    assert (np.abs(G) <= 1.0 + 1e-12).all()
    z = 1j * 4.2
    assert abs(1 + z + z ** 2 / 2 + 3 * z ** 3 / 16 + z ** 4 / 32 + z ** 5 / 128) > 1.0


def test_rk_step_boundary_nodes_and_masks(orc):
    """Stages never touch boundary nodes (bc = 0 keeps them frozen)."""
    P = orc.params(bc=0)
    xyz = synth.jet_grid(12, 10, 8)
    M = orc.metrics(xyz, (0, 0, 1))
    Q = orc.init_jet(P, xyz, 1)
    Q1, dt = orc.rk_step(P, Q, M, xyz, 0.0)
    for sl in [(slice(None), 0), (slice(None), -1), (slice(None), slice(None), 0),
               (slice(None), slice(None), -1)]:
        assert np.array_equal(Q1[sl], Q[sl])
    assert np.abs(Q1[:, 1:-1, 1:-1] - Q[:, 1:-1, 1:-1]).max() > 0


# --------------------------------------------------------------- time step

def test_time_step_closed_form(orc):
    """Uniform state on a Cartesian grid with spacings (hx, hy, hz):
    dt = CFL / sum_d (|u_d| + a)/h_d."""
    n = (6, 6, 6)
    hs = (0.1, 0.2, 0.05)
    xyz, shift = synth.box_grid(n, tuple(m * h for m, h in zip(n, hs)))
    P = orc.params(periodic=(1, 1, 1), bc=0, cfl=0.7)
    M = orc.metrics(xyz, (1, 1, 1), shift)
    vel = (0.3, -0.8, 0.1)
    Q = orc.prim_to_cons(P, synth.uniform_prim(n, u=vel[0], v=vel[1], w=vel[2]))
    expect = 0.7 / sum((abs(vel[d]) + 1.0) / hs[d] for d in range(3))
    assert abs(orc.dt(P, Q, M) - expect) < 1e-15 * expect * 10


def test_local_time_steps_closed_form(orc):
    """Local steps on a Cartesian grid with a non-uniform state:
    dt_n = CFL / sum_d (|u_d| + a)/h_d node by node; their minimum is the
    global CFL step, and a step in local mode advances the clock by it."""
    n = (6, 7, 5)
    hs = (0.1, 0.2, 0.05)
    xyz, shift = synth.box_grid(n, tuple(m * h for m, h in zip(n, hs)))
    P = orc.params(periodic=(1, 1, 1), bc=0, cfl=0.7, dt_mode=2)
    M = orc.metrics(xyz, (1, 1, 1), shift)
    prim = synth.smooth_periodic_prim(xyz, tuple(m * h for m, h in zip(n, hs)), amp=0.3, seed=5)
    Q = orc.prim_to_cons(P, prim)
    rho, u, v, w, p = prim
    a = np.sqrt(1.4 * p / rho)
    expect = 0.7 / ((np.abs(u) + a) / hs[0] + (np.abs(v) + a) / hs[1] + (np.abs(w) + a) / hs[2])
    got = orc.dt_local(P, Q, M)
    assert np.allclose(got, expect, rtol=1e-14, atol=0)
    assert orc.dt(P, Q, M) == got.min()
    _, dt = orc.rk_step(P, Q, M, xyz, 0.0)
    assert dt == got.min()


def test_local_steps_keep_the_free_stream_and_differ_from_global(orc):
    """A free stream is a fixed point of the local-step march as of the
    global one; on a non-uniform state the two marches differ (node-dependent
    steps), while a uniform-lambda state would make them agree."""
    xyz = synth.jet_grid(12, 10, 8)
    M = orc.metrics(xyz, (0, 0, 1))
    Pl = orc.params(dt_mode=2, bc=0)
    Pg = orc.params(dt_mode=0, bc=0)
    Qu = orc.prim_to_cons(Pl, synth.uniform_prim(xyz.shape[1:], u=0.6, v=0.1, w=-0.2))
    Q1, _ = orc.rk_step(Pl, Qu, M, xyz, 0.0)
    assert np.abs(Q1 - Qu).max() < 1e-13
    Q0 = orc.init_jet(Pl, xyz, seed=2, noise=1e-2)
    Ql, dtl = orc.rk_step(Pl, Q0, M, xyz, 0.0)
    Qg, dtg = orc.rk_step(Pg, Q0, M, xyz, 0.0)
    assert dtl == dtg
    assert np.abs(Ql - Qg).max() > 1e-6


# --------------------------------------------------------- boundaries

def _jet_setup(orc, n=(10, 12, 8), **kw):
    P = orc.params(**kw)
    xyz = synth.jet_grid(*n)
    M = orc.metrics(xyz, (0, 0, 1))
    return P, xyz, M


def _prim(Q):
    rho = Q[0]
    u, v, w = Q[1] / rho, Q[2] / rho, Q[3] / rho
    p = 0.4 * (Q[4] - 0.5 * rho * (u * u + v * v + w * w))
    return rho, u, v, w, p


def test_far_field_keeps_free_stream(orc):
    P, xyz, M = _jet_setup(orc)
    Q = orc.prim_to_cons(P, synth.uniform_prim(xyz.shape[1:]))
    Qb = orc.bc_jet(P, Q, M, xyz, 0.0)
    assert np.allclose(Qb[:, 1:-1, -1], Q[:, 1:-1, -1], rtol=0, atol=1e-14)


def test_far_field_riemann_invariants(orc):
    """Subsonic branches: the boundary state carries the interior R+ and the
    free-stream R-, and the entropy of its source state."""
    P, xyz, M = _jet_setup(orc)
    n = xyz.shape[1:]
    rng = np.random.default_rng(2)
    prim = synth.uniform_prim(n)
    prim[0] = 1.0 + 0.05 * rng.standard_normal(n)
    prim[1:4] = 0.3 * rng.standard_normal((3,) + n)
    prim[4] = (1 / GAMMA) * (1.0 + 0.05 * rng.standard_normal(n))
    Q = orc.prim_to_cons(P, prim)
    Qb = orc.bc_jet(P, Q, M, xyz, 0.0)
    rho, u, v, w, p = _prim(Q[:, 1:-1, -2])
    rf, uf, vf, wf, pf = _prim(Qb[:, 1:-1, -1])
    e = M[3:6, 1:-1, -1]
    nvec = e / np.sqrt((e ** 2).sum(axis=0))
    qe = u * nvec[0] + v * nvec[1] + w * nvec[2]
    ae = np.sqrt(GAMMA * p / rho)
    qf = uf * nvec[0] + vf * nvec[1] + wf * nvec[2]
    af = np.sqrt(GAMMA * pf / rf)
    sub = np.abs(qe / ae) < 1
    assert sub.sum() > 10
    assert np.allclose((qf + 5 * af)[sub], (qe + 5 * ae)[sub], atol=1e-12)
    assert np.allclose((qf - 5 * af)[sub], -5.0, atol=1e-12)
    out = sub & (qe >= 0)
    inn = sub & (qe < 0)
    assert out.sum() > 0 and inn.sum() > 0
    assert np.allclose((pf / rf ** GAMMA)[out], (p / rho ** GAMMA)[out], rtol=1e-12)
    assert np.allclose((pf / rf ** GAMMA)[inn], 1 / GAMMA, rtol=1e-12)
    # tangential velocity of the source state is kept
    tan = lambda a, b, c, q: np.stack([a - q * nvec[0], b - q * nvec[1], c - q * nvec[2]])
    assert np.allclose(tan(uf, vf, wf, qf)[:, out], tan(u, v, w, qe)[:, out], atol=1e-12)
    assert np.allclose(tan(uf, vf, wf, qf)[:, inn], 0.0, atol=1e-12)


def _free_stream_cons():
    # the far field's free stream at rest: rho = 1, u = v = w = 0, p = 1/gamma
    return np.array([1.0, 0.0, 0.0, 0.0, (1.0 / GAMMA) / (GAMMA - 1.0)])


def test_far_field_supersonic_branches(orc):
    """Supersonic branches of the far-field rule (Sec. "Far Field Boundary"):
    where the interior state leaves through the boundary faster than sound
    (q_n/a >= 1 along the outward normal grad(eta)/|grad(eta)|) the boundary
    node takes the adjacent interior node's conserved values unchanged; where
    it enters faster than sound (q_n/a <= -1) the free-stream state is
    imposed.  Interior nodes are given q_n = +-1.5 a plus a random tangential
    velocity, and a density and pressure of their own."""
    P, xyz, M = _jet_setup(orc)
    n = xyz.shape[1:]
    rng = np.random.default_rng(31)
    e = M[3:6, :, -1]
    nvec = e / np.sqrt((e ** 2).sum(axis=0))  # unit outward normal at (i, nj-1, k)
    rho = 1.0 + 0.2 * rng.random((n[0], n[2]))
    p = (1.0 / GAMMA) * (1.0 + 0.3 * rng.random((n[0], n[2])))
    a = np.sqrt(GAMMA * p / rho)
    sign = np.where(rng.random((n[0], n[2])) < 0.5, 1.5, -1.5)
    t = rng.standard_normal((3, n[0], n[2]))
    t -= (t * nvec).sum(axis=0) * nvec  # tangential part only
    vel = sign * a * nvec + 0.3 * t
    prim = synth.uniform_prim(n)
    prim[0, :, -2], prim[4, :, -2] = rho, p
    prim[1:4, :, -2] = vel
    Q = orc.prim_to_cons(P, prim)
    Qb = orc.bc_jet(P, Q, M, xyz, 0.0)
    _, u, v, w, _ = _prim(Q[:, :, -2])
    mach = (u * nvec[0] + v * nvec[1] + w * nvec[2]) / a
    inner = np.zeros((n[0], n[2]), bool)
    inner[1:-1] = True  # the far-field rule covers 0 < i < ni-1
    out = inner & (mach >= 1.0)
    inn = inner & (mach <= -1.0)
    assert out.sum() > 5 and inn.sum() > 5 and (out | inn).sum() == inner.sum()
    # supersonic exit: the interior node's conserved values, bit for bit
    assert np.array_equal(Qb[:, :, -1][:, out], Q[:, :, -2][:, out])
    # supersonic entrance: the free stream at rest
    fs = _free_stream_cons()
    got = Qb[:, :, -1][:, inn]
    assert np.allclose(got, fs[:, None], rtol=1e-15, atol=1e-15)


def test_characteristic_entrance_supersonic_branches(orc):
    """The same two branches at the entrance above the jet (bc = 2), whose
    outward normal is -x on the jet grid: u <= -a leaves the domain
    supersonically (the node (1, j, k) is copied), u >= a enters it (free
    stream).  The sonic edges are taken exactly with gamma = 2, rho = 1,
    p = 1/2 (a = 1 and the conserved round trip are exact in binary) at the
    nodes whose unit normal is exactly -1 in floating point: q_n/a = +1 is
    an exit (q_n/a >= 1 copies), q_n/a = -1 the supersonic entrance."""
    rng = np.random.default_rng(32)
    for exact in (False, True):
        gam = 2.0 if exact else GAMMA
        P, xyz, M = _jet_setup(orc, bc=2, gamma=gam)
        n = xyz.shape[1:]
        above = _entrance_split(xyz)
        assert np.abs(M[1:3, 0]).max() < 1e-14 and (M[0, 0] > 0).all()
        prim = synth.uniform_prim(n, p=1.0 / gam)
        if exact:
            ex = M[0, 0]
            above = above & (ex * (1.0 / np.sqrt(ex * ex)) == 1.0)
            ux = np.where(rng.random((n[1], n[2])) < 0.5, -1.0, 1.0)
        else:
            prim[0, 1] = 1.0 + 0.2 * rng.random((n[1], n[2]))
            prim[4, 1] = (1.0 / gam) * (1.0 + 0.3 * rng.random((n[1], n[2])))
            a = np.sqrt(gam * prim[4, 1] / prim[0, 1])
            ux = np.where(rng.random((n[1], n[2])) < 0.5, -1.5, 1.5) * a
            prim[2:4, 1] = 0.3 * rng.standard_normal((2, n[1], n[2]))
        prim[1, 1] = ux
        Q = orc.prim_to_cons(P, prim)
        Qb = orc.bc_jet(P, Q, M, xyz, 0.0)
        leave = above & (ux < 0)
        enter = above & (ux > 0)
        assert leave.sum() > 3 and enter.sum() > 3
        assert np.array_equal(Qb[:, 0][:, leave], Q[:, 1][:, leave])
        fs = np.array([1.0, 0.0, 0.0, 0.0, (1.0 / gam) / (gam - 1.0)])
        assert np.allclose(Qb[:, 0][:, enter], fs[:, None], rtol=1e-15, atol=1e-15)


def _entrance_split(xyz, r_jet=0.5):
    r = np.sqrt(xyz[1, 0] ** 2 + xyz[2, 0] ** 2)
    return r > r_jet


def test_characteristic_entrance_above_the_jet(orc):
    """bc = 2, entrance above the jet: the far-field rule with the outward
    normal -x (the jet grid's xi is the axial direction).  A quiescent
    interior stays quiescent; otherwise R+ comes from the node (1, j, k),
    R- from the free stream, and the entropy and tangential velocity from the
    source state of the branch (interior for outflow through the plane,
    free stream for inflow)."""
    P, xyz, M = _jet_setup(orc, bc=2)
    n = xyz.shape[1:]
    above = _entrance_split(xyz)
    assert above.sum() > 10 and (~above).sum() > 10
    Qr = orc.prim_to_cons(P, synth.uniform_prim(n))
    Qb = orc.bc_jet(P, Qr, M, xyz, 0.0)
    assert np.abs(Qb[:, 0][:, above] - Qr[:, 0][:, above]).max() < 1e-14
    rng = np.random.default_rng(6)
    prim = synth.uniform_prim(n)
    prim[0] = 1.0 + 0.05 * rng.standard_normal(n)
    prim[1] = 0.4 * rng.standard_normal(n)
    prim[2:4] = 0.2 * rng.standard_normal((2,) + n)
    prim[4] = (1 / GAMMA) * (1.0 + 0.05 * rng.standard_normal(n))
    Q = orc.prim_to_cons(P, prim)
    Qb = orc.bc_jet(P, Q, M, xyz, 0.0)
    rho, u, v, w, p = (a[above] for a in _prim(Q[:, 1]))
    rf, uf, vf, wf, pf = (a[above] for a in _prim(Qb[:, 0]))
    qe, qf = -u, -uf  # outward normal -x
    ae, af = np.sqrt(GAMMA * p / rho), np.sqrt(GAMMA * pf / rf)
    assert np.abs(M[1:3, 0]).max() < 1e-14  # the normal is exactly -x
    sub = np.abs(qe / ae) < 1
    out, inn = sub & (qe >= 0), sub & (qe < 0)
    assert out.sum() > 3 and inn.sum() > 3
    assert np.allclose((qf + 5 * af)[sub], (qe + 5 * ae)[sub], atol=1e-12)
    assert np.allclose((qf - 5 * af)[sub], -5.0, atol=1e-12)
    assert np.allclose((pf / rf ** GAMMA)[out], (p / rho ** GAMMA)[out], rtol=1e-12)
    assert np.allclose((pf / rf ** GAMMA)[inn], 1 / GAMMA, rtol=1e-12)
    assert np.allclose(vf[out], v[out], atol=1e-13) and np.allclose(wf[out], w[out], atol=1e-13)
    assert np.abs(vf[inn]).max() < 1e-13 and np.abs(wf[inn]).max() < 1e-13
    # the jet area of a supersonic jet keeps the Dirichlet jet state (bc = 1)
    P1, _, _ = _jet_setup(orc, bc=1)
    Q1 = orc.bc_jet(P1, Q, M, xyz, 0.0)
    assert np.array_equal(Qb[:, 0][:, ~above], Q1[:, 0][:, ~above])
    # the rest of the boundary is the same as with bc = 1
    assert np.array_equal(Qb[:, 1:], Q1[:, 1:])


def test_subsonic_jet_characteristic_entrance(orc):
    """bc = 2 with a subsonic jet (Mj = 0.9): in the jet area u is the target
    profile, v and w come from the node (1, j, k), and T, p follow the jet's
    total temperature and the isentropic relation; at the target's own
    design point (u = Mj, v = w = 0) that is exactly T = 1, p = 1/gamma."""
    P, xyz, M = _jet_setup(orc, bc=2, Mj=0.9)
    n = xyz.shape[1:]
    jet = ~_entrance_split(xyz)
    rng = np.random.default_rng(9)
    prim = synth.uniform_prim(n)
    prim[2:4] = 0.1 * rng.standard_normal((2,) + n)
    Q = orc.prim_to_cons(P, prim)
    Qb = orc.bc_jet(P, Q, M, xyz, 0.0)
    rf, uf, vf, wf, pf = (a[jet] for a in _prim(Qb[:, 0]))
    r = np.sqrt(xyz[1, 0] ** 2 + xyz[2, 0] ** 2)[jet]
    ut = 0.45 * (1.0 + np.tanh((0.5 - r) / 0.1))
    assert np.allclose(uf, ut, rtol=1e-14, atol=1e-15)
    assert np.allclose(vf, prim[2, 1][jet], atol=1e-15)
    assert np.allclose(wf, prim[3, 1][jet], atol=1e-15)
    Tt = 1.0 + 0.2 * 0.81
    T = Tt / (1.0 + 0.2 * (ut ** 2 + vf ** 2 + wf ** 2))
    assert np.allclose(GAMMA * pf / rf, T, rtol=1e-13)
    assert np.allclose(pf, T ** 3.5 / GAMMA, rtol=1e-13)
    prim0 = synth.uniform_prim(n, u=0.9)
    P0, _, _ = _jet_setup(orc, bc=2, Mj=0.9, theta_m=1e-6)
    Qb0 = orc.bc_jet(P0, orc.prim_to_cons(P0, prim0), M, xyz, 0.0)
    rf0, uf0, _, _, pf0 = (a[jet] for a in _prim(Qb0[:, 0]))
    assert np.allclose(uf0, 0.9, rtol=1e-15) and np.allclose(pf0, 1 / GAMMA, rtol=1e-14)
    assert np.allclose(rf0, 1.0, rtol=1e-14)


def test_exit_and_inner_ring(orc):
    P, xyz, M = _jet_setup(orc)
    n = xyz.shape[1:]
    prim = synth.uniform_prim(n)
    rng = np.random.default_rng(8)
    prim[0] = 1.0 + 0.1 * rng.random(n)
    prim[1] = np.where(np.arange(n[1])[None, :, None] < 5, 2.0, 0.3) + 0 * prim[1]
    prim[4] = (1 / GAMMA) * (1.0 + 0.1 * rng.random(n))
    Q = orc.prim_to_cons(P, prim)
    Qb = orc.bc_jet(P, Q, M, xyz, 0.0)
    # inner ring = azimuthal mean of the first interior ring
    assert np.allclose(Qb[:, 1:-1, 0, :], Q[:, 1:-1, 1, :].mean(axis=-1, keepdims=True), atol=1e-15)
    # exit: supersonic rows copy, subsonic rows keep T and u with p = p_inf
    rho, u, v, w, p = _prim(Qb[:, -2])
    rf, uf, vf, wf, pf = _prim(Qb[:, -1])
    sup = (u / np.sqrt(GAMMA * p / rho)) >= 1.0
    assert sup.any() and (~sup).any()
    assert np.allclose(Qb[:, -1][:, sup], Qb[:, -2][:, sup], rtol=0, atol=0)
    assert np.allclose(pf[~sup], 1 / GAMMA, rtol=1e-13)
    assert np.allclose((pf / rf)[~sup], (p / rho)[~sup], rtol=1e-13)
    assert np.allclose(uf[~sup], u[~sup], rtol=1e-13)


def test_inflow_forcing(orc):
    """Entrance plane: profile plus the 16-mode forcing at time t."""
    amp = synth.forcing_amplitudes(3)
    P, xyz, M = _jet_setup(orc, amp=tuple(amp))
    Q = orc.prim_to_cons(P, synth.uniform_prim(xyz.shape[1:]))
    t = 0.37
    Qb = orc.bc_jet(P, Q, M, xyz, t)
    y, z = xyz[1, 0], xyz[2, 0]
    r, th = np.sqrt(y * y + z * z), np.arctan2(z, y)
    u = 0.7 * (1 + np.tanh((0.5 - r) / 0.1))
    g = np.exp(-((r - 0.5) / 0.05) ** 2)
    St = (0.25, 0.5, 0.75, 1.0)
    for m in range(4):
        for f in range(4):
            u = u + amp[m * 4 + f] * g * np.cos(m * th - 2 * np.pi * St[f] * 1.4 * t)
    assert np.allclose(Qb[1, 0], u, rtol=1e-14, atol=1e-15)
    assert np.allclose(Qb[0, 0], 1.0) and np.abs(Qb[2:4, 0]).max() == 0


def test_azimuthal_rotation_equivariance(orc):
    """Rotating the initial state by one azimuthal index rotates the result of
    a full step (periodic wrap, BCs and reductions are index-shift
    invariant on the rotationally symmetric grid)."""
    P, xyz, M = _jet_setup(orc, n=(10, 12, 8), sgs_model=2)
    Q = orc.init_jet(P, xyz, 11)
    Q1, dt1 = orc.rk_step(P, Q, M, xyz, 0.0)
    c, s = math.cos(2 * math.pi / 8), math.sin(2 * math.pi / 8)

    def rotate(A):  # shift one azimuthal index and turn (v, w) with it
        B = np.roll(A, 1, axis=3)
        v, w = B[2].copy(), B[3].copy()
        B[2], B[3] = c * v - s * w, s * v + c * w
        return B

    Q2, dt2 = orc.rk_step(P, rotate(Q), M, xyz, 0.0)
    assert abs(dt1 - dt2) < 1e-12 * dt1
    assert np.allclose(rotate(Q1), Q2, rtol=0, atol=1e-12)


# ------------------------------------------- true centerline grid (A27)

def _cylinder(ni, nj, nk, R=0.5, L=1.0):
    """Uniform cylinder x in [0, L], r in [0, R] (r_0 = 0: the axis),
    theta_k = 2 pi k / nk."""
    x = np.linspace(0.0, L, ni)
    r = np.linspace(0.0, R, nj)
    th = 2.0 * math.pi * np.arange(nk) / nk
    xyz = np.empty((3, ni, nj, nk))
    xyz[0] = x[:, None, None]
    xyz[1] = r[None, :, None] * np.cos(th)[None, None, :]
    xyz[2] = r[None, :, None] * np.sin(th)[None, None, :]
    return xyz


def test_axis_grid_metrics(orc):
    """On a true centerline grid (r_0 = 0) the zeta tangent vanishes on the
    axis, so J^-1 = 0 there exactly and the axis nodes keep the J^-1-scaled
    metrics: the xi and eta rows are 0 and the zeta row is x_xi x x_eta =
    x_xi r_eta (0, -sin theta, cos theta), with r_eta the one-sided
    second-order difference at j = 0.  Every other node satisfies the metric
    identity and J^-1 = det, as on the annular grid."""
    ni, nj, nk = 12, 10, 16
    xyz = synth.jet_grid(ni, nj, nk, r0=0.0)
    x, r, th = synth.jet_lines(ni, nj, nk, r0=0.0)
    assert r[0] == 0.0
    for form in (0, 1):
        M = orc.metrics(xyz, form=form)
        assert np.isfinite(M).all()
        assert (M[9][:, 0] == 0.0).all() and (M[9][:, 1:] > 0.0).all()
    M = orc.metrics(xyz)
    assert (M[0:7][:, :, 0] == 0.0).all()
    xd = np.gradient(x, edge_order=2)[:, None]
    rd0 = np.gradient(r, edge_order=2)[0]
    assert np.allclose(M[7][:, 0], -xd * rd0 * np.sin(th)[None, :], rtol=1e-13, atol=1e-15)
    assert np.allclose(M[8][:, 0], xd * rd0 * np.cos(th)[None, :], rtol=1e-13, atol=1e-15)
    X = _coord_jacobian(xyz, (0, 0, 1), np.zeros(9))
    Mm = M[:9].reshape((3, 3) + xyz.shape[1:])
    ident = np.einsum("dc...,ce...->de...", Mm, X)[:, :, :, 1:]
    assert np.abs(ident - np.eye(3)[:, :, None, None, None]).max() < 1e-12
    det = np.linalg.det(np.moveaxis(X, (0, 1), (-2, -1)))
    assert np.allclose(det[:, 1:], M[9][:, 1:], rtol=1e-13, atol=0)


@pytest.mark.parametrize("sgs", [0, 1, 2])
@pytest.mark.parametrize("form", [0, 1])
def test_axis_free_stream_preservation(orc, sgs, form):
    """A uniform state on the centerline grid gives a zero residual at every
    interior node, ring 1 included: the axis nodes' J^-1-scaled metrics and
    the radii they take from ring 1 keep the central flux, the dissipation
    (no NaN from the axis) and the weighted interface metrics exact."""
    ni, nj, nk = 12, 10, 16
    xyz = synth.jet_grid(ni, nj, nk, r0=0.0)
    M = orc.metrics(xyz, form=form)
    P = orc.params(sgs_model=sgs, Re=400.0, axis=1)
    prim = np.empty((5,) + xyz.shape[1:])
    prim[0], prim[1], prim[2], prim[3], prim[4] = 1.0, 0.3, 0.1, -0.2, 1.0 / GAMMA
    Q = orc.prim_to_cons(P, prim)
    R = orc.rhs(P, Q, M)
    scale = np.abs(M[9]).max() * 1.5
    assert np.isfinite(R).all()
    assert np.abs(R).max() < 1e-13 * scale


def test_axis_residual_converges(orc):
    """J * RHS on uniform cylinders with an axis against the exact flux
    divergence of the manufactured solution (viscous, Re = 20, no
    dissipation, whose fourth difference meets the paper's boundary closure
    at the faces): second order from ring 3 outward and convergent at ring 1.
    The paper's plain mean of the two nodes' metrics makes ring 1 diverge
    (|grad zeta| ~ 1/r changes by O(1) between rings 1 and 2); the weighted
    mean of Reading A27 and the axis rules restore convergence."""
    f_prim, f_res, _ = _mms_exact_divergence(20.0)
    P = orc.params(periodic=(0, 0, 1), bc=0, Re=20.0, sgs_model=0, k2=0.0, k4=0.0, axis=1)
    far, ring1 = [], []
    for n in (8, 16, 32):
        xyz = _cylinder(n, n, 2 * n)
        M = orc.metrics(xyz, (0, 0, 1))
        prim = np.array([np.broadcast_to(f, xyz.shape[1:]) for f in f_prim(*xyz)])
        Q = orc.prim_to_cons(P, prim)
        R = orc.rhs(P, Q, M)
        inner = (slice(None), slice(1, -1), slice(1, -1), slice(None))
        JR = R[inner] / M[9][1:-1, 1:-1][None]
        exact = np.array([np.broadcast_to(f, xyz.shape[1:]) for f in f_res(*xyz)])[inner]
        err = np.abs(JR - exact)
        ring1.append(err[:, :, 0].max())
        far.append(err[:, :, 2:].max())
    assert far[0] / far[1] > 3.0 and far[1] / far[2] > 3.3, far
    assert ring1[0] / ring1[1] > 2.0 and ring1[1] / ring1[2] > 2.0, ring1


def test_axis_viscosity_is_the_ring_mean(orc):
    """The SGS viscosity of an axis node is the azimuthal mean of ring 1's at
    its plane (the centerline rule), its laminar part its own (Sutherland at
    its temperature); kappa follows with Pr and Pr_sgs."""
    ni, nj, nk = 12, 10, 16
    xyz = synth.jet_grid(ni, nj, nk, r0=0.0)
    M = orc.metrics(xyz)
    for sgs in (1, 2):
        P = orc.params(sgs_model=sgs, Re=400.0, axis=1)
        Q = orc.init_jet(P, xyz, seed=5, noise=3e-2)
        P0 = orc.params(sgs_model=0, Re=400.0, axis=1)
        MK, MK0 = orc.mu_eff(P, Q, M), orc.mu_eff(P0, Q, M)
        mu_sgs = MK[0] - MK0[0]
        assert np.abs(mu_sgs[:, 1]).max() > 0.0
        ring_mean = mu_sgs[:, 1].mean(axis=1)
        assert np.allclose(mu_sgs[:, 0], ring_mean[:, None], rtol=1e-12, atol=1e-18)
        kap_sgs = MK[1] - MK0[1]
        assert np.allclose(kap_sgs[:, 0], ring_mean[:, None] / (0.4 * 0.9), rtol=1e-12, atol=1e-18)


def test_axis_supersonic_exit(orc):
    """A uniform supersonic axial stream leaves through the exit: every exit
    node copies its upstream neighbour (as the other boundary rules left it),
    the axis nodes too (their xi row is 0, so they take ring 1's outward
    normal)."""
    ni, nj, nk = 12, 10, 16
    xyz = synth.jet_grid(ni, nj, nk, r0=0.0)
    M = orc.metrics(xyz)
    P = orc.params(axis=1)
    prim = np.empty((5,) + xyz.shape[1:])
    # p above the free stream's: the subsonic exit rule would change the state
    prim[0], prim[1], prim[2], prim[3], prim[4] = 1.0, 1.6, 0.0, 0.0, 1.3 / GAMMA
    Q = orc.prim_to_cons(P, prim)
    Qb = orc.bc_jet(P, Q, M, xyz, 0.0)
    assert np.array_equal(Qb[:, -1], Qb[:, -2])


# ------------------------------------------------- adjoint window functional

def test_surface_functional_ring_area_closed_form(orc):
    """The window functional's term for a state whose pressure exceeds 1/gamma
    by c on the ring j is w c^2 times the ring's eta-face area.  On the
    cylindrical jet grid J^-1 |grad eta| = |x_zeta x x_xi| = x_xi r_j
    sin(2 pi / nk) exactly (x depends on i only, y and z on j and k only), so
    the area is nk r_j sin(2 pi / nk) sum_i x_xi(i), with x_xi the metrics'
    second-order differences (numpy's gradient with second-order edges).  The
    pressure is the System I one: random density and velocity at p = 1/gamma
    give 0.  The xi or zeta rows in place of the eta row, a missing J^-1, or
    the kinetic energy left in p all fail here."""
    P = orc.params()
    ni, nj, nk = 20, 12, 16
    xyz = synth.jet_grid(ni, nj, nk)
    M = orc.metrics(xyz)
    x, r, _ = synth.jet_lines(ni, nj, nk)
    rng = np.random.default_rng(11)
    prim = np.empty((5, ni, nj, nk))
    prim[0] = 0.8 + 0.4 * rng.random((ni, nj, nk))
    prim[1:4] = 0.5 * rng.standard_normal((3, ni, nj, nk))
    for j in (0, 5, nj - 1):
        ring = nk * r[j] * math.sin(2.0 * math.pi / nk) * np.gradient(x, edge_order=2).sum()
        for c in (0.0, 0.03, -0.05):
            prim[4] = 1.0 / GAMMA + c
            Q = orc.prim_to_cons(P, prim)
            for w in (1.0, 2.5e-4):
                J = orc.surface_functional(P, Q, M, j, w)
                assert J == pytest.approx(w * c * c * ring, rel=1e-12, abs=1e-28)
    # only the ring j enters
    prim[4] = 1.0 / GAMMA
    prim[4][:, 4] += 0.1
    Q = orc.prim_to_cons(P, prim)
    assert orc.surface_functional(P, Q, M, 5, 1.0) < 1e-28
    assert orc.surface_functional(P, Q, M, 4, 1.0) > 0.0
    with pytest.raises(ValueError):
        orc.surface_functional(P, Q, M, nj, 1.0)


def test_oracle_results_do_not_depend_on_the_thread_count(orc):
    """The OpenMP loops only split independent per-node work: one thread and
    all threads give the same bits (one step with SGS and jet BCs, and the
    dynamic procedure)."""
    xyz = synth.jet_grid(16, 12, 8)
    M = orc.metrics(xyz, (0, 0, 1))
    outs = []
    full = orc.num_threads()
    for nt in (1, full):
        orc.set_num_threads(nt)
        try:
            P = orc.params(sgs_model=1)
            Q0 = orc.init_jet(P, xyz, seed=7, noise=1e-2)
            Q1, dt = orc.rk_step(P, Q0, M, xyz, 0.0)
            P3 = orc.params(sgs_model=3)
            dyn = orc.dynamic_coefficients(P3, Q0, M)
            outs.append((Q1, dt, dyn))
        finally:
            orc.set_num_threads(full)
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
    assert outs[0][2] == outs[1][2]
