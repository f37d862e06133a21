"""Differentiable FP64 restatement of one time step of the scheme and of the
far-field functional, in plain PyTorch tensor operations on the CPU.

TEST INFRASTRUCTURE, under the same rules as the rest of this package: only
the test-suite may import it.  It is a third implementation, independent of
both the C oracle and the CUDA library, written for one purpose: to give
torch.autograd gradients against which the hand-written discrete adjoint is
checked on small grids.  It covers the configuration that adjoint supports:
jet boundary conditions on the annular grid (periodic in zeta only), no SGS
model, viscosity frozen at Q^n over the five stages, fixed time step.

Where the C oracle loops over nodes and interfaces, this module shifts whole
arrays.  The readings of the paper are the same:
- primitives from System I energy; radii lambda_d = |U_d| + a |grad d| and
  the anisotropic lbar of Sec. "Spatial Discretization";
- pressure sensor nu = |d2p| / (p+ + 2p + p-), a face node taking its inward
  neighbour's value; d = lambda [eps2 dW - eps4 d3W] with eps2 = k2 max(nu),
  eps4 = max(0, k4 - eps2), W = Q + (0,0,0,0,p), J^-1 applied once at the
  interface, and a missing outside difference replaced by minus the first
  inside one (Eqs. dissip_term, eps_2/4_dissip, W_dissip);
- compact interface gradients: normal difference of the two nodes, tangential
  mean of their central differences, Cartesian gradients through the mean
  metrics; Sutherland viscosity times M_j/Re, Fourier heat flux
  (Eqs. hat-flux-Ev/Fv/Gv, tau_mod, q_mod);
- five stages Q^(l) = Q^(0) - alpha_l dt J RHS(Q^(l-1)) on interior nodes
  (Eq. localdt), then the boundary conditions of Sec. "Boundary Conditions"
  (forced Dirichlet entrance, Riemann far field, inner-ring mean, exit from
  the updated column ni-2).
At non-differentiable points the derivative follows the branch the forward
value takes: |x| is written x < 0 ? -x : x (slope +1 at 0) and max(a, b) as
a > b ? a : b.

With axis=True it restates, for the forward residual and step only, the
rules of a true centerline grid (ring j = 0 on the axis, J^-1 = 0 there, its
metrics J^-1-scaled): the axis nodes take ring 1's radii, every interface
metric is the J^-1-weighted mean of the two nodes', and an exit node on the
axis takes ring 1's outward normal.
"""
from __future__ import annotations

import math

import torch

ALPHA = (1.0 / 4.0, 1.0 / 6.0, 3.0 / 8.0, 1.0 / 2.0, 1.0)


def _abs(x):
    return torch.where(x < 0, -x, x)


def _sl(d, start, stop):
    """Index tuple taking [start:stop] along direction d of a (ni, nj, nk) field."""
    idx = [slice(None)] * 3
    idx[d] = slice(start, stop)
    return tuple(idx)


class Case:
    """Grid data of one run: metrics M [10][ni][nj][nk] (constants), the
    entrance-plane radius and angle, and the scalar parameters."""

    def __init__(self, M, xyz, *, gamma=1.4, Pr=0.72, Mj=1.4, Re=1.0e5, T_ref=288.15,
                 k2=0.25, k4=0.016, r_jet=0.5, theta_m=0.05, force_width=0.05,
                 St=(0.25, 0.5, 0.75, 1.0), axis=False):
        self.M = torch.as_tensor(M, dtype=torch.float64)
        xyz = torch.as_tensor(xyz, dtype=torch.float64)
        self.shape = tuple(self.M.shape[1:])
        y0, z0 = xyz[1, 0], xyz[2, 0]
        self.r0 = torch.sqrt(y0 * y0 + z0 * z0)
        self.th0 = torch.atan2(z0, y0)
        self.gamma, self.Pr, self.Mj, self.Re, self.T_ref = gamma, Pr, Mj, Re, T_ref
        self.k2, self.k4 = k2, k4
        self.r_jet, self.theta_m, self.force_width, self.St = r_jet, theta_m, force_width, St
        self.per = (False, False, True)
        self.axis = axis
        ni, nj, nk = self.shape
        inter = torch.zeros(self.shape, dtype=torch.bool)
        inter[1:ni - 1, 1:nj - 1, :] = True
        self.interior = inter

    # ---------------------------------------------------------- node data
    def primitives(self, Q):
        g = self.gamma
        rho = Q[0]
        u, v, w = Q[1] / rho, Q[2] / rho, Q[3] / rho
        p = (g - 1.0) * (Q[4] - 0.5 * rho * (u * u + v * v + w * w))
        T = g * p / rho
        a = torch.sqrt(g * p / rho)
        return rho, u, v, w, p, T, a

    def viscosity(self, Q):
        """mu_eff, kappa_eff of Q (laminar Sutherland only: no SGS model)."""
        *_, T, _ = self.primitives(Q)
        if self.Re <= 0.0:
            z = torch.zeros_like(T)
            return z, z
        S = 110.4 / self.T_ref
        mu = (self.Mj / self.Re) * T ** 1.5 * (1.0 + S) / (T + S)
        return mu, mu / ((self.gamma - 1.0) * self.Pr)

    def _shift(self, f, d, s):
        """f at the node s steps along d (periodic d only)."""
        return torch.roll(f, -s, dims=d)

    def _sensor(self, p, d):
        if self.per[d]:
            pp, pm = self._shift(p, d, 1), self._shift(p, d, -1)
            return _abs(pp - 2.0 * p + pm) / (pp + 2.0 * p + pm)
        n = p.shape[d]
        pp, pc, pm = p[_sl(d, 2, n)], p[_sl(d, 1, n - 1)], p[_sl(d, 0, n - 2)]
        inner = _abs(pp - 2.0 * pc + pm) / (pp + 2.0 * pc + pm)
        return torch.cat([inner[_sl(d, 0, 1)], inner, inner[_sl(d, n - 3, n - 2)]], dim=d)

    def _central(self, f, t):
        """phi(+t) - phi(-t) at nodes with both neighbours, 0 on the faces of
        a non-periodic direction (those values reach only interfaces whose
        residual is not used)."""
        if self.per[t]:
            return self._shift(f, t, 1) - self._shift(f, t, -1)
        n = f.shape[t]
        inner = f[_sl(t, 2, n)] - f[_sl(t, 0, n - 2)]
        z = torch.zeros_like(f[_sl(t, 0, 1)])
        return torch.cat([z, inner, z], dim=t)

    # ---------------------------------------------------------- interfaces
    def _pair(self, f, d):
        """(f_a, f_b) over the interfaces (a, a + e_d) along d."""
        if self.per[d]:
            return f, self._shift(f, d, 1)
        n = f.shape[d]
        return f[_sl(d, 0, n - 1)], f[_sl(d, 1, n)]

    def _flux(self, Q, MK, prim, lbar, nu, d):
        """Interface fluxes F = F_inviscid - J^-1 d - F_viscous along d."""
        rho, u, v, w, p, T, a = prim
        M = self.M
        P = lambda f: self._pair(f, d)
        Jinv = M[9]
        m = [M[3 * d + c] for c in range(3)]
        Th = m[0] * u + m[1] * v + m[2] * w
        Fn = [Jinv * (Q[0] * Th), Jinv * (Q[1] * Th + p * m[0]), Jinv * (Q[2] * Th + p * m[1]),
              Jinv * (Q[3] * Th + p * m[2]), Jinv * ((Q[4] + p) * Th)]
        W = [Q[0], Q[1], Q[2], Q[3], Q[4] + p]
        nua, nub = P(nu[d])
        eps2 = self.k2 * torch.where(nua > nub, nua, nub)
        e4 = self.k4 - eps2
        eps4 = torch.where(e4 < 0, torch.zeros_like(e4), e4)
        la, lb = P(lbar[d])
        lam = 0.5 * (la + lb)
        Ja, Jb = P(Jinv)
        Jh = 0.5 * (Ja + Jb)
        F = []
        for q in range(5):
            Fa, Fb = P(Fn[q])
            if self.per[d]:
                D1 = self._shift(W[q], d, 1) - W[q]
                Dm = self._shift(D1, d, -1)
                Dp = self._shift(D1, d, 1)
            else:
                n = W[q].shape[d]
                D1 = W[q][_sl(d, 1, n)] - W[q][_sl(d, 0, n - 1)]
                Dm = torch.cat([-D1[_sl(d, 0, 1)], D1[_sl(d, 0, n - 2)]], dim=d)
                Dp = torch.cat([D1[_sl(d, 1, n - 1)], -D1[_sl(d, n - 2, n - 1)]], dim=d)
            D3 = Dp - 2.0 * D1 + Dm
            F.append(0.5 * (Fa + Fb) - Jh * (lam * (eps2 * D1 - eps4 * D3)))
        # viscous flux from compact interface gradients
        phis = [u, v, w, T]
        dphi = [[None] * 3 for _ in range(4)]
        for q, f in enumerate(phis):
            fa, fb = P(f)
            for t in range(3):
                if t == d:
                    dphi[q][t] = fb - fa
                else:
                    ca, cb = P(self._central(f, t))
                    dphi[q][t] = 0.25 * (ca + cb)
        mh = [[None] * 3 for _ in range(3)]
        for t in range(3):
            for c in range(3):
                ma, mb = P(M[3 * t + c])
                if self.axis:
                    # J^-1-weighted mean; axis nodes hold scaled metrics
                    sa = torch.where(Ja == 0, ma, Ja * ma)
                    sb = torch.where(Jb == 0, mb, Jb * mb)
                    mh[t][c] = (sa + sb) / (Ja + Jb)
                else:
                    mh[t][c] = 0.5 * (ma + mb)
        gr = [[mh[0][c] * dphi[q][0] + mh[1][c] * dphi[q][1] + mh[2][c] * dphi[q][2]
               for c in range(3)] for q in range(4)]
        mua, mub = P(MK[0])
        ka, kb = P(MK[1])
        mu, kap = 0.5 * (mua + mub), 0.5 * (ka + kb)
        div = gr[0][0] + gr[1][1] + gr[2][2]
        txx = mu * (2.0 * gr[0][0] - (2.0 / 3.0) * div)
        tyy = mu * (2.0 * gr[1][1] - (2.0 / 3.0) * div)
        tzz = mu * (2.0 * gr[2][2] - (2.0 / 3.0) * div)
        txy = mu * (gr[0][1] + gr[1][0])
        txz = mu * (gr[0][2] + gr[2][0])
        tyz = mu * (gr[1][2] + gr[2][1])
        ua, ub = P(u)
        va, vb = P(v)
        wa, wb = P(w)
        uf, vf, wf = 0.5 * (ua + ub), 0.5 * (va + vb), 0.5 * (wa + wb)
        bx = txx * uf + txy * vf + txz * wf + kap * gr[3][0]
        by = txy * uf + tyy * vf + tyz * wf + kap * gr[3][1]
        bz = txz * uf + tyz * vf + tzz * wf + kap * gr[3][2]
        mx, my, mz = mh[d]
        F[1] = F[1] - Jh * (mx * txx + my * txy + mz * txz)
        F[2] = F[2] - Jh * (mx * txy + my * tyy + mz * tyz)
        F[3] = F[3] - Jh * (mx * txz + my * tyz + mz * tzz)
        F[4] = F[4] - Jh * (mx * bx + my * by + mz * bz)
        return F

    def rhs(self, Q, MK):
        """Residual sum_d (F_{+1/2} - F_{-1/2}) on interior nodes, 0 elsewhere."""
        prim = self.primitives(Q)
        rho, u, v, w, p, T, a = prim
        M = self.M
        lam = []
        for d in range(3):
            mx, my, mz = M[3 * d], M[3 * d + 1], M[3 * d + 2]
            lam.append(_abs(mx * u + my * v + mz * w) + a * torch.sqrt(mx * mx + my * my + mz * mz))
        lbar = [lam[0] * (1.0 + torch.sqrt(lam[1] / lam[0]) + torch.sqrt(lam[2] / lam[0])),
                lam[1] * (1.0 + torch.sqrt(lam[0] / lam[1]) + torch.sqrt(lam[2] / lam[1])),
                lam[2] * (1.0 + torch.sqrt(lam[0] / lam[2]) + torch.sqrt(lam[1] / lam[2]))]
        if self.axis:  # the axis nodes take ring 1's radii
            lbar = [torch.cat([lb[:, 1:2], lb[:, 1:]], dim=1) for lb in lbar]
        nu = [self._sensor(p, d) for d in range(3)]
        R = [torch.zeros_like(rho) for _ in range(5)]
        for d in range(3):
            F = self._flux(Q, MK, prim, lbar, nu, d)
            for q in range(5):
                if self.per[d]:
                    R[q] = R[q] + (F[q] - self._shift(F[q], d, -1))
                else:
                    n = rho.shape[d]
                    inner = F[q][_sl(d, 1, n - 1)] - F[q][_sl(d, 0, n - 2)]
                    z = torch.zeros_like(rho[_sl(d, 0, 1)])
                    R[q] = R[q] + torch.cat([z, inner, z], dim=d)
        zero = torch.zeros_like(rho)
        return torch.stack([torch.where(self.interior, r, zero) for r in R])

    # ------------------------------------------------------------ boundary
    def _cons(self, rho, u, v, w, p):
        return torch.stack([rho, rho * u, rho * v, rho * w,
                            p / (self.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)])

    def boundary(self, Qs, amps, t):
        g, gm1 = self.gamma, self.gamma - 1.0
        p_inf = 1.0 / g
        ni, nj, nk = self.shape
        M = self.M
        Q1 = Qs.clone()
        # entrance i = 0: forced jet profile
        r, th = self.r0, self.th0
        u = 0.5 * self.Mj * (1.0 + torch.tanh((self.r_jet - r) / (2.0 * self.theta_m)))
        gr = torch.exp(-((r - self.r_jet) / self.force_width) ** 2)
        for mm in range(4):
            for f in range(4):
                u = u + amps[mm * 4 + f] * gr * torch.cos(
                    mm * th - 2.0 * math.pi * self.St[f] * self.Mj * t)
        one = torch.ones_like(u)
        zero = torch.zeros_like(u)
        Q1[:, 0] = self._cons(one, u, zero, zero, p_inf * one)
        # far field j = nj-1, 0 < i < ni-1, from the column j = nj-2
        e = M[3:6, 1:ni - 1, nj - 1]
        nrm = e / torch.sqrt((e * e).sum(0))
        rho, u, v, w, p, T, a_e = self.primitives(Qs[:, 1:ni - 1, nj - 2])
        qne = u * nrm[0] + v * nrm[1] + w * nrm[2]
        Rp = qne + 2.0 * a_e / gm1
        Rm = 0.0 - 2.0 * 1.0 / gm1
        qnf = 0.5 * (Rp + Rm)
        af = 0.25 * gm1 * (Rp - Rm)
        Mn = qne / a_e
        rfB = (rho ** g * af * af / (g * p)) ** (1.0 / gm1)
        QB = self._cons(rfB, u + (qnf - qne) * nrm[0], v + (qnf - qne) * nrm[1],
                        w + (qnf - qne) * nrm[2], rfB * af * af / g)
        rfC = (af * af / (g * p_inf)) ** (1.0 / gm1)
        QC = self._cons(rfC, qnf * nrm[0], qnf * nrm[1], qnf * nrm[2], rfC * af * af / g)
        ones = torch.ones_like(qne)
        QD = self._cons(ones, 0.0 * ones, 0.0 * ones, 0.0 * ones, p_inf * ones)
        QA = Qs[:, 1:ni - 1, nj - 2]
        Qf = torch.where(Mn >= 1.0, QA, torch.where(Mn >= 0.0, QB, torch.where(Mn > -1.0, QC, QD)))
        Q1[:, 1:ni - 1, nj - 1] = Qf
        # inner ring j = 0: azimuthal mean of ring j = 1
        mean = Qs[:, 1:ni - 1, 1].sum(dim=-1, keepdim=True) / nk
        Q1[:, 1:ni - 1, 0] = mean.expand(-1, -1, nk)
        # exit i = ni-1 from the updated column ni-2
        e = M[0:3, ni - 1]
        if self.axis:  # an exit node on the axis takes ring 1's normal
            e = torch.cat([e[:, 1:2], e[:, 1:]], dim=1)
        inv = 1.0 / torch.sqrt((e * e).sum(0))
        Qe = Q1[:, ni - 2]
        rho, u, v, w, p, T, a_e = self.primitives(Qe)
        qn = (u * e[0] + v * e[1] + w * e[2]) * inv
        e_int = p / (gm1 * rho)
        rf = p_inf / (gm1 * e_int)
        Qsub = torch.stack([rf, rf * u, rf * v, rf * w, rf * (e_int + 0.5 * (u * u + v * v + w * w))])
        Q2 = Q1.clone()
        Q2[:, ni - 1] = torch.where(qn / a_e >= 1.0, Qe, Qsub)
        return Q2

    # ---------------------------------------------------------- time march
    def step(self, Q, amps, t, dt):
        """Q^{n+1} = BC(RK5(Q^n)) with the boundary conditions at t + dt."""
        MK = self.viscosity(Q)
        J9 = self.M[9]
        Jn = 1.0 / torch.where(J9 == 0, torch.ones_like(J9), J9)  # axis nodes are not advanced
        Q0, Qs = Q, Q
        for al in ALPHA:
            R = self.rhs(Qs, MK)
            Qs = torch.where(self.interior, Q0 - al * dt * (Jn * R), Q0)
        return self.boundary(Qs, amps, t + dt)

    def functional_term(self, Q, j_surface, dt):
        """dt sum_{i,k} (p(i, j_s, k) - 1/gamma)^2 J^-1 |grad eta| at (i, j_s, k)."""
        *_, p, _, _ = self.primitives(Q[:, :, j_surface:j_surface + 1])
        e = self.M[3:6, :, j_surface:j_surface + 1]
        dA = self.M[9, :, j_surface:j_surface + 1] * torch.sqrt((e * e).sum(0))
        dp = p - 1.0 / self.gamma
        return dt * (dp * dp * dA).sum()

    def window(self, Q0, amps, t0, dt, nsteps, j_surface):
        """J over nsteps steps from Q0 at t0 (terms after every step)."""
        Q = Q0
        J = torch.zeros((), dtype=torch.float64)
        for n in range(nsteps):
            Q = self.step(Q, amps, t0 + n * dt, dt)
            J = J + self.functional_term(Q, j_surface, dt)
        return J, Q
