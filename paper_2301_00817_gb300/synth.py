"""Seeded synthetic inputs: grids and primitive fields.

This module generates the coordinates and the primitive (rho, u, v, w, p)
fields that stand in for the paper's jet meshes A-I (Table tab:mesh, 361
azimuthal points, 5.9M to 1.04B points) and its jet flow.  It holds none of
the method's arithmetic (no equation of state, no flux, no metric): both the
CUDA path and the CPU oracle take its arrays as data.

Jet grid (annular cylinder, the configuration of Sec. "Boundary Conditions"):
  * axial x in [0, 20 D], geometric spacing dx_{i+1} = 1.01 dx_i;
  * radial r in [0.02 D, 10 D], hyperbolic-tangent clustering at r = 0.5 D:
    r(s) = r0 + (r1 - r0) g(s)/g(1), g(s) = s - (A/beta)[tanh(beta(s - s_c))
    + tanh(beta s_c)], s = j/(nj-1), A = 0.9, beta = 8, s_c chosen by
    bisection so that r(s_c) = 0.5 D (spacing there is (1-A) of the mean);
  * azimuth theta_k = 2 pi k / nk (nk distinct points, periodic);
  * x = x_i, y = r_j cos theta_k, z = r_j sin theta_k (right-handed, J > 0).
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------- jet grid


def jet_axial(ni: int, length: float = 20.0, ratio: float | None = None) -> np.ndarray:
    """Axial stations x_0 = 0 ... x_{ni-1} = length, dx_{i+1} = ratio dx_i.

    The default ratio is 1.01 up to 288 planes (the Mesh-A size); finer grids
    refine that same geometric mapping, ratio = 1.01^(288/ni), so the spacing
    still grows 17-fold over the domain.  (Taken literally at 2000 planes, a
    ratio of 1.01 would make the first cell 4.6e-10 D long, 4.3e8 times
    shorter than the last, and the convective CFL step viscously unstable.)"""
    if ratio is None:
        ratio = 1.01 if ni <= 288 else 1.01 ** (288.0 / ni)
    i = np.arange(ni, dtype=np.float64)
    if ratio == 1.0:
        return length * i / (ni - 1)
    dx0 = length * (ratio - 1.0) / (ratio ** (ni - 1) - 1.0)
    return dx0 * (ratio ** i - 1.0) / (ratio - 1.0)


def _tanh_map(s, sc, A, beta):
    return s - (A / beta) * (np.tanh(beta * (s - sc)) + np.tanh(beta * sc))


def jet_radial(nj: int, r0: float = 0.02, r1: float = 10.0, r_c: float = 0.5,
               A: float = 0.9, beta: float = 8.0) -> np.ndarray:
    """Radial stations clustered at r_c (spacing minimum (1-A) x mean)."""
    def r_of(s, sc):
        return r0 + (r1 - r0) * _tanh_map(s, sc, A, beta) / _tanh_map(1.0, sc, A, beta)

    lo, hi = 0.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if r_of(mid, mid) < r_c:
            lo = mid
        else:
            hi = mid
    sc = 0.5 * (lo + hi)
    s = np.arange(nj, dtype=np.float64) / (nj - 1)
    return r_of(s, sc)


def jet_azimuth(nk: int) -> np.ndarray:
    return 2.0 * math.pi * np.arange(nk, dtype=np.float64) / nk


def jet_lines(ni: int, nj: int, nk: int, r0: float = 0.02):
    """The three 1-D coordinate lines (x_i, r_j, theta_k) of the jet grid."""
    return jet_axial(ni), jet_radial(nj, r0=r0), jet_azimuth(nk)


def jet_grid(ni: int, nj: int, nk: int, r0: float = 0.02) -> np.ndarray:
    """Cartesian coordinates [3, ni, nj, nk] (FP64) of the jet grid: annular
    for r0 > 0 (the default), a true centerline grid (r_0 = 0 exactly, the nk
    nodes of ring j = 0 on the axis) for r0 = 0."""
    x, r, th = jet_lines(ni, nj, nk, r0)
    xyz = np.empty((3, ni, nj, nk))
    xyz[0] = x[:, None, None]
    xyz[1] = r[None, :, None] * np.cos(th)[None, None, :]
    xyz[2] = r[None, :, None] * np.sin(th)[None, None, :]
    return xyz


def jet_grid_block(ni: int, nj: int, nk: int, ii, jj, kk) -> np.ndarray:
    """Coordinates [3, len(ii), len(jj), len(kk)] of the nodes (ii x jj x kk)
    of the ni x nj x nk jet grid (index arrays; kk may wrap)."""
    x, r, th = jet_lines(ni, nj, nk)
    x, r, th = x[np.asarray(ii)], r[np.asarray(jj)], th[np.asarray(kk) % nk]
    xyz = np.empty((3, len(x), len(r), len(th)))
    xyz[0] = x[:, None, None]
    xyz[1] = r[None, :, None] * np.cos(th)[None, None, :]
    xyz[2] = r[None, :, None] * np.sin(th)[None, None, :]
    return xyz


def jet_grid_torch(ni: int, nj: int, nk: int, device):
    """jet_grid assembled on a torch device from the host's 1-D lines, for
    grids too large to build on the host: every coordinate is the same single
    product as in jet_grid, so the two agree bit for bit."""
    import torch
    x, r, th = jet_lines(ni, nj, nk)
    xt = torch.from_numpy(x).to(device)
    rt = torch.from_numpy(r).to(device)
    ct = torch.from_numpy(np.cos(th)).to(device)
    st = torch.from_numpy(np.sin(th)).to(device)
    xyz = torch.empty((3, ni, nj, nk), dtype=torch.float64, device=device)
    xyz[0] = xt[:, None, None]
    xyz[1] = rt[None, :, None] * ct[None, None, :]
    xyz[2] = rt[None, :, None] * st[None, None, :]
    return xyz


JET_PERIODIC = (0, 0, 1)
JET_SHIFT = np.zeros(9)

# ------------------------------------------------------- periodic test boxes


def box_grid(n: tuple[int, int, int], L: tuple[float, float, float] = (1.0, 1.0, 1.0),
             wave: float = 0.0):
    """Triply periodic box, optionally with a smooth non-separable wave.

    Returns (xyz, shift) where shift[d] is the coordinate jump over one period
    of computational direction d.  With wave > 0 every coordinate is displaced
    by a periodic function of all three indices, so the metrics are fully 3-D.
    """
    ni, nj, nk = n
    s = [np.arange(m, dtype=np.float64) / m for m in n]
    S0, S1, S2 = np.meshgrid(*s, indexing="ij")
    tp = 2.0 * math.pi
    x = L[0] * S0 + wave * L[0] * np.sin(tp * S1) * np.sin(tp * S2) / tp
    y = L[1] * S1 + wave * L[1] * np.sin(tp * S0) * np.cos(tp * S2) / tp
    z = L[2] * S2 + wave * L[2] * np.cos(tp * S0) * np.sin(tp * S1) / tp
    xyz = np.stack([x, y, z])
    shift = np.zeros((3, 3))
    shift[0, 0], shift[1, 1], shift[2, 2] = L
    return xyz, shift.reshape(9)


def smooth_periodic_prim(xyz: np.ndarray, L=(1.0, 1.0, 1.0), amp: float = 0.1,
                         seed: int = 0) -> np.ndarray:
    """Smooth periodic primitive fields (rho,u,v,w,p) [5, ...] on a box."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0.0, 2.0 * math.pi, size=(5, 3))
    kx = [2.0 * math.pi / Lc for Lc in L]
    x, y, z = xyz
    fields = []
    base = [1.0, 0.3, -0.2, 0.1, 1.0 / 1.4]
    for c in range(5):
        f = (np.sin(kx[0] * x + ph[c, 0]) * np.cos(kx[1] * y + ph[c, 1]) +
             0.5 * np.sin(kx[2] * z + ph[c, 2]) * np.cos(kx[0] * x - ph[c, 1]))
        scale = amp * (base[c] if c in (0, 4) else 1.0)
        fields.append(base[c] + scale * f)
    return np.stack(fields)


def uniform_prim(shape, rho=1.0, u=0.0, v=0.0, w=0.0, p=1.0 / 1.4) -> np.ndarray:
    out = np.empty((5,) + tuple(shape))
    out[0], out[1], out[2], out[3], out[4] = rho, u, v, w, p
    return out


def forcing_amplitudes(seed: int, scale: float = 1.0e-3 * 1.4) -> np.ndarray:
    """16 inflow-forcing amplitudes a_{m f} ~ N(0, scale), index m*4 + f."""
    return np.random.default_rng(seed).normal(0.0, scale, size=16)


# Workloads standing in for the paper's meshes (Table tab:mesh).
CONFIGS = {
    "c1": dict(shape=(48, 24, 32), Re=1.0e5, steps=20),
    "c2": dict(shape=(288, 160, 128), Re=1.0e5, steps=100),
    "c3": dict(shape=(576, 320, 256), Re=1.0e6, steps=200),
    "c4": dict(shape=(192, 96, 128), Re=1.0e5, steps=50),
    "c5": dict(shape=(2000, 500, 1024), Re=1.0e5, steps=20),
}
