"""Shared helpers of the GPU parity tests: both sides get the same grid and
the same initial bits; norms follow one convention for every comparison."""
import numpy as np


def rel_linf(a, b):
    """Max over the 5 components of max|a_c - b_c| / max|b_c|; the three
    momentum components share the momentum-magnitude scale (rho v and rho w
    are ~1e-3 of rho u in the jet)."""
    a = np.asarray(a)
    b = np.asarray(b)
    mom = max(np.abs(b[1]).max(), np.abs(b[2]).max(), np.abs(b[3]).max())
    worst = 0.0
    for c in range(5):
        scale = mom if c in (1, 2, 3) else np.abs(b[c]).max()
        if scale == 0:
            scale = 1.0
        worst = max(worst, np.abs(a[c] - b[c]).max() / scale)
    return worst


def rel_l2(a, b, comps=(0, 1, 4)):
    """Max over the listed components of ||a_c - b_c||_2 / ||b_c||_2."""
    return max(np.linalg.norm((a[c] - b[c]).ravel()) / np.linalg.norm(b[c].ravel())
               for c in comps)


def device_ctx(lj, torch, shape, xyz, shift=None, **kw):
    ctx = lj.Context(lj.make_params(**kw), shape, "cuda:0")
    xyz_d = torch.from_numpy(np.ascontiguousarray(xyz)).cuda()
    ctx.les_set_grid(xyz_d, shift)
    return ctx, xyz_d


def oracle_params(orc, **kw):
    kw = dict(kw)
    kw.pop("precision", None)
    return orc.params(**kw)
