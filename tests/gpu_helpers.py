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
    kw.pop("metric_form", None)
    return orc.params(**kw)


BLOCK_HALF = 13  # one step reaches 12 nodes: 5 stages x 2, viscosity 1, block metrics 1


def take_blocks(torch, Q, centres, nk, half=BLOCK_HALF):
    """Host copies of the (2 half + 1)^3 blocks of device state Q around the
    given (i, j, k) centres (k wraps)."""
    out = []
    for (i, j, k) in centres:
        kk = torch.arange(k - half, k + half + 1, device=Q.device) % nk
        blk = Q[:, i - half:i + half + 1, j - half:j + half + 1][:, :, :, kk]
        out.append(blk.cpu().numpy())
    return out


def check_blocks(orc, synth, shape, Q_after, centres, blocks, dt, tol, half=BLOCK_HALF, **kw):
    """One oracle step on each block (faces frozen, fixed dt) against the
    device state after one step at the block centre; tolerance relative to
    the component scale (rho v, rho w share the momentum scale)."""
    ni, nj, nk = shape
    for (i, j, k), Qb in zip(centres, blocks):
        assert half <= i <= ni - 1 - half and half <= j <= nj - 1 - half
        ii = np.arange(i - half, i + half + 1)
        jj = np.arange(j - half, j + half + 1)
        kk = np.arange(k - half, k + half + 1)
        xyzb = synth.jet_grid_block(ni, nj, nk, ii, jj, kk)
        Mb = orc.metrics(xyzb, (0, 0, 0))
        P = orc.params(dt_mode=1, dt_fixed=dt, bc=0, periodic=(0, 0, 0), **kw)
        Qb1, _ = orc.rk_step(P, Qb, Mb, xyzb, 0.0)
        ref = Qb1[:, half, half, half]
        got = Q_after[:, i, j, k].cpu().numpy()
        mom = np.abs(Qb[1:4]).max()
        scale = np.array([np.abs(Qb[0]).max(), mom, mom, mom, np.abs(Qb[4]).max()])
        assert np.all(np.abs(got - ref) <= tol * scale), ((i, j, k), got, ref)
