"""GPU parity of the velocity extension (Sec. 3.3.1, Eq. press_inv) through
the C ABI against the oracle (oracle/extension.py, a direct sparse solve).

Both sides build the same sub-domain (layer codes are exact integer work),
the same couplings (the same separately rounded operations) and sources that
differ only through the plane constants' last bits and the two ways of
measuring the cut area (polygon fan about the centroid in the oracle;
projected shoelace here).  The GPU solves by conjugate gradients to a
residual of 1e-14 of the initial one; the corrections then agree to a few
1e-12 of the largest correction (the condition number of these thin
sub-domains is O(10^2)): checked at 1e-9.  The sub-domain's faces, and the
zero faces (liquid cells, walls, outside), are compared exactly.
"""
import zlib

import numpy as np
import pytest

from oracle import Grid as OGrid
from oracle.extension import velocity_extension
from paper_2001_03477_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RHO_L, RHO_G = 958.0, 0.6


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_03477_gb300 import build
    build.build()
    import paper_2001_03477_gb300 as P
    return P


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype=torch.float64)


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def case(name):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    if name == "plane":
        c = np.zeros((12, 4, 4))
        c[:5] = 1.0
        c[5] = 0.35
        return c, np.where((c > 0) & (c < 1), 0.05, 0.0), (0, 0, 1), 0.01
    if name in ("drop", "bubble"):
        n = 20
        h = 1.0 / n
        c = W.sphere_fractions((n, n, n), h, (0.5, 0.48, 0.52), 0.23, inside=1.0 if name == "drop" else 0.0, nsub=10)
        mixed = (c > 1e-12) & (c < 1 - 1e-12)
        return c, np.where(mixed, 0.02 + 0.01 * rng.random(c.shape), 0.0), (1, 1, 1), h
    if name == "ragged_periodic":
        nx, ny, nz = 23, 17, 13
        h = 1.0 / 16
        c = W.ellipsoid_fractions((nz, ny, nx), h, (0.7, 0.5, 0.4), (0.35, 0.3, 0.25),
                                  rot=np.linalg.qr(rng.normal(size=(3, 3)))[0], nsub=8)
        mixed = (c > 1e-12) & (c < 1 - 1e-12)
        return c, np.where(mixed, 0.03 * rng.random(c.shape), 0.0), (0, 1, 0), h
    raise KeyError(name)


CASES = ["plane", "drop", "bubble", "ragged_periodic"]


def active_faces(sub, liquid, axis, bc):
    """Faces that may carry a correction: a sub-domain cell on one side, no
    liquid cell on either side, not a zero-gradient wall (face layout of
    `axis`; a periodic face n is face 0)."""
    ax = 2 - axis  # numpy axis of `axis`
    n = sub.shape[ax]
    lo = np.concatenate([np.take(sub, [n - 1], axis=ax), sub], axis=ax)
    hi = np.concatenate([sub, np.take(sub, [0], axis=ax)], axis=ax)
    llo = np.concatenate([np.take(liquid, [n - 1], axis=ax), liquid], axis=ax)
    lhi = np.concatenate([liquid, np.take(liquid, [0], axis=ax)], axis=ax)
    act = (lo | hi) & ~llo & ~lhi
    if bc[axis] != 0:
        idx = [slice(None)] * 3
        idx[ax] = 0
        act[tuple(idx)] = False
        idx[ax] = n
        act[tuple(idx)] = False
    return act


@pytest.mark.parametrize("name", CASES)
def test_velocity_extension_parity(P, name):
    import torch
    c, mdot, bc, h = case(name)
    nz, ny, nx = c.shape
    dt = 1e-3
    og = OGrid(nx, ny, nz, bc, h, 1.0, 1.0, 1.0)
    uo, vo, wo, layer, _ = velocity_extension(og, c, mdot, RHO_L, RHO_G, dt)
    g = P.Grid(nx, ny, nz, bc, h, 1.0, 1.0, 1.0)
    cd, md = dev(c), dev(mdot)
    shapes = [og.face_shape(a) for a in range(3)]
    ut, vt, wt = (torch.full(s, 7.0, dtype=torch.float64, device="cuda") for s in shapes)
    base = [np.random.default_rng(a).random(s) for a, s in enumerate(shapes)]
    u, v, w = (dev(b) for b in base)
    it, res = P.vof_velocity_extension(g, cd, md, RHO_L, RHO_G, dt, tol=1e-14, u=u, v=v, w=w, ut=ut, vt=vt, wt=wt)
    assert it >= 1
    got = [host(ut), host(vt), host(wt)]
    want = [uo, vo, wo]
    scale = max(np.abs(x).max() for x in want)
    assert scale > 0
    sub = layer >= 0
    liquid = c >= 1 - 1e-12
    for axis, (gt, wn) in enumerate(zip(got, want)):
        active = active_faces(sub, liquid, axis, bc)
        assert np.all(gt[~active] == 0.0) and np.all(wn[~active] == 0.0)
        assert np.abs(gt - wn).max() <= 1e-9 * scale
    # u_l = u + u~ (the same additions)
    for b, t_out, gt in zip(base, (u, v, w), got):
        assert np.array_equal(host(t_out), b + gt)


def test_plane_closed_form_on_gpu(P):
    import torch
    c, mdot, bc, h = case("plane")
    g = P.Grid(4, 4, 12, bc, h, 1.0, 1.0, 1.0)
    wt = torch.empty((13, 4, 4), dtype=torch.float64, device="cuda")
    ut = torch.empty((12, 4, 5), dtype=torch.float64, device="cuda")
    vt = torch.empty((12, 5, 4), dtype=torch.float64, device="cuda")
    P.vof_velocity_extension(g, dev(c), dev(mdot), RHO_L, RHO_G, 1e-3, tol=1e-14, ut=ut, vt=vt, wt=wt)
    jump = 0.05 * (1 / RHO_G - 1 / RHO_L)
    want = np.zeros(13)
    want[6:9] = -jump
    assert np.abs(host(wt) - want[:, None, None]).max() <= 1e-12 * jump


def test_no_free_flow_face_on_gpu(P):
    import torch
    c = np.zeros((5, 2, 2))
    c[:2] = 1.0
    c[2] = 0.5
    g = P.Grid(2, 2, 5, (0, 0, 0), 0.1, 1.0, 1.0, 1.0)
    ut = torch.zeros((5, 2, 3), dtype=torch.float64, device="cuda")
    vt = torch.zeros((5, 3, 2), dtype=torch.float64, device="cuda")
    wt = torch.zeros((6, 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(P.VofError):
        P.vof_velocity_extension(g, dev(c), dev(np.where(c == 0.5, 0.01, 0.0)), RHO_L, RHO_G, 1e-3, ut=ut, vt=vt,
                                 wt=wt)


def test_iteration_cap_reports_esolve(P):
    import torch
    c, mdot, bc, h = case("drop")
    n = c.shape[0]
    g = P.Grid(n, n, n, bc, h, 1.0, 1.0, 1.0)
    ut, vt, wt = (torch.zeros(s, dtype=torch.float64, device="cuda")
                  for s in ((n, n, n + 1), (n, n + 1, n), (n + 1, n, n)))
    with pytest.raises(P.VofError) as err:
        P.vof_velocity_extension(g, dev(c), dev(mdot), RHO_L, RHO_G, 1e-3, tol=1e-300, max_iter=1, ut=ut, vt=vt,
                                 wt=wt)
    assert err.value.status == P.VOF_ESOLVE
