"""vof_step_noalloc: the time step for callers that cannot allocate device
memory while they step (it keeps its scratch in a fixed array inside the
library instead of a caller-provided workspace).  Checked through the C ABI
against vof_step on the same inputs, two steps in a row (the second step
finds the array holding the first step's leftovers), with the parity
tolerances of the other GPU tests.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C_TOL = 1e-12
T_TOL = 1e-11
SUM_TOL = 1e-13


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_03477_gb300 import build
    build.build()
    import paper_2001_03477_gb300 as P
    return P


def _case(P):
    from paper_2001_03477_gb300 import workloads as W
    rng = np.random.default_rng(2024)
    nx, ny, nz = 45, 38, 29  # ragged, several CTA tiles, 49590 cells
    h = 1.0 / 40
    g = P.Grid(nx, ny, nz, (0, 1, 0), h, 1000.0, 1.0, 1.0)
    c = W.ellipsoid_fractions((nz, ny, nx), h, (0.55, 0.45, 0.36), (0.3, 0.25, 0.2),
                              rot=np.linalg.qr(rng.normal(size=(3, 3)))[0], nsub=8)
    u, v, w = W.deformation_faces((nz, ny, nx), h, 0.3)
    T = 1.0 + 0.1 * rng.random((nz, ny, nx))
    e = (1000.0 * c + (1 - c)) * T
    return g, c, e, (u, v, w), 0.2 * h / 2.0, -0.02


def test_noalloc_matches_vof_step_two_calls(P):
    import torch
    g, c, e, (u, v, w), dt, dd = _case(P)
    dev = torch.device("cuda")
    ud, vd, wd = (torch.from_numpy(a).to(dev) for a in (u, v, w))
    # reference: the existing entry point with a caller workspace
    st = P.Stepper(g, device=dev)
    c1, e1 = torch.from_numpy(c).to(dev), torch.from_numpy(e).to(dev)
    # no-alloc entry point
    c2, e2 = torch.from_numpy(c).to(dev), torch.from_numpy(e).to(dev)
    sums2 = torch.zeros(P.VOF_NSUMS, dtype=torch.float64, device=dev)
    for s in range(2):
        s1 = st.step(c1, e1, ud, vd, wd, dt, s, dd_uniform=dd).cpu().numpy()
        P.vof_step_noalloc(g, c2, e2, ud, vd, wd, dt, s, dd_uniform=dd, sums=sums2)
        torch.cuda.synchronize()
        a1, a2 = c1.cpu().numpy(), c2.cpu().numpy()
        b1, b2 = e1.cpu().numpy(), e2.cpu().numpy()
        assert np.abs(a1 - a2).max() <= C_TOL
        T1 = b1 / (1000.0 * a1 + (1 - a1))
        T2 = b2 / (1000.0 * a2 + (1 - a2))
        assert (np.abs(T1 - T2) / np.abs(T1)).max() <= T_TOL
        s2 = sums2.cpu().numpy()
        assert abs(s2[0] - s1[0]) <= SUM_TOL * abs(s1[0])
        assert abs(s2[1] - s1[1]) <= SUM_TOL * abs(s1[1])
        # the same kernels in the same order: the same bits, whatever the
        # scratch held before
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
        assert np.array_equal(s1[:2], s2[:2])


def test_noalloc_after_other_grid(P):
    """The array still holds what a call on a grid of another shape left in
    it (other offsets of the frozen state, counters and lists): a step on
    the 45x38x29 case after two steps on a thin 64x8x8 grid must match
    vof_step with a fresh workspace."""
    import torch
    from paper_2001_03477_gb300 import workloads as W
    dev = torch.device("cuda")
    # a thin periodic grid with a tilted slab of liquid and uniform velocity
    h0 = 1.0 / 64
    g0 = P.Grid(64, 8, 8, (0, 0, 0), h0, 1000.0, 1.0, 1.0)
    zz, yy, xx = np.meshgrid(np.arange(8), np.arange(8), np.arange(64), indexing="ij")
    c0 = np.clip(0.5 + (20.0 - xx - 0.7 * yy - 0.3 * zz) / 3.0, 0.0, 1.0)
    e0 = (1000.0 * c0 + (1 - c0)) * 1.5
    f0 = [np.full(s, v) for s, v in (((8, 8, 65), 0.8), ((8, 9, 64), -0.3), ((9, 8, 64), 0.2))]
    cg0, eg0 = torch.from_numpy(c0).to(dev), torch.from_numpy(e0).to(dev)
    fd0 = [torch.from_numpy(a).to(dev) for a in f0]
    for s in range(2):
        P.vof_step_noalloc(g0, cg0, eg0, *fd0, 0.2 * h0, s, dd_uniform=0.01)
    torch.cuda.synchronize()
    assert np.isfinite(cg0.cpu().numpy()).all()

    g, c, e, (u, v, w), dt, dd = _case(P)
    ud, vd, wd = (torch.from_numpy(a).to(dev) for a in (u, v, w))
    c1, e1 = torch.from_numpy(c).to(dev), torch.from_numpy(e).to(dev)
    s1 = P.Stepper(g, device=dev).step(c1, e1, ud, vd, wd, dt, 0, dd_uniform=dd).cpu().numpy()
    c2, e2 = torch.from_numpy(c).to(dev), torch.from_numpy(e).to(dev)
    sums2 = torch.zeros(P.VOF_NSUMS, dtype=torch.float64, device=dev)
    P.vof_step_noalloc(g, c2, e2, ud, vd, wd, dt, 0, dd_uniform=dd, sums=sums2)
    torch.cuda.synchronize()
    a1, a2 = c1.cpu().numpy(), c2.cpu().numpy()
    b1, b2 = e1.cpu().numpy(), e2.cpu().numpy()
    assert np.abs(a1 - a2).max() <= C_TOL
    T1 = b1 / (1000.0 * a1 + (1 - a1))
    T2 = b2 / (1000.0 * a2 + (1 - a2))
    assert (np.abs(T1 - T2) / np.abs(T1)).max() <= T_TOL
    s2 = sums2.cpu().numpy()
    assert abs(s2[0] - s1[0]) <= SUM_TOL * abs(s1[0])
    assert abs(s2[1] - s1[1]) <= SUM_TOL * abs(s1[1])
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    assert np.array_equal(s1[:2], s2[:2])


def test_noalloc_rejects_large_grid(P):
    import torch
    g = P.Grid(65, 64, 64)  # one plane above the limit
    assert g.cells > P.VOF_NOALLOC_MAX_CELLS
    cg = g.c_struct()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    st = P.lib().vof_step_noalloc(ctypes.byref(cg), p, p, p, p, p, 0.1, 0, None, 0.0, None, None)
    assert st == P.VOF_EINVAL
