"""GPU parity of the Lagrangian-explicit sweeps (vof_grid.scheme =
VOF_SCHEME_LE, Li's scheme, the alternative Step 1 named in Sec. 3.3.1)
through the C ABI against the FP64 oracle's orc_sweep_le / orc_step_scheme,
element by element on the inputs of the Weymouth-Yue parity tests.

Tolerances as for the Weymouth-Yue form (c 1e-12 absolute, T 1e-11
relative, totals 1e-13 relative): the fluxes are the same slab volumes of
the same planes, with the width |a| / J and the factor J formed by the same
separately rounded operations on both sides.  In full steps, cells that the
shift finds cut only at a corner are held to 1e-10 (see test_step_le).
"""
import numpy as np
import pytest

import oracle as O
from test_parity_gpu import C_TOL, SUM_TOL, T_TOL, CASES, case, dev, host, ogrid, temperature

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_03477_gb300 import build
    build.build()
    import paper_2001_03477_gb300 as P
    return P


def le_grid(P, g, precision=0):
    return P.Grid(g.nx, g.ny, g.nz, g.bc, g.h, g.Cp_l, g.Cp_g, g.T_sat, g.eps_mixed, precision=precision,
                  scheme=P.VOF_SCHEME_LE)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sweep_le(P, name, axis):
    import torch
    g, c, e, vel, dt, _ = case(name)
    og = ogrid(g)
    co, eo, clip, Fo, Go = O.sweep_le(og, axis, c, e, vel[axis], dt, want_flux=True)
    gl = le_grid(P, g)
    cd, ed, uf = dev(c), dev(e), dev(vel[axis])
    c2 = torch.empty_like(cd); e2 = torch.empty_like(ed)
    flux = torch.zeros(g.face_shape(axis), dtype=torch.float64, device="cuda")
    diag = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.SWEEPS[axis](gl, cd, ed, c2, e2, uf, dt, None, None, flux, diag)
    cg, eg = host(c2), host(e2)
    assert np.abs(cg - co).max() <= C_TOL
    To, Tg = temperature(g, co, eo), temperature(g, cg, eg)
    assert (np.abs(Tg - To) / np.maximum(np.abs(To), 1e-300)).max() <= T_TOL
    assert np.abs(host(flux) - Fo).max() <= C_TOL
    assert abs(host(diag)[0] - clip) <= C_TOL
    # unfused: the VOF-only sweep, then the energy from its fluxes == fused
    c3 = torch.empty_like(cd); e3 = torch.empty_like(ed)
    flux2 = torch.zeros_like(flux)
    P.SWEEPS[axis](gl, cd, None, c3, None, uf, dt, None, None, flux2, None)
    P.energy_advect_consistent(gl, axis, cd, c3, ed, e3, flux2, uf, dt)
    assert torch.equal(c3, c2) and torch.equal(flux2, flux)
    assert torch.equal(e3, e2)


@pytest.mark.parametrize("name", CASES)
def test_step_le(P, name):
    """Full steps against the oracle's.  The sweeps agree to ~1 ulp per cell
    (plane constants differ in the last bits), and the shift of a cell cut
    only at a corner (c within 1e-6 of 0 or 1 after the sweeps) turns a
    1-ulp change of its c into ~1e4 ulps of its shifted volume (the plane
    position goes as the cube root of the corner volume): such cells are
    held to 1e-10, all others to the per-cell bound."""
    g, c, e, (u, v, w), dt, dd = case(name)
    og = ogrid(g)
    st = P.Stepper(le_grid(P, g))
    ud, vd, wd = dev(u), dev(v), dev(w)
    ci, ei = c, e
    for s in range(2):
        co, eo, so = O.step(og, ci, ei, u, v, w, dt, s, dd_uniform=dd, scheme=1)
        cs, es = ci, ei
        for ax in ([0, 1, 2] if s % 2 == 0 else [2, 1, 0]):
            cs, es, _ = O.sweep_le(og, ax, cs, es, (u, v, w)[ax], dt)
        corner = ((cs > 1e-12) & (cs < 1e-6)) | ((cs > 1 - 1e-6) & (cs < 1 - 1e-12))
        cd, ed = dev(ci), dev(ei)
        sg = host(st.step(cd, ed, ud, vd, wd, dt, s, dd_uniform=dd)).copy()
        cg, eg = host(cd), host(ed)
        err = np.abs(cg - co)
        assert err[~corner].max() <= C_TOL
        assert err.max() <= 1e-10
        To, Tg = temperature(g, co, eo), temperature(g, cg, eg)
        assert (np.abs(Tg - To) / np.abs(To)).max() <= T_TOL
        assert abs(sg[0] - so[0]) <= SUM_TOL * abs(so[0])
        assert abs(sg[1] - so[1]) <= SUM_TOL * abs(so[1])
        for k in (2, 3, 4, 5):
            assert abs(sg[k] - so[k]) <= 1e-12 * max(1.0, abs(so[k]))
        ci, ei = co, eo


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_linear_velocity_moves_a_plane_exactly_on_gpu(P, axis):
    """The oracle's exactness pin on the GPU: a velocity linear along the
    sweep axis moves a plane interface x = x0 to x0 + a(x0) exactly."""
    import torch
    n, m = 24, 3
    shape = [m, m, m]
    shape[2 - axis] = n
    shape = tuple(shape)
    beta, xs, x0 = -0.05, 11.3, 9.6
    sh = [1, 1, 1]
    sh[2 - axis] = n
    k = np.arange(n, dtype=float)
    c = np.broadcast_to(np.clip(x0 - k, 0.0, 1.0).reshape(sh), shape).copy()
    fshape = list(shape)
    fshape[2 - axis] += 1
    sh2 = [1, 1, 1]
    sh2[2 - axis] = n + 1
    uf = np.broadcast_to((beta * (np.arange(n + 1) - xs)).reshape(sh2), tuple(fshape)).copy()
    bc = [0, 0, 0]
    bc[axis] = 1
    g = P.Grid(shape[2], shape[1], shape[0], tuple(bc), 1.0, 3.0, 1.0, 1.0, scheme=P.VOF_SCHEME_LE)
    e = (3.0 * c + (1 - c)) * 2.0
    cd, ed = dev(c), dev(e)
    c2 = torch.empty_like(cd); e2 = torch.empty_like(ed)
    P.SWEEPS[axis](g, cd, ed, c2, e2, dev(uf), 1.0)
    x1 = x0 + beta * (x0 - xs)
    want = np.broadcast_to(np.clip(x1 - k, 0.0, 1.0).reshape(sh), shape)
    cg, eg = host(c2), host(e2)
    assert np.abs(cg - want).max() < 1e-14
    assert np.abs(eg / (3.0 * cg + (1 - cg)) - 2.0).max() < 1e-14


def test_scheme_validation(P):
    import ctypes
    g = P.Grid(8, 8, 8, scheme=2).c_struct()
    assert P.lib().vof_step_workspace_bytes(ctypes.byref(g)) == 0
