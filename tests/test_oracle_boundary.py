"""Pins of the oracle's zero-gradient boundary (CPU only).

The paper gives no boundary treatment for the split sweeps (Sec. 3.3.1);
the reading taken is that a zero-gradient boundary fills the cells beyond
it with copies of the boundary layer (dc/dn = 0), and that a donor there is
reconstructed like any other cell, from its own 3x3x3 stencil of that
filled field (Sec. 3.2).  The filled field is invariant along the normal
beyond the wall, so its exact liquid flux through the wall face in a sweep
of CFL number a is a times the boundary cell's c, whatever the interface
looks like inside the domain.  The pins below check that closed form on
tilted planes that cross the walls, and that a sweep along an axis whose
boundary layer is invariant along that axis leaves it unchanged.
"""
import math
import os

import numpy as np
import pytest

import oracle as O


def plane_field(shape, n, d):
    """Exact cell fractions of {x : n . x <= d} on a grid of unit cells (x
    in cell units from the grid's low corner), by the oracle's volume
    function (pinned in test_oracle_geometry against brute force)."""
    nz, ny, nx = shape
    l1 = np.abs(n).sum()
    m = n / l1
    c = np.empty(shape)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c[k, j, i] = O.volume(m, (d - n @ np.array([i, j, k], float)) / l1)
    return c


def frozen_zero(c):
    return (c > 0.5).astype(np.uint8), np.zeros_like(c)


NORMALS = [np.array(v, float) / np.linalg.norm(v) for v in ((0.45, 0.8, 0.4), (-0.3, 0.7, -0.65),
                                                             (0.6, -0.5, 0.62))]


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("ni", range(len(NORMALS)))
def test_inflow_through_zero_gradient_wall_is_a_times_c(axis, ni):
    n = NORMALS[ni]
    shape = (9, 10, 11)
    c = plane_field(shape, n, d=float(n @ np.array([5.3, 4.9, 4.4])))
    g = O.Grid(11, 10, 9, (1, 1, 1), 0.1, 1.0, 1.0, 0.0)
    e = c.copy()
    cc, th = frozen_zero(c)
    fshape = list(shape)
    fshape[2 - axis] += 1
    for a in (0.3, -0.3):
        uf = np.full(fshape, a * 0.1 / 0.01)  # h = 0.1, dt = 0.01: CFL a on every face
        _, _, _, F, _ = O.sweep(g, axis, c, e, uf, 0.01, cc, th, want_flux=True)
        Fm = np.moveaxis(F, 2 - axis, 0)
        cm = np.moveaxis(c, 2 - axis, 0)
        face, cell = (0, 0) if a > 0 else (-1, -1)
        cb = cm[cell]
        mixed = (cb > 1e-12) & (cb < 1 - 1e-12)
        assert mixed.sum() >= 4
        # closed form of the boundary-filled field: F = a c_boundary
        assert np.abs(Fm[face] - a * cb).max() <= 1e-14
        # the plane itself is tilted across the wall: the boundary cell's own
        # plane (the reading that copies the reconstruction rather than c)
        # would flux a different volume
        own = []
        for idx in zip(*np.nonzero(mixed)):
            pos = [0, 0, 0]
            rest = [ax for ax in (2, 1, 0) if ax != axis]
            pos[2 - axis] = 0 if a > 0 else shape[2 - axis] - 1
            pos[2 - rest[0]], pos[2 - rest[1]] = idx
            k, j, i = pos
            s = np.zeros((3, 3, 3))
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        kk = min(max(k + dz, 0), shape[0] - 1)
                        jj = min(max(j + dy, 0), shape[1] - 1)
                        ii = min(max(i + dx, 0), shape[2] - 1)
                        s[dz + 1, dy + 1, dx + 1] = c[kk, jj, ii]
            m = O.myc(s)
            al = O.alpha(m, c[k, j, i])
            da = abs(a)
            own.append(O.slab_volume(m, al, axis, 1.0 - da if a > 0 else 0.0, da) * np.sign(a))
        assert np.abs(np.array(own) - a * cb[mixed]).max() > 1e-3


def test_layer_invariant_along_axis_stays():
    # A boundary layer invariant along x next to an interior that is too:
    # the whole field is x-invariant, every face fluxes a c of its donor,
    # and a sweep along x with uniform inflow leaves every cell unchanged.
    n = np.array((0.0, 0.8, 0.6))
    c = plane_field((8, 9, 10), n, d=4.3)
    g = O.Grid(10, 9, 8, (1, 1, 1), 0.1, 1.0, 1.0, 0.0)
    cc, th = frozen_zero(c)
    uf = np.full((8, 9, 11), 0.35 * 0.1 / 0.01)
    c1, _, _ = O.sweep(g, 0, c, c.copy(), uf, 0.01, cc, th)
    assert np.abs(c1 - c).max() <= 1e-15


def test_thread_count_does_not_change_results():
    # every sum is taken in cell order from per-cell values: the step is
    # bit-identical for 1 and several host threads
    from paper_2001_03477_gb300 import workloads as W
    wl = W.translating_sphere(n=20, nsteps=0, dd=-0.01, nsub=8)
    g = O.Grid(20, 20, 20, wl.bc, wl.h, wl.Cp_l, wl.Cp_g, wl.T_sat)
    out = []
    for nt in (1, max(2, os.cpu_count() or 2)):
        O.set_threads(nt)
        c, e = wl.c.copy(), wl.e.copy()
        sums = None
        for s in range(3):
            c, e, sums = O.step(g, c, e, wl.u, wl.v, wl.w, wl.dt, s, dd_uniform=-0.01)
        out.append((c, e, np.asarray(sums)))
    O.set_threads(os.cpu_count() or 1)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
