"""Pins of the oracle's velocity extension (Sec. 3.3.1: Eq. press_inv, the
correction u~ and u_l = u^{n+1} + u~) against what the mathematics fixes
(CPU only).

* A plane interface with a uniform mass flux: the source sits in the mixed
  layer, no-slip closes the liquid side, and continuity carries the whole
  flux through the two gas layers to the free-flow faces, so u~ normal to the
  plane equals -mdot (1/rho_g - 1/rho_l) on the mixed cells' gas-side face
  and on the faces of both gas layers, and vanishes everywhere else -- the
  jump of the one-fluid velocity across an evaporating interface, removed.
* Any interface: the discrete divergence of u~ in every sub-domain cell is
  -mdot (1/rho_g - 1/rho_l) A / h (A the PLIC area), to solver round-off,
  and u~ vanishes on every face of a liquid cell.
* Symmetry: a centred sphere with a uniform mass flux gives a mirror-
  symmetric u~.
* mdot = 0 gives u~ = 0; a sub-domain with no free-flow face is rejected.
"""
import numpy as np
import pytest

import oracle as O
from oracle.extension import subdomain_layers, velocity_extension
from paper_2001_03477_gb300 import workloads as W

RHO_L, RHO_G = 958.0, 0.6


def div(ut, vt, wt, h):
    return ((ut[:, :, 1:] - ut[:, :, :-1]) + (vt[:, 1:, :] - vt[:, :-1, :]) + (wt[1:] - wt[:-1])) / h


@pytest.mark.parametrize("liquid_below", [True, False])
def test_plane_interface_closed_form(liquid_below):
    nx = ny = 4
    nz = 12
    k0, frac = 5, 0.35
    c = np.zeros((nz, ny, nx))
    if liquid_below:
        c[:k0] = 1.0
        c[k0] = frac
    else:
        c[k0 + 1:] = 1.0
        c[k0] = frac
    h, dt, md = 0.01, 1e-3, 0.05
    g = O.Grid(nx, ny, nz, (0, 0, 1), h, 1.0, 1.0, 1.0)
    mdot = np.where((c > 0) & (c < 1), md, 0.0)
    ut, vt, wt, layer, p = velocity_extension(g, c, mdot, RHO_L, RHO_G, dt)
    jump = md * (1.0 / RHO_G - 1.0 / RHO_L)
    want = np.zeros(nz + 1)
    if liquid_below:
        want[k0 + 1:k0 + 4] = -jump  # faces above the mixed layer, through layer 2
    else:
        want[k0 - 2:k0 + 1] = jump   # the same, mirrored: the gas lies below
    assert np.abs(wt - want[:, None, None]).max() <= 1e-12 * jump
    assert np.abs(ut).max() <= 1e-12 * jump and np.abs(vt).max() <= 1e-12 * jump
    assert np.count_nonzero(layer == 0) == nx * ny and np.count_nonzero(layer == 2) == nx * ny


def sphere_case(n=20, seed=1, liquid_inside=True):
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    c = W.sphere_fractions((n, n, n), h, (0.5, 0.48, 0.52), 0.23, inside=1.0 if liquid_inside else 0.0, nsub=10)
    mixed = (c > 1e-12) & (c < 1 - 1e-12)
    mdot = np.where(mixed, 0.02 + 0.01 * rng.random(c.shape), 0.0)
    return c, mdot, h


@pytest.mark.parametrize("liquid_inside", [True, False])
def test_divergence_cancels_the_source(liquid_inside):
    c, mdot, h = sphere_case(liquid_inside=liquid_inside)
    n = c.shape[0]
    g = O.Grid(n, n, n, (1, 1, 1), h, 1.0, 1.0, 1.0)
    dt = 1e-3
    ut, vt, wt, layer, p = velocity_extension(g, c, mdot, RHO_L, RHO_G, dt)
    m, al, mixed = O.reconstruct(g, c)
    src = np.zeros(c.shape)
    for P in zip(*np.nonzero(mixed)):
        src[P] = mdot[P] * (1 / RHO_G - 1 / RHO_L) * O.plane_area(m[(slice(None),) + P], al[P]) / h
    d = div(ut, vt, wt, h)
    sub = layer >= 0
    assert np.abs(d[sub] + src[sub]).max() <= 1e-9 * np.abs(src).max()
    # nothing moves through a liquid cell's faces
    liquid = c >= 1 - 1e-12
    for L in zip(*np.nonzero(liquid)):
        k, j, i = L
        assert ut[k, j, i] == 0 and ut[k, j, i + 1] == 0
        assert vt[k, j, i] == 0 and vt[k, j + 1, i] == 0
        assert wt[k, j, i] == 0 and wt[k + 1, j, i] == 0
    # the gas side carries the outflow: u~ . r < 0 (liquid inside) on the
    # outermost sub-domain faces is the removed expansion


def test_centred_sphere_is_mirror_symmetric():
    n = 16
    h = 1.0 / n
    c = W.sphere_fractions((n, n, n), h, (0.5, 0.5, 0.5), 0.26, nsub=10)
    mdot = np.where((c > 1e-12) & (c < 1 - 1e-12), 0.03, 0.0)
    g = O.Grid(n, n, n, (0, 0, 0), h, 1.0, 1.0, 1.0)
    ut, vt, wt, layer, p = velocity_extension(g, c, mdot, RHO_L, RHO_G, 1e-3)
    scale = np.abs(ut).max()
    assert scale > 0
    # each component is odd under the mirror of its own axis (faces f and
    # n - f) and even under the mirrors of the other two (cells j, n-1-j)
    for t, ax in ((ut, 2), (vt, 1), (wt, 0)):
        assert np.abs(t + np.flip(t, axis=ax)).max() <= 1e-10 * scale
        for other in {0, 1, 2} - {ax}:
            assert np.abs(t - np.flip(t, axis=other)).max() <= 1e-10 * scale


def test_zero_mass_flux_gives_zero():
    c, mdot, h = sphere_case(n=12)
    g = O.Grid(12, 12, 12, (1, 1, 1), h, 1.0, 1.0, 1.0)
    ut, vt, wt, _, _ = velocity_extension(g, c, 0.0 * mdot, RHO_L, RHO_G, 1e-3)
    assert not ut.any() and not vt.any() and not wt.any()


def test_no_free_flow_face_is_rejected():
    # a periodic box whose every gas cell lies within two layers of the
    # interface: nothing fixes p~
    c = np.zeros((5, 2, 2))
    c[:2] = 1.0
    c[2] = 0.5
    g = O.Grid(2, 2, 5, (0, 0, 0), 0.1, 1.0, 1.0, 1.0)
    with pytest.raises(ValueError):
        velocity_extension(g, c, np.where(c == 0.5, 0.01, 0.0), RHO_L, RHO_G, 1e-3)


def test_layers_follow_faces():
    c = np.zeros((9, 9, 9))
    c[4, 4, 4] = 0.5  # one mixed cell in gas
    g = O.Grid(9, 9, 9, (1, 1, 1), 0.1, 1.0, 1.0, 1.0)
    layer = subdomain_layers(g, c)
    assert np.count_nonzero(layer == 0) == 1
    assert np.count_nonzero(layer == 1) == 6     # face neighbours
    assert np.count_nonzero(layer == 2) == 18    # the octahedron shell |dx|+|dy|+|dz| = 2
