"""Pins of the oracle's Lagrangian-explicit sweep (Li's split scheme, the
alternative Step 1 named in Sec. 3.3.1) against what the mathematics fixes
(CPU only).

* Uniform velocity: the stretch J = 1, the preimage of the region beyond a
  face is the Eulerian donor slab, and the sweep is the (independently
  pinned) Weymouth-Yue sweep, whose dilatation terms vanish.
* A velocity linear along the sweep axis maps every point exactly (the
  scheme's own assumption holds everywhere): a plane interface x = x0 moves
  to x0 + a(x0), so every cell's new fraction is known in closed form, for
  compression and expansion and either orientation.
* A uniform temperature stays uniform under any velocity (Sec. 3.4.1).
* Volume: the fluxes telescope, so on a periodic line the total changes by
  sum_i c_i (a_r - a_l)_i (the cells' own stretch) and the clipped volume.
"""
import numpy as np
import pytest

import oracle as O
from paper_2001_03477_gb300 import workloads as W


def random_field(shape, rng):
    c = rng.random(shape)
    c[c < 0.25] = 0.0
    c[c > 0.75] = 1.0
    return c


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_uniform_velocity_equals_weymouth_yue(axis):
    rng = np.random.default_rng(10 + axis)
    n = 12
    h = 1.0 / n
    g = O.Grid(n, n, n, (0, 0, 0), h, 7.0, 1.0, 1.0)
    c = W.ellipsoid_fractions((n, n, n), h, (0.5, 0.45, 0.55), (0.3, 0.2, 0.25),
                              rot=np.linalg.qr(rng.normal(size=(3, 3)))[0], nsub=8)
    T = 1.0 + rng.random(c.shape)
    e = (7.0 * c + (1 - c)) * T
    vel = [0.3, -0.45, 0.6][axis]
    uf = W.uniform_faces((n, n, n), (vel, vel, vel))[axis]
    dt = 0.5 * h
    cc, th = O.frozen(g, c, e)
    cw, ew, _, Fw, _ = O.sweep(g, axis, c, e, uf, dt, cc, th, want_flux=True)
    cl, el, _, Fl, _ = O.sweep_le(g, axis, c, e, uf, dt, want_flux=True)
    assert np.array_equal(Fl, Fw)
    assert np.abs(cl - cw).max() < 1e-15
    assert np.abs(el - ew).max() < 1e-15 * np.abs(ew).max()


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("beta,liquid_low", [(-0.05, True), (0.04, True), (-0.05, False), (0.03, False)])
def test_linear_velocity_moves_a_plane_exactly(axis, beta, liquid_low):
    n, m = 24, 3
    shape = [m, m, m]
    shape[2 - axis] = n
    shape = tuple(shape)
    h, dt = 1.0, 1.0
    xs, x0 = 11.3, 9.6  # velocity node, interface position (cell units)

    def frac(pos):
        k = np.arange(n, dtype=float)
        f = np.clip(pos - k, 0.0, 1.0)
        return f if liquid_low else 1.0 - f

    def along(v):
        sh = [1, 1, 1]
        sh[2 - axis] = n
        return np.broadcast_to(v.reshape(sh), shape).copy()

    c = along(frac(x0))
    fshape = list(shape)
    fshape[2 - axis] += 1
    fx = np.arange(n + 1, dtype=float)
    sh = [1, 1, 1]
    sh[2 - axis] = n + 1
    uf = np.broadcast_to((beta * (fx - xs)).reshape(sh), tuple(fshape)).copy()
    bc = [0, 0, 0]
    bc[axis] = 1
    g = O.Grid(shape[2], shape[1], shape[0], tuple(bc), h, 3.0, 1.0, 1.0)
    e = (3.0 * c + (1 - c)) * 2.0
    c1, e1, clip = O.sweep_le(g, axis, c, e, uf, dt)
    x1 = x0 + beta * (x0 - xs)
    assert np.abs(c1 - along(frac(x1))).max() < 1e-14
    assert clip == 0.0
    # the same uniform T
    T1 = e1 / (3.0 * c1 + (1 - c1))
    assert np.abs(T1 - 2.0).max() < 1e-14


def test_uniform_temperature_stays_uniform():
    rng = np.random.default_rng(3)
    n = 10
    g = O.Grid(n, n, n, (0, 0, 0), 0.1, 3236.3, 1.0, 1.5)
    c = random_field((n, n, n), rng)
    e = (3236.3 * c + (1 - c)) * 1.5
    for axis in range(3):
        uf = 0.3 * rng.uniform(-1, 1, g.face_shape(axis))  # compressive, not divergence free
        c, e, _ = O.sweep_le(g, axis, c, e, uf, 0.1)
    T = e / (3236.3 * c + (1 - c))
    assert np.abs(T - 1.5).max() < 1e-13 * 3236.3


def test_volume_identity_periodic():
    rng = np.random.default_rng(4)
    n = 9
    g = O.Grid(n, n, n, (0, 0, 0), 0.1, 2.0, 1.0, 1.0)
    c = random_field((n, n, n), rng)
    e = (2.0 * c + (1 - c)) * (1 + rng.random(c.shape))
    uf = 0.35 * rng.uniform(-1, 1, g.face_shape(1))
    lam = 0.1 / 0.1
    c1, _, clip = O.sweep_le(g, 1, c, e, uf, 0.1)
    a = uf * lam
    stretch = a[:, 1:, :] - a[:, :-1, :]  # a_r - a_l of every cell (periodic: face n = face 0 is not read)
    stretch[:, -1, :] = a[:, 0, :] - a[:, -2, :]
    want = c.sum() + (c * stretch).sum() - clip
    assert abs(c1.sum() - want) < 1e-12


def test_step_scheme_one_runs_le_sweeps():
    """orc_step_scheme(scheme=1) = three LE sweeps (x, y, z) + the shift."""
    rng = np.random.default_rng(5)
    n = 10
    h = 0.1
    g = O.Grid(n, n, n, (0, 0, 0), h, 4.0, 1.0, 1.0)
    c = W.sphere_fractions((n, n, n), h, (0.5, 0.5, 0.5), 0.3, nsub=8)
    e = (4.0 * c + (1 - c)) * (1 + 0.1 * rng.random(c.shape))
    u, v, w = (0.2 * rng.uniform(-1, 1, g.face_shape(a)) for a in range(3))
    c2, e2, _ = O.step(g, c, e, u, v, w, 0.05, 0, dd_uniform=-0.01, scheme=1)
    cs, es = c, e
    for axis, uf in zip(range(3), (u, v, w)):
        cs, es, _ = O.sweep_le(g, axis, cs, es, uf, 0.05)
    cs, es, _ = O.phase_shift(g, cs, es, dd_uniform=-0.01)
    assert np.array_equal(c2, cs) and np.array_equal(e2, es)
