"""Input generators (no method arithmetic): the seeded smooth temperature
field and the deformation workload of the precision-form comparison."""
import math

import numpy as np

from paper_2001_03477_gb300 import workloads as W


def test_fourier_field_is_its_modal_sum():
    n = 16
    T = W.fourier_field((n, n, n), 1.0 / n, seed=7)
    # the same seeded draws, summed mode by mode on the cell centres
    rng = np.random.default_rng(7)
    ks = rng.integers(-3, 4, size=(8, 3))
    ks[np.all(ks == 0, axis=1), 0] = 1
    amps = 0.1 * rng.uniform(0.5, 1.0, 8) / 8
    phis = rng.uniform(0.0, 2 * np.pi, 8)
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    direct = 1.0 + sum(amps[m] * np.sin(2 * np.pi * (ks[m, 0] * X + ks[m, 1] * Y + ks[m, 2] * Z) + phis[m])
                       for m in range(8))
    assert np.abs(T - direct).max() < 1e-14
    # every mode has a nonzero wave vector below the Nyquist limit: the
    # midpoint mean over the periodic box is exactly 1
    assert abs(T.mean() - 1.0) < 1e-14
    assert np.abs(T - 1.0).max() <= 0.1


def test_deformation_sphere_workload():
    n = 48
    wl = W.deformation_sphere(n=n, nsub=8)
    assert wl.shape == (n, n, n) and wl.dd_uniform == 0.0
    # the sphere's volume in cells, to the midpoint rule's accuracy
    assert abs(wl.c.sum() / (4.0 / 3.0 * math.pi * 0.15 ** 3 * n ** 3) - 1.0) < 1e-3
    # exact face averages of a divergence-free field: every cell's net
    # outflow vanishes to round-off, and nothing crosses the boundary
    div = (np.diff(wl.u, axis=2) + np.diff(wl.v, axis=1) + np.diff(wl.w, axis=0))
    assert np.abs(div).max() < 1e-14
    assert np.abs(wl.u[:, :, [0, -1]]).max() < 1e-15
    # face CFL 0.5 at the fastest face
    assert abs(np.abs(wl.u).max() * wl.dt / wl.h - 0.5) < 0.01
    T = wl.e / (wl.Cp_l * wl.c + wl.Cp_g * (1 - wl.c))
    assert np.abs(T - W.fourier_field((n, n, n), wl.h, seed=3)).max() < 1e-12
