"""Training stencils of the learned normal (workloads.training_stencils),
checked against what fixes them (CPU):

* plane stencils: the chord-integrated fractions are within 1e-3 of the
  exact plane-cut volumes (the oracle's PLIC volume) at 12 x 12 points and
  converge at second order;
* curved stencils: the same fractions as the grid generator
  (ellipsoid_fractions) for the same ellipsoid;
* labels: the nearest points agree with the oracle's scalar bisection, the
  labels are unit vectors pointing from liquid to gas (positive against the
  MYC normal of their stencil);
* any index range is generated alone, the central cell is always mixed,
  and the kinds cycle.
"""
import numpy as np

import oracle as O
import oracle.mlp as M
from paper_2001_03477_gb300 import workloads as W


def test_plane_fractions_match_the_exact_cut():
    rng = np.random.default_rng(3)
    K = 200
    n = rng.normal(size=(K, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    d = rng.uniform(-0.4, 0.4, K) * np.abs(n).sum(axis=1)
    exact = np.array([[O.volume(n[k] / np.abs(n[k]).sum(), (d[k] - n[k] @ (o - 0.5)) / np.abs(n[k]).sum())
                       for o in W._STENCIL] for k in range(K)])
    err = {ns: np.abs(W._plane_fractions(n, d, ns) - exact).max() for ns in (12, 24)}
    # midpoint rule on a chord length that is linear but for its kinks:
    # second order in the sub-cell size
    assert err[12] <= 1e-3 and err[24] <= err[12] / 3.0


def test_curved_fractions_match_the_grid_generator():
    rng = np.random.default_rng(4)
    for kind in ("sphere", "ellipsoid") * 6:
        axes, R, centre, inside = W._curved_params(rng, kind)
        got = W._curved_fractions(axes[None], R[None], centre[None], np.array([inside]), 8)[0]
        want = W.ellipsoid_fractions((3, 3, 3), 1.0, tuple(centre + 1.5), tuple(axes), rot=R, inside=inside, nsub=8)
        assert np.abs(got - want.reshape(27)).max() <= 1e-12


def test_nearest_points_match_the_oracle():
    rng = np.random.default_rng(5)
    axes = np.exp(rng.uniform(0, np.log(50), (100, 3)))
    y = rng.normal(size=(100, 3)) * axes * rng.uniform(0.5, 2.0, (100, 1))
    got = W.nearest_on_ellipsoids(axes, y)
    for k in range(100):
        want = M.ellipsoid_nearest(axes[k], y[k])
        assert np.abs(got[k] - want).max() <= 1e-9 * max(1.0, np.abs(want).max())


def test_labels_and_stencils():
    X, Y = W.training_stencils(300, seed=9)
    assert np.abs(np.linalg.norm(Y, axis=1) - 1.0).max() < 1e-12
    assert ((X[:, 13] > 1e-6) & (X[:, 13] < 1 - 1e-6)).all()
    assert X.min() >= 0.0 and X.max() <= 1.0
    for s, n in zip(X, Y):
        assert O.myc(s.reshape(3, 3, 3)) @ n > 0.0
    X2, Y2 = W.training_stencils(7, seed=9, start=120)
    assert np.array_equal(X2, X[120:127]) and np.array_equal(Y2, Y[120:127])
