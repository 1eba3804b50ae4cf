"""Pins of the learned-normal oracle (oracle/mlp.py): data, network,
gradients and the MYC fallback, against what the mathematics fixes (CPU).

* The analytic gradient of the loss equals central finite differences.
* GELU: x Phi(x) satisfies gelu(x) - gelu(-x) = x, and its derivative
  equals finite differences.
* BF16 rounding equals a library conversion (torch's bfloat16), ties to even.
* Labels: the nearest point of an ellipsoid lies on it with the offset along
  the surface normal; for equal axes it is the radial projection; every
  label points from liquid to gas like the MYC normal of its stencil.
* Plane residual: zero for a plane stencil and its own normal, above the
  1e-3 fallback threshold for a normal 5 degrees off; an untrained network
  therefore falls back to MYC on planes.
* Fallback bound (1.25 x MYC's residual + 1e-3): a fixed 1e-3 alone rejects
  the exact normal on nearly every curved stencil; the bound accepts the
  exact normal on curved stencils, rejects most normals 45 degrees off, and
  keeps MYC's exact plane wherever MYC fits a plane stencil exactly.
* Adam on a few hundred stencils lowers the loss several-fold.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.mlp as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    X, Y = M.dataset(24, rng)
    p = M.init_params(rng)
    _, g = M.loss_and_grad(p, X, Y)
    eps = 1e-6
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            q = {a: b.copy() for a, b in p.items()}
            q[k][idx] += eps
            lp, _ = M.loss_and_grad(q, X, Y)
            q[k][idx] -= 2 * eps
            lm, _ = M.loss_and_grad(q, X, Y)
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[k][idx]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9


def test_gelu_identities():
    x = np.linspace(-6, 6, 241)
    assert np.abs(M.gelu(x) - M.gelu(-x) - x).max() < 1e-14
    assert M.gelu(np.array([0.0]))[0] == 0.0
    h = 1e-6
    fd = (M.gelu(x + h) - M.gelu(x - h)) / (2 * h)
    assert np.abs(fd - M.gelu_grad(x)).max() < 1e-8


def test_bf16_matches_library_rounding():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-30, 30, 2000),
                        1.0 + np.arange(1, 512) * 2.0 ** -16,       # ties and near ties
                        -(1.0 + np.arange(1, 512) * 2.0 ** -16), [0.0, -0.0, 1e-40]])
    # exact ties (the dropped 16 bits are 0x8000) above both even and odd
    # upper halves, so that round-to-even is told apart from any fixed rule
    upper = rng.integers(0x0080, 0x7F00, size=1000).astype(np.uint32)
    ties = ((upper << 16) | 0x8000).view(np.float32).astype(np.float64)
    assert (upper & 1).any() and not (upper & 1).all()
    x = np.concatenate([x, ties, -ties])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    assert np.array_equal(M.bf16(x), want)


def test_ellipsoid_nearest_point():
    rng = np.random.default_rng(3)
    for _ in range(200):
        axes = np.exp(rng.uniform(0, math.log(50), 3))
        y = rng.normal(size=3) * axes * rng.uniform(0.5, 2.0)
        x = M.ellipsoid_nearest(axes, y)
        assert abs(np.sum(x * x / axes ** 2) - 1.0) < 1e-10
        gq = x / axes ** 2
        r = y - x
        assert np.linalg.norm(np.cross(r, gq)) <= 1e-8 * max(1.0, np.linalg.norm(r)) * np.linalg.norm(gq)
    a = np.full(3, 7.0)
    y = np.array([3.0, -2.0, 9.0])
    assert np.abs(M.ellipsoid_nearest(a, y) - 7.0 * y / np.linalg.norm(y)).max() < 1e-10


@pytest.mark.parametrize("kind", ["sphere", "ellipsoid", "plane"])
def test_labels_point_liquid_to_gas(kind):
    rng = np.random.default_rng(4)
    for _ in range(40):
        s, n = M.surface_stencil(kind, rng)
        assert abs(np.linalg.norm(n) - 1.0) < 1e-12
        m = O.myc(s.reshape(3, 3, 3))
        assert m @ n > 0.0


def test_plane_residual_and_fallback():
    rng = np.random.default_rng(5)
    p = M.init_params(rng)  # untrained: far from any plane's normal
    nfall = 0
    for _ in range(30):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        s = M.plane_stencil(n, rng.uniform(-0.3, 0.3) * np.abs(n).sum())
        if not 1e-6 < s[13] < 1 - 1e-6:
            continue
        assert M.plane_residual(s, n) < 1e-13
        # 5 degrees off
        axis = np.cross(n, rng.normal(size=3))
        axis /= np.linalg.norm(axis)
        ang = math.radians(5.0)
        n5 = n * math.cos(ang) + np.cross(axis, n) * math.sin(ang)
        assert M.plane_residual(s, n5) > 1e-3
        m, fell = M.learned_normal(p, s)
        if fell:
            nfall += 1
            assert np.array_equal(m, O.myc(s.reshape(3, 3, 3)))
    assert nfall >= 20


def test_training_lowers_the_loss():
    rng = np.random.default_rng(6)
    X, Y = M.dataset(600, rng)
    p = M.init_params(rng)
    l0, _ = M.loss_and_grad(p, X, Y)
    hist = M.adam(p, X, Y, steps=300, lr=3e-3, batch=128, rng=rng)
    l1, _ = M.loss_and_grad(p, X, Y)
    assert l1 < 0.2 * l0
    assert hist[-1] < hist[0]


def _tilted(n, deg, rng):
    axis = np.cross(n, rng.normal(size=3))
    axis /= np.linalg.norm(axis)
    a = math.radians(deg)
    return n * math.cos(a) + np.cross(axis, n) * math.sin(a)


def test_fallback_bound_on_curved_stencils():
    rng = np.random.default_rng(7)
    X, Y = M.dataset(240, rng, kinds=("sphere", "ellipsoid"))
    over_fixed = accepted_exact = accepted_far = 0
    for s, n in zip(X, Y):
        r_exact = M.plane_residual(s, n)
        over_fixed += r_exact > 1e-3
        bound = M.accept_bound(s)
        accepted_exact += r_exact <= bound
        accepted_far += M.plane_residual(s, _tilted(n, 45.0, rng)) <= bound
    N = len(X)
    assert over_fixed >= 0.95 * N      # a fixed 1e-3 would reject the exact normal
    assert accepted_exact >= 0.98 * N  # the bound keeps it
    assert accepted_far <= 0.10 * N    # and rejects most normals 45 degrees off


def test_fallback_keeps_myc_where_it_is_exact():
    rng = np.random.default_rng(8)
    p = M.init_params(rng)
    checked = 0
    for _ in range(60):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        s = M.plane_stencil(n, rng.uniform(-0.3, 0.3) * np.abs(n).sum())
        if not 1e-6 < s[13] < 1 - 1e-6:
            continue
        m_myc = O.myc(s.reshape(3, 3, 3))
        if M.plane_residual(s, m_myc) > 1e-13:
            continue  # MYC is exact only where the columns span the plane
        checked += 1
        assert M.plane_residual(s, _tilted(n, 0.5, rng)) > M.accept_bound(s)
        # a network whose output is that slightly tilted normal falls back
        q = {k: v.copy() for k, v in p.items()}
        q["W3"][:] = 0.0
        q["b3"][:] = _tilted(n, 0.5, rng)
        m, fell = M.learned_normal(q, s, weights=lambda w: w)
        assert fell and np.array_equal(m, m_myc)
    assert checked >= 15


def test_adam_first_step_closed_form():
    # Adam (Kingma & Ba) with bias-corrected moments: after one step the
    # corrected first moment is g and the second g^2, so every parameter
    # moves by -lr g / (|g| + eps).  All rows of the batch are one stencil,
    # so the sampled mini-batch's gradient is the full gradient.
    rng = np.random.default_rng(7)
    X1, N1 = M.dataset(1, rng)
    X, N = np.repeat(X1, 32, axis=0), np.repeat(N1, 32, axis=0)
    p0 = M.init_params(np.random.default_rng(8))
    _, g = M.loss_and_grad(p0, X, N)
    p = {k: v.copy() for k, v in p0.items()}
    lr, eps = 1e-3, 1e-8
    M.adam(p, X, N, 1, lr=lr, batch=16, rng=np.random.default_rng(9), eps=eps)
    for k in p:
        want = p0[k] - lr * g[k] / (np.abs(g[k]) + eps)
        assert np.allclose(p[k], want, rtol=1e-12, atol=1e-15), k
