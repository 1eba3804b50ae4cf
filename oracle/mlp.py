"""Learned interface normal (the learned-normal form: a small MLP maps the
27 volume fractions of a 3 x 3 x 3 stencil to the interface normal, with the
MYC normal as fallback): FP64 CPU oracle of its data, network, gradients and
fallback rule.

TEST INFRASTRUCTURE ONLY: plain numpy; only the test suite, the package
smoke check and the benchmark's CPU-baseline leg may use it.  It shares no
code with a GPU path.

Pieces:
  * training stencils from analytic surfaces -- spheres (radius log-uniform
    in [1, 50] cells), ellipsoids (semi-axes log-uniform in [1, 50]) and
    planes, random orientation and sub-cell offset; input the 27 volume
    fractions (chord integration for spheres and ellipsoids, the exact plane
    cut for planes), label the unit normal, liquid -> gas, at the surface
    point nearest the central cell's centre (for an ellipsoid found from the
    stationarity condition of the distance, solved by bisection);
  * the network 27 -> 64 -> 64 -> 3 with GELU (x Phi(x), exact), inputs
    2 c - 1, output direction y / |y|; loss the mean squared distance of
    the unit vectors; its exact gradient by the chain rule; Adam;
  * BF16 weights: round-to-nearest-even of the FP32 pattern to its upper 16
    bits, the rest of the arithmetic in FP64 (the accumulation the GPU does
    in FP32 is bounded by the FP64 result);
  * fallback: the plane through the central cell with a normal
    (L1-normalised, plane constant from the central c) is tested on the 26
    neighbours by the RMS of (its volume in each neighbour - c), the plane
    residual.  The predicted normal is replaced by the MYC normal when its
    residual exceeds 1.25 x MYC's own residual + 1e-3.  Reading: a fixed
    bound of 1e-3 alone would reject the exact normal itself on nearly every
    curved stencil (the residual of any plane there is dominated by the
    curvature: median about 0.06 over radii of 1-50 cells), leaving the
    network active only on planes, where MYC is already exact; measured
    against MYC's residual the bound still reduces to 1e-3 where MYC's plane
    fits the stencil exactly, accepts the exact normal on curved stencils and
    rejects most normals tens of degrees off.
"""
from __future__ import annotations

import math

import numpy as np

from . import alpha, myc, volume

# ---------------------------------------------------------------------------
# data
# ---------------------------------------------------------------------------


def _rotation(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def _offsets():
    return np.array([[dx, dy, dz] for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)], dtype=float)


def ellipsoid_nearest(axes, y):
    """Point of the ellipsoid sum x_i^2 / a_i^2 = 1 (principal frame) nearest
    to y: x_i = a_i^2 y_i / (a_i^2 + t) with t solving sum (a_i y_i /
    (a_i^2 + t))^2 = 1, found by bisection (the sum decreases in t on the
    branch t > -min a_i^2)."""
    a2 = np.asarray(axes, dtype=float) ** 2
    y = np.asarray(y, dtype=float)
    f = lambda t: float(np.sum(a2 * y * y / (a2 + t) ** 2)) - 1.0
    lo = -a2.min() + 1e-12 * a2.min()
    hi = float(np.sqrt(a2).max() * np.abs(y).max() * 2.0 + a2.max())
    while f(hi) > 0:
        hi *= 2.0
    if f(lo) < 0:  # y is the centre direction degenerate: take lo
        t = lo
    else:
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if f(mid) > 0:
                lo = mid
            else:
                hi = mid
        t = 0.5 * (lo + hi)
    return a2 * y / (a2 + t)


def plane_stencil(n, d):
    """27 exact volume fractions of {x : n . x <= d} (x relative to the
    central cell's centre, cell units, n a unit normal liquid -> gas)."""
    m = n / np.abs(n).sum()
    l1 = np.abs(n).sum()
    s = np.zeros(27)
    for k, o in enumerate(_offsets()):
        # cell with centre o: local x' = x - (o - 1/2), m . x' <= (d - n . (o - 1/2)) / |n|_1
        a = (d - n @ (o - 0.5)) / l1
        s[k] = volume(m, a)
    return s


def surface_stencil(kind, rng, nsub=12):
    """(s[27], unit normal liquid -> gas) for a random surface of `kind`
    ('sphere', 'ellipsoid', 'plane') crossing the central cell."""
    from paper_2001_03477_gb300 import workloads as W
    for _ in range(1000):
        if kind == "plane":
            n = rng.normal(size=3)
            n /= np.linalg.norm(n)
            d = rng.uniform(-0.4, 0.4) * np.abs(n).sum()
            s = plane_stencil(n, d)
            label = n
        else:
            if kind == "sphere":
                axes = np.full(3, math.exp(rng.uniform(0.0, math.log(50.0))))
            else:
                axes = np.exp(rng.uniform(0.0, math.log(50.0), 3))
            R = _rotation(rng)
            # a surface point near the central cell's centre: a random
            # direction on the ellipsoid, shifted so that it lands near the
            # origin, plus a sub-cell offset
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            p_local = u / np.sqrt(np.sum(u * u / axes ** 2))   # on the surface
            centre = -(R @ p_local) + rng.uniform(-0.5, 0.5, 3)
            inside = 1.0 if rng.random() < 0.5 else 0.0
            # fractions of the 3x3x3 block around the origin: cells of size 1
            # with the block's low corner at (-1.5, -1.5, -1.5)
            c = W.ellipsoid_fractions((3, 3, 3), 1.0, tuple(centre + 1.5), tuple(axes), rot=R, inside=inside,
                                      nsub=nsub)
            s = c.reshape(27)
            y = R.T @ (-centre)  # the central cell's centre in the principal frame
            xn = ellipsoid_nearest(axes, y)
            gradq = R @ (xn / axes ** 2)  # outward normal direction
            nrm = gradq / np.linalg.norm(gradq)
            label = nrm if inside == 1.0 else -nrm  # liquid -> gas
        if 1e-6 < s[13] < 1 - 1e-6:
            return s, label
    raise RuntimeError("no stencil with a mixed central cell")


def dataset(n, rng, kinds=("sphere", "ellipsoid", "plane")):
    X = np.zeros((n, 27))
    Y = np.zeros((n, 3))
    for i in range(n):
        X[i], Y[i] = surface_stencil(kinds[i % len(kinds)], rng)
    return X, Y


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------

SIZES = (27, 64, 64, 3)


def gelu(x):
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def init_params(rng):
    p = {}
    for k, (a, b) in enumerate(zip(SIZES[:-1], SIZES[1:]), start=1):
        p[f"W{k}"] = rng.normal(0.0, math.sqrt(2.0 / a), size=(b, a))
        p[f"b{k}"] = np.zeros(b)
    return p


def bf16(x):
    """Round to BF16 (nearest even on the FP32 pattern's upper 16 bits),
    returned as FP64."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(nan, np.nan, out)


def forward(p, X, weights=lambda w: w):
    """Returns (y, cache); X: (B, 27) volume fractions."""
    a0 = 2.0 * X - 1.0
    z1 = a0 @ weights(p["W1"]).T + p["b1"]
    a1 = gelu(z1)
    z2 = a1 @ weights(p["W2"]).T + p["b2"]
    a2 = gelu(z2)
    y = a2 @ weights(p["W3"]).T + p["b3"]
    return y, (a0, z1, a1, z2, a2)


def loss_and_grad(p, X, N):
    """Mean squared distance of the predicted unit normals from the labels
    N, and its gradient with respect to every parameter."""
    y, (a0, z1, a1, z2, a2) = forward(p, X)
    B = X.shape[0]
    ny = np.linalg.norm(y, axis=1, keepdims=True)
    yh = y / ny
    diff = yh - N
    loss = float(np.sum(diff * diff) / B)
    g_yh = 2.0 * diff / B
    # d yh / d y = (I - yh yh^T) / |y|
    g_y = (g_yh - yh * np.sum(g_yh * yh, axis=1, keepdims=True)) / ny
    g = {}
    g["W3"] = g_y.T @ a2
    g["b3"] = g_y.sum(axis=0)
    g_a2 = g_y @ p["W3"]
    g_z2 = g_a2 * gelu_grad(z2)
    g["W2"] = g_z2.T @ a1
    g["b2"] = g_z2.sum(axis=0)
    g_a1 = g_z2 @ p["W2"]
    g_z1 = g_a1 * gelu_grad(z1)
    g["W1"] = g_z1.T @ a0
    g["b1"] = g_z1.sum(axis=0)
    return loss, g


def adam(p, X, N, steps, lr=1e-3, batch=256, rng=None, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam on mini-batches; returns the loss of every step."""
    rng = rng or np.random.default_rng(0)
    mom = {k: np.zeros_like(v) for k, v in p.items()}
    vel = {k: np.zeros_like(v) for k, v in p.items()}
    hist = []
    for t in range(1, steps + 1):
        idx = rng.integers(0, X.shape[0], size=min(batch, X.shape[0]))
        loss, g = loss_and_grad(p, X[idx], N[idx])
        hist.append(loss)
        for k in p:
            mom[k] = beta1 * mom[k] + (1 - beta1) * g[k]
            vel[k] = beta2 * vel[k] + (1 - beta2) * g[k] * g[k]
            mh = mom[k] / (1 - beta1 ** t)
            vh = vel[k] / (1 - beta2 ** t)
            p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return hist


# ---------------------------------------------------------------------------
# normal with fallback
# ---------------------------------------------------------------------------


def plane_residual(s, m):
    """RMS over the 26 neighbours of (volume of the plane with normal m
    through the central cell's plane constant) - c."""
    s = np.asarray(s, dtype=float).reshape(27)
    mm = np.asarray(m, dtype=float)
    mm = mm / np.abs(mm).sum()
    al = alpha(mm, s[13])
    r = []
    for k, o in enumerate(_offsets()):
        if k == 13:
            continue
        r.append(volume(mm, al - mm @ o) - s[k])
    return math.sqrt(float(np.mean(np.square(r))))


FALLBACK_RATIO = 1.25
FALLBACK_TOL = 1e-3


def accept_bound(s):
    """The largest plane residual a predicted normal may have on stencil s:
    FALLBACK_RATIO x the MYC normal's residual + FALLBACK_TOL."""
    return FALLBACK_RATIO * plane_residual(s, myc(np.asarray(s).reshape(3, 3, 3))) + FALLBACK_TOL


def learned_normal(p, s, weights=bf16):
    """(m L1-normalised liquid -> gas, used_fallback): the network's normal
    unless its plane residual exceeds accept_bound(s), else MYC."""
    y, _ = forward(p, np.asarray(s, dtype=float).reshape(1, 27), weights)
    m = y[0] / np.abs(y[0]).sum()
    if plane_residual(s, m) > accept_bound(s):
        return myc(np.asarray(s).reshape(3, 3, 3)), True
    return m, False
