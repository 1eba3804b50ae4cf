"""Seeded synthetic inputs shaped like the paper's validation cases.

This module only builds initial data (volume fractions of analytic shapes,
temperature fields, face velocities).  It contains none of the method's
arithmetic: no interface normal, no plane constant, no flux.  Volume
fractions are obtained by integrating chord lengths of the analytic shape
through each cell on an n x n midpoint rule, so they depend only on the
shape, not on any PLIC routine.

Cases (Sec. 4 of Malan et al.):
  * translating sphere with T = 1 in the liquid (periodic box),
  * vapour bubble in superheated liquid (Sec. 4.4), radial liquid velocity
    built from exact face solid angles (discretely divergence free),
  * deformation field (LeVeque) with exact face averages,
  * many small periodic droplet boxes (batched form),
  * training stencils of the learned normal: 3 x 3 x 3 fractions around
    spheres, ellipsoids and planes with the unit normal at the nearest
    surface point as label.

Water / steam data are those of Table atm_water (Sec. 4.3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Table atm_water: saturated water at 1 atm
RHO_L, RHO_G = 958.0, 0.6
CP_L_SPEC, CP_G_SPEC = 4216.0, 2080.0
H_FG_WATER = 2.257e6  # J/kg, not printed in the paper; reproduces delta(10 s)
T_SAT_WATER = 373.15


# ---------------------------------------------------------------------------
# Volume fractions of analytic shapes by chord integration
# ---------------------------------------------------------------------------

def _chord_fraction(lo_x, hi_x, ys, zs, chord_fn):
    """Mean over (y,z) points of the length of {x in [lo_x,hi_x]} inside the
    shape divided by (hi_x - lo_x).  chord_fn(y, z) -> (x0, x1) interval
    (x0 > x1 when empty).  Arrays broadcast over cells."""
    x0, x1 = chord_fn(ys, zs)
    a = np.maximum(x0, lo_x[..., None, None])
    b = np.minimum(x1, hi_x[..., None, None])
    ln = np.clip(b - a, 0.0, None)
    return ln.mean(axis=(-1, -2)) / (hi_x - lo_x)


def ellipsoid_fractions(shape, h, centre, axes, rot=None, inside=1.0, nsub=32, chunk=4096):
    """Volume fraction of the ellipsoid {(R^T (x - c))_i^2 / a_i^2 <= 1} in
    each cell of a grid with cell size h (tuple or scalar), shape (nz,ny,nx).
    inside=1 gives liquid inside; inside=0 gives the complement."""
    nz, ny, nx = shape
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    c = np.asarray(centre, dtype=np.float64)
    ax = np.asarray(axes, dtype=np.float64)
    R = np.eye(3) if rot is None else np.asarray(rot, dtype=np.float64)
    # quadratic form Q = R diag(1/a^2) R^T
    Q = R @ np.diag(1.0 / ax ** 2) @ R.T
    rmax = ax.max()
    rmin = ax.min()
    zc = (np.arange(nz) + 0.5) * hz
    yc = (np.arange(ny) + 0.5) * hy
    xc = (np.arange(nx) + 0.5) * hx
    # classify by distance of the cell centre (conservative bounds), one
    # z-plane at a time (large grids would not fit the temporaries)
    half_diag = 0.5 * math.sqrt(hx * hx + hy * hy + hz * hz)
    Y, X = np.meshgrid(yc, xc, indexing="ij")
    frac = np.empty((nz, ny, nx))
    idx = []
    for k in range(nz):
        d = np.stack([X - c[0], Y - c[1], np.full_like(X, zc[k] - c[2])], axis=-1)
        qv = np.einsum("...i,ij,...j->...", d, Q, d)
        dist = np.sqrt(np.einsum("...i,...i->...", d, d))
        frac[k] = qv <= 1.0
        # cells that can intersect the surface: inside the outer shell,
        # outside the inner one
        cand = (dist <= rmax + half_diag) & ~(dist < rmin - half_diag)
        jj, ii = np.nonzero(cand)
        if len(jj):
            idx.append(np.stack([np.full_like(jj, k), jj, ii], axis=1))
    # exact classification of candidates by sub-integration
    idx = np.concatenate(idx) if idx else np.zeros((0, 3), dtype=np.int64)
    t = (np.arange(nsub) + 0.5) / nsub
    qxx, qxy, qxz, qyy, qyz, qzz = Q[0, 0], Q[0, 1], Q[0, 2], Q[1, 1], Q[1, 2], Q[2, 2]

    def chord(ys, zs):
        # solve qxx x^2 + 2 x (qxy y + qxz z) + (qyy y^2 + 2 qyz y z + qzz z^2 - 1) = 0 in local coords
        b = qxy * ys + qxz * zs
        cc = qyy * ys * ys + 2.0 * qyz * ys * zs + qzz * zs * zs - 1.0
        disc = b * b - qxx * cc
        sq = np.sqrt(np.clip(disc, 0.0, None))
        x0 = (-b - sq) / qxx
        x1 = (-b + sq) / qxx
        empty = disc < 0.0
        x0 = np.where(empty, 1.0, x0)
        x1 = np.where(empty, 0.0, x1)
        return x0 + c[0], x1 + c[0]

    for s in range(0, len(idx), chunk):
        blk = idx[s:s + chunk]
        k, j, i = blk[:, 0], blk[:, 1], blk[:, 2]
        lo_x = i * hx
        hi_x = (i + 1) * hx
        ys = (j[:, None, None] + t[None, :, None]) * hy - c[1]
        zs = (k[:, None, None] + t[None, None, :]) * hz - c[2]
        ys, zs = np.broadcast_arrays(ys, zs)
        frac[k, j, i] = np.clip(_chord_fraction(lo_x, hi_x, ys, zs, chord), 0.0, 1.0)
    if inside == 0.0:
        np.subtract(1.0, frac, out=frac)
    return frac


def sphere_fractions(shape, h, centre, radius, inside=1.0, nsub=32):
    return ellipsoid_fractions(shape, h, centre, (radius, radius, radius), inside=inside, nsub=nsub)


# ---------------------------------------------------------------------------
# Face velocities
# ---------------------------------------------------------------------------

def uniform_faces(shape, vel):
    nz, ny, nx = shape
    u = np.full((nz, ny, nx + 1), float(vel[0]))
    v = np.full((nz, ny + 1, nx), float(vel[1]))
    w = np.full((nz + 1, ny, nx), float(vel[2]))
    return u, v, w


def _solid_angle_tri(r1, r2, r3):
    """Signed solid angle of triangle (r1,r2,r3) seen from the origin
    (Van Oosterom & Strackee 1983)."""
    l1 = np.linalg.norm(r1, axis=-1)
    l2 = np.linalg.norm(r2, axis=-1)
    l3 = np.linalg.norm(r3, axis=-1)
    num = np.einsum("...i,...i->...", r1, np.cross(r2, r3))
    den = (l1 * l2 * l3 + np.einsum("...i,...i->...", r1, r2) * l3
           + np.einsum("...i,...i->...", r1, r3) * l2 + np.einsum("...i,...i->...", r2, r3) * l1)
    return 2.0 * np.arctan2(num, den)


def radial_faces(shape, h, centre, strength, r_cut):
    """Face-normal velocities of the source field strength * r_hat / r^2
    about `centre`: each face gets strength * Omega / h^2 with Omega the
    exact signed solid angle of the face (oriented along +axis).  Faces whose
    centre lies closer than r_cut get 0 (deep inside the vapour, where the
    field is irrelevant).  Cells away from the cut are divergence free to
    round-off."""
    nz, ny, nx = shape
    c = np.asarray(centre, dtype=np.float64)
    out = []
    # a centred source in a cubic box: y and z faces are the x faces with
    # the axes permuted (same solid angles), so compute x faces only
    sym = (nx == ny == nz) and np.allclose(c, c[0]) and abs(c[0] - 0.5 * nx * h) < 1e-15
    for axis in range(1 if sym else 3):
        fs = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][axis]
        e1 = np.zeros(3); e2 = np.zeros(3)
        t1, t2 = [(1, 2), (2, 0), (0, 1)][axis]  # right-handed: t1 x t2 = +axis
        e1[t1] = h; e2[t2] = h
        vel = np.empty(fs)
        for k0 in range(0, fs[0], 8):  # a few z-planes at a time (bounded temporaries)
            k1 = min(k0 + 8, fs[0])
            kk, jj, ii = np.meshgrid(np.arange(k0, k1), np.arange(fs[1]), np.arange(fs[2]), indexing="ij")
            # low corner of the face in physical coordinates
            base = np.stack([ii * h, jj * h, kk * h], axis=-1) - c
            p0 = base
            p1 = base + e1
            p2 = base + e1 + e2
            p3 = base + e2
            om = _solid_angle_tri(p0, p1, p2) + _solid_angle_tri(p0, p2, p3)
            fc = base + 0.5 * (e1 + e2)
            rc = np.linalg.norm(fc, axis=-1)
            v_ = strength * om / (h * h)
            vel[k0:k1] = np.where(rc < r_cut, 0.0, v_)
        out.append(vel)
    if sym:
        u = out[0]
        out.append(np.ascontiguousarray(np.swapaxes(u, 1, 2)))   # v[k][f][i] = u[k][i][f]
        out.append(np.ascontiguousarray(np.transpose(u, (2, 1, 0))))  # w[f][j][i] = u[i][j][f]
    return tuple(out)


def deformation_faces(shape, h, t, period=3.0):
    """Exact face averages of the LeVeque (1996) deformation field
       u =  2 sin^2(pi x) sin(2 pi y) sin(2 pi z) g(t)
       v = -sin(2 pi x) sin^2(pi y) sin(2 pi z) g(t)
       w = -sin(2 pi x) sin(2 pi y) sin^2(pi z) g(t),  g = cos(pi t / T)
    on a grid of cell size h over [0, n h]."""
    nz, ny, nx = shape
    g = math.cos(math.pi * t / period)

    def avg_sin2pi(n):  # average of sin(2 pi s) over each cell [i h, (i+1) h]
        lo = np.arange(n) * h
        return (np.cos(2 * np.pi * lo) - np.cos(2 * np.pi * (lo + h))) / (2 * np.pi * h)

    def avg_sin2(n):  # average of sin^2(pi s) = 1/2 - cos(2 pi s)/2
        lo = np.arange(n) * h
        return 0.5 - (np.sin(2 * np.pi * (lo + h)) - np.sin(2 * np.pi * lo)) / (4 * np.pi * h)

    xf = np.arange(nx + 1) * h
    yf = np.arange(ny + 1) * h
    zf = np.arange(nz + 1) * h
    u = 2.0 * g * (np.sin(np.pi * xf) ** 2)[None, None, :] * avg_sin2pi(ny)[None, :, None] * avg_sin2pi(nz)[:, None, None]
    v = -g * avg_sin2pi(nx)[None, None, :] * (np.sin(np.pi * yf) ** 2)[None, :, None] * avg_sin2pi(nz)[:, None, None]
    w = -g * avg_sin2pi(nx)[None, None, :] * avg_sin2pi(ny)[None, :, None] * (np.sin(np.pi * zf) ** 2)[:, None, None]
    return (np.ascontiguousarray(u), np.ascontiguousarray(v), np.ascontiguousarray(w))


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    shape: tuple          # (nz, ny, nx)
    bc: tuple             # per axis (x, y, z): 0 periodic, 1 zero-gradient
    h: float
    Cp_l: float
    Cp_g: float
    T_sat: float
    dt: float
    nsteps: int
    dd_uniform: float
    c: np.ndarray
    e: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    eps: float = 1e-12

    @property
    def cells(self):
        return int(np.prod(self.shape))


def translating_sphere(n=32, nsteps=64, dd=-0.01, nsub=32):
    """Sphere R=0.2 at (0.4,0.4,0.4) in the periodic unit box, velocity
    (1, 0.5, 0.25) at CFL 0.25 (dt = 0.25 h), T = 1 in the liquid and 0 in
    the gas, volumetric heat capacity ratio 1000:1, radial shift dd cells per
    step (negative: evaporation)."""
    h = 1.0 / n
    shape = (n, n, n)
    c = sphere_fractions(shape, h, (0.4, 0.4, 0.4), 0.2, nsub=nsub)
    Cp_l, Cp_g = 1000.0, 1.0
    e = c * Cp_l * 1.0
    u, v, w = uniform_faces(shape, (1.0, 0.5, 0.25))
    dt = 0.25 * h
    return Workload("translating-sphere-%d^3" % n, shape, (0, 0, 0), h, Cp_l, Cp_g, 1.0, dt, nsteps, dd, c, e, u, v, w)


def bubble_growth(n=256, nsteps=500, R0=0.1, delta=0.02, Ja=0.5, cells_per_step=0.02, nsub=16):
    """Vapour bubble R0 at the centre of the unit box (liquid outside,
    zero-gradient faces), water/steam properties of Table atm_water.
    T = T_sat in the vapour and T_sat + dT erf((r-R0)/delta) in the liquid,
    dT = Ja rho_g h_fg / (rho_l c_pl).  Radial liquid velocity
    (1 - rho_g/rho_l) Rdot (R0/r)^2 from face solid angles, Rdot such that
    the interface moves `cells_per_step` cells per step; Step 2 shift
    dd = -(rho_g/rho_l) Rdot dt / h."""
    h = 1.0 / n
    shape = (n, n, n)
    centre = (0.5, 0.5, 0.5)
    c = sphere_fractions(shape, h, centre, R0, inside=0.0, nsub=nsub)
    Cp_l = RHO_L * CP_L_SPEC
    Cp_g = RHO_G * CP_G_SPEC
    dT = Ja * RHO_G * H_FG_WATER / (RHO_L * CP_L_SPEC)
    zc = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(zc, zc, zc, indexing="ij")
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    from scipy.special import erf
    T = np.where(r > R0, T_SAT_WATER + dT * erf((r - R0) / delta), T_SAT_WATER)
    e = (Cp_l * c + Cp_g * (1.0 - c)) * T
    dt = 1.0e-3
    Rdot = cells_per_step * h / dt
    A = (1.0 - RHO_G / RHO_L) * Rdot * R0 * R0
    u, v, w = radial_faces(shape, h, centre, A, 0.5 * R0)
    dd = -(RHO_G / RHO_L) * Rdot * dt / h
    return Workload("bubble-growth-%d^3" % n, shape, (1, 1, 1), h, Cp_l, Cp_g, T_SAT_WATER, dt, nsteps, dd,
                    c, e, u, v, w)


def fourier_field(shape, h, nmodes=8, amp=0.1, kmax=3, seed=0):
    """1 + sum of `nmodes` seeded modes amp_m sin(2 pi k_m . x + phi_m) with
    integer wave vectors |k_i| <= kmax (smooth, periodic on the unit box),
    evaluated as one matrix product of separable complex exponentials."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    ks = rng.integers(-kmax, kmax + 1, size=(nmodes, 3))
    ks[np.all(ks == 0, axis=1), 0] = 1
    amps = amp * rng.uniform(0.5, 1.0, nmodes) / nmodes
    phis = rng.uniform(0.0, 2 * np.pi, nmodes)
    xs = (np.arange(nx) + 0.5) * h
    ys = (np.arange(ny) + 0.5) * h
    zs = (np.arange(nz) + 0.5) * h
    exs = [np.exp(2j * np.pi * k[0] * xs) for k in ks]
    # T[z] = 1 + sum_m sin(t_m(z)) Re(E_m) + cos(t_m(z)) Im(E_m) with
    # E_m = a_m exp(2 pi i (k_y y + k_x x)), t_m(z) = 2 pi k_z z + phi_m:
    # one (nz x 2M) by (2M x ny nx) product
    B = np.empty((2 * nmodes, ny * nx))
    A = np.empty((nz, 2 * nmodes))
    for m, k in enumerate(ks):
        E = amps[m] * np.outer(np.exp(2j * np.pi * k[1] * ys), exs[m])
        B[2 * m] = E.real.ravel()
        B[2 * m + 1] = E.imag.ravel()
        t = 2 * np.pi * k[2] * zs + phis[m]
        A[:, 2 * m] = np.sin(t)
        A[:, 2 * m + 1] = np.cos(t)
    T = (A @ B).reshape(shape)
    T += 1.0
    return T


def deformation_sphere(n=512, nsteps=50, cfl=0.5, nsub=8, seed=3):
    """Sphere R = 0.15 at (0.35, 0.35, 0.35) in the LeVeque deformation field
    (period 3, the field at t = 0, exact face averages), zero-gradient faces,
    dt for face CFL `cfl` (max |u| = 2), water/steam heat capacities of Table
    atm_water, a seeded smooth T of 8 Fourier modes (T = 1 +- 0.1), no
    phase change."""
    h = 1.0 / n
    shape = (n, n, n)
    c = sphere_fractions(shape, h, (0.35, 0.35, 0.35), 0.15, nsub=nsub)
    Cp_l = RHO_L * CP_L_SPEC
    Cp_g = RHO_G * CP_G_SPEC
    T = fourier_field(shape, h, seed=seed)
    e = (Cp_l * c + Cp_g * (1.0 - c)) * T
    u, v, w = deformation_faces(shape, h, 0.0)
    dt = cfl * h / 2.0
    return Workload("deformation-sphere-%d^3" % n, shape, (1, 1, 1), h, Cp_l, Cp_g, 1.0, dt, nsteps, 0.0,
                    c, e, u, v, w)


def droplet_subdomain(index, seed=4, n_lo=24, n_hi=96, nsub=6):
    """Subdomain `index` of the batched droplet workload (many independent
    periodic boxes): edge N ~ U{n_lo..n_hi}; one sphere or ellipsoid (equal
    odds), radius / semi-axes ~ U(0.15, 0.35) of the box, random rotation,
    centre 0.5 +- U(-0.1, 0.1); T = 1 in the liquid, 0 in the gas, heat
    capacity ratio 1000:1; a uniform velocity with |u| ~ U(0, 1) in a
    uniform random direction, dt for a face CFL number of 0.25; a uniform
    shift dd ~ U(-0.02, 0.02).  Each index draws from its own seeded stream,
    so any subdomain is generated alone, in any order."""
    rng = np.random.default_rng([seed, index])
    n = int(rng.integers(n_lo, n_hi + 1))
    h = 1.0 / n
    shape = (n, n, n)
    centre = tuple(0.5 + rng.uniform(-0.1, 0.1, 3))
    rot, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if rng.random() < 0.5:
        r = rng.uniform(0.15, 0.35)
        axes = (r, r, r)
    else:
        axes = tuple(rng.uniform(0.15, 0.35, 3))
    c = ellipsoid_fractions(shape, h, centre, axes, rot=rot, nsub=nsub)
    Cp_l, Cp_g = 1000.0, 1.0
    e = Cp_l * c
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    speed = rng.uniform(0.0, 1.0)
    vel = speed * d
    u, v, w = uniform_faces(shape, tuple(vel))
    amax = float(np.abs(vel).max())
    dt = 0.25 * h / amax if amax > 0 else 0.25 * h
    dd = float(rng.uniform(-0.02, 0.02))
    return Workload("droplet-%d-%d^3" % (index, n), shape, (0, 0, 0), h, Cp_l, Cp_g, 1.0, dt, 1, dd,
                    c, e, u, v, w)


# ---------------------------------------------------------------------------
# Training stencils for the learned interface normal
# ---------------------------------------------------------------------------

# offsets of the 27 cells of a stencil, index (dz*3+dy)*3+dx with dx, dy, dz
# in {0, 1, 2} for offsets -1, 0, 1 (x fastest)
_STENCIL = np.array([[dx, dy, dz] for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)], dtype=float)


def _curved_params(rng, kind):
    if kind == "sphere":
        axes = np.full(3, math.exp(rng.uniform(0.0, math.log(50.0))))
    else:
        axes = np.exp(rng.uniform(0.0, math.log(50.0), 3))
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    R = q * np.sign(np.linalg.det(q))
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    p_local = u / np.sqrt(np.sum(u * u / axes ** 2))  # a point of the surface
    centre = -(R @ p_local) + rng.uniform(-0.5, 0.5, 3)
    inside = 1.0 if rng.random() < 0.5 else 0.0
    return axes, R, centre, inside


def _plane_params(rng):
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    d = rng.uniform(-0.4, 0.4) * np.abs(n).sum()
    return n, d


def nearest_on_ellipsoids(axes, y, iters=200):
    """Points of the ellipsoids sum x_i^2 / a_i^2 = 1 (principal frames,
    axes [K, 3]) nearest to the points y [K, 3]: x_i = a_i^2 y_i / (a_i^2 +
    t) with t the root of sum (a_i y_i / (a_i^2 + t))^2 = 1 on t > -min
    a_i^2, by bisection (the sum decreases in t there)."""
    a2 = np.asarray(axes, dtype=float) ** 2
    y = np.asarray(y, dtype=float)
    f = lambda t: np.sum(a2 * y * y / (a2 + t[:, None]) ** 2, axis=1) - 1.0
    lo = -a2.min(axis=1) + 1e-12 * a2.min(axis=1)
    hi = np.sqrt(a2).max(axis=1) * np.abs(y).max(axis=1) * 2.0 + a2.max(axis=1)
    for _ in range(64):
        grow = f(hi) > 0
        if not grow.any():
            break
        hi = np.where(grow, hi * 2.0, hi)
    degenerate = f(lo) < 0  # y at the centre along the shortest axis: take lo
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        pos = f(mid) > 0
        lo = np.where(pos, mid, lo)
        hi = np.where(pos, hi, mid)
    t = np.where(degenerate, lo, 0.5 * (lo + hi))
    return a2 * y / (a2 + t[:, None])


def _curved_fractions(axes, R, centre, inside, nsub, chunk=96):
    """[K, 27] volume fractions of the stencils' cells (unit cells centred
    on the offsets) for ellipsoids {(x - c)^T Q (x - c) <= 1}, Q = R
    diag(1/a^2) R^T, by chord integration along x on an nsub x nsub
    midpoint rule (a few stencils at a time: small temporaries)."""
    if len(axes) > chunk:
        return np.concatenate([_curved_fractions(axes[s:s + chunk], R[s:s + chunk], centre[s:s + chunk],
                                                 inside[s:s + chunk], nsub, chunk)
                               for s in range(0, len(axes), chunk)])
    Q = np.einsum("kij,kj,klj->kil", R, 1.0 / axes ** 2, R)
    t = (np.arange(nsub) + 0.5) / nsub - 0.5
    o = _STENCIL[None, :, :]
    c = centre[:, None, :]
    ys = (o[..., 1] - c[..., 1])[..., None, None] + t[None, None, :, None]
    zs = (o[..., 2] - c[..., 2])[..., None, None] + t[None, None, None, :]
    ys, zs = np.broadcast_arrays(ys, zs)
    q = lambda a, b: Q[:, a, b][:, None, None, None]
    b = q(0, 1) * ys + q(0, 2) * zs
    cc = q(1, 1) * ys * ys + 2.0 * q(1, 2) * ys * zs + q(2, 2) * zs * zs - 1.0
    disc = b * b - q(0, 0) * cc
    sq = np.sqrt(np.clip(disc, 0.0, None))
    x0 = (-b - sq) / q(0, 0)
    x1 = (-b + sq) / q(0, 0)
    empty = disc < 0.0
    x0 = np.where(empty, 1.0, x0) + c[..., 0][..., None, None]
    x1 = np.where(empty, 0.0, x1) + c[..., 0][..., None, None]
    lo = (o[..., 0] - 0.5)[..., None, None]
    ln = np.clip(np.minimum(x1, lo + 1.0) - np.maximum(x0, lo), 0.0, None)
    frac = np.clip(ln.mean(axis=(-1, -2)), 0.0, 1.0)
    return np.where(inside[:, None] == 1.0, frac, 1.0 - frac)


def _plane_fractions(n, d, nsub, chunk=96):
    """[K, 27] volume fractions of {x : n . x <= d} by chord integration
    along each plane's dominant axis (where the chord is linear in the other
    two coordinates) on an nsub x nsub midpoint rule."""
    if len(n) > chunk:
        return np.concatenate([_plane_fractions(n[s:s + chunk], d[s:s + chunk], nsub, chunk)
                               for s in range(0, len(n), chunk)])
    K = n.shape[0]
    a = np.argmax(np.abs(n), axis=1)
    others = np.array([[1, 2], [0, 2], [0, 1]])[a]
    ar = np.arange(K)
    na = n[ar, a][:, None, None, None]
    nb = n[ar, others[:, 0]][:, None, None, None]
    nc = n[ar, others[:, 1]][:, None, None, None]
    oa = _STENCIL[:, a].T[:, :, None, None]
    ob = _STENCIL[:, others[:, 0]].T[:, :, None, None]
    oc = _STENCIL[:, others[:, 1]].T[:, :, None, None]
    t = (np.arange(nsub) + 0.5) / nsub - 0.5
    xb = ob + t[None, None, :, None]
    xc = oc + t[None, None, None, :]
    bound = (d[:, None, None, None] - nb * xb - nc * xc) / na  # n_a x_a <= ... on the dominant axis
    lo = oa - 0.5
    below = np.clip(bound - lo, 0.0, 1.0)  # length of {x_a <= bound} in the cell
    ln = np.where(na > 0, below, 1.0 - below)
    return np.clip(ln.mean(axis=(-1, -2)), 0.0, 1.0)


def _training_batch(kinds_i, rngs, nsub):
    K = len(kinds_i)
    X = np.zeros((K, 27))
    Y = np.zeros((K, 3))
    curved = [k for k in range(K) if kinds_i[k] != "plane"]
    planes = [k for k in range(K) if kinds_i[k] == "plane"]
    if curved:
        ps = [_curved_params(rngs[k], kinds_i[k]) for k in curved]
        axes = np.array([p[0] for p in ps])
        R = np.array([p[1] for p in ps])
        centre = np.array([p[2] for p in ps])
        inside = np.array([p[3] for p in ps])
        X[curved] = _curved_fractions(axes, R, centre, inside, nsub)
        yp = np.einsum("kji,kj->ki", R, -centre)  # the stencil centre in each principal frame
        xn = nearest_on_ellipsoids(axes, yp)
        g = np.einsum("kij,kj->ki", R, xn / axes ** 2)  # outward normal direction
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        Y[curved] = np.where(inside[:, None] == 1.0, g, -g)
    if planes:
        ps = [_plane_params(rngs[k]) for k in planes]
        n = np.array([p[0] for p in ps])
        d = np.array([p[1] for p in ps])
        X[planes] = _plane_fractions(n, d, nsub)
        Y[planes] = n
    return X, Y


def training_stencils(count, seed=50, start=0, kinds=("sphere", "ellipsoid", "plane"), nsub=12, batch=2048):
    """Training stencils of the learned interface normal: (X [count, 27]
    volume fractions of the 3 x 3 x 3 block around a mixed cell, Y [count,
    3] unit normals, liquid -> gas, at the surface point nearest the
    central cell's centre).  Sample i (global index start + i) has kind
    kinds[i % len(kinds)] and draws from its own stream, so any range is
    generated alone, in any order:
      * sphere: radius log-uniform in [1, 50] cells; ellipsoid: semi-axes
        log-uniform in [1, 50]; random rotation; the surface passes within
        half a cell (per axis) of the central cell's centre; liquid inside
        or outside with equal odds;
      * plane: uniform normal, offset U(-0.4, 0.4) |n|_1 from the central
        cell's centre;
    redrawn until the central cell is mixed (1e-6 < c < 1 - 1e-6).  Volume
    fractions by chord integration on an nsub x nsub midpoint rule (curved
    shapes along x, planes along their dominant axis)."""
    X = np.zeros((count, 27))
    Y = np.zeros((count, 3))
    for s in range(0, count, batch):
        idx = list(range(s, min(s + batch, count)))
        rngs = [np.random.default_rng([seed, start + i]) for i in idx]
        kinds_i = [kinds[(start + i) % len(kinds)] for i in idx]
        todo = list(range(len(idx)))
        for _ in range(1000):
            if not todo:
                break
            xb, yb = _training_batch([kinds_i[k] for k in todo], [rngs[k] for k in todo], nsub)
            ok = (xb[:, 13] > 1e-6) & (xb[:, 13] < 1 - 1e-6)
            for j, k in enumerate(todo):
                if ok[j]:
                    X[idx[k]] = xb[j]
                    Y[idx[k]] = yb[j]
            todo = [k for j, k in enumerate(todo) if not ok[j]]
        if todo:
            raise RuntimeError("no stencil with a mixed central cell")
    return X, Y
