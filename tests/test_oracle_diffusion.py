"""Pins of the oracle's interface-Dirichlet heat diffusion (Sec. 3.4.2,
Eqs. T_diff_disc and mod_branchesT) against what the mathematics fixes
(CPU only).

* A temperature linear in the distance to a plane interface on each side,
  T_Gamma on the plane: every one-sided gradient of the irregular stencil is
  the exact gradient (heights and plane distances are exact for planes), so
  the operator vanishes at every node whose stencil stays inside the domain.
* T = T_Gamma everywhere is a fixed point of the implicit step.
* A liquid slab between a no-flux wall and the interface, T - T_Gamma =
  cos(pi x / 2 L) initially: the discrete decay converges to exp(-k/C_p
  (pi / 2 L)^2 t) as h and dt shrink together, at about first order in dt
  (backward Euler) with the interface off the grid nodes (theta < h).
* The height function and its fallback agree for planes along every axis.
* A wall at fixed temperature (wall_T) half a cell from the first node:
  between it and a plane interface the steady gas profile is the straight
  line from T_w to T_Gamma, node by node.
* heat_capacity="phase" is the "mixture" step wherever no cell is mixed; in
  a mixed cell the node changes temperature at its phase's heat capacity,
  and the cell's energy changes by exactly the heat conducted into it.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from oracle.diffusion import diffuse, diffusion_operator, interface_distance
from test_oracle_mass_transfer import plane_fractions


def tilted(seed):
    rng = np.random.default_rng(seed)
    n = np.array([rng.uniform(-0.25, 0.25), rng.uniform(-0.25, 0.25), 1.0])
    if seed % 2:
        n = -n
    n /= np.linalg.norm(n)
    D = float(n @ np.array([6.0, 6.0, 6.0 + rng.uniform(-0.4, 0.4)]))
    return n, D


def nodes(shape):
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    return X, Y, Z


@pytest.mark.parametrize("seed", range(4))
def test_linear_profile_is_steady(seed):
    shape = (12, 12, 12)
    n, D = tilted(seed)
    X, Y, Z = nodes(shape)
    # keep every node more than the cap (1e-3 cells) from the plane, where
    # theta would be eps h instead of the distance
    while np.abs(D - (n[0] * X + n[1] * Y + n[2] * Z)).min() < 2e-2:
        D += 0.031
    c = plane_fractions(shape, n, D)
    h, Tg = 0.1, 2.0
    s = (D - (n[0] * X + n[1] * Y + n[2] * Z))  # cells, > 0 in the liquid
    T = np.where(s > 0, Tg + 3.0 * s * h, Tg - 1.5 * s * h)
    g = O.Grid(12, 12, 12, (1, 1, 1), h, 4.0, 1.0, Tg)
    L = diffusion_operator(g, c, T, 0.7, 0.03).reshape(shape)
    inner = np.zeros(shape, bool)
    inner[1:-1, 4:-4, 4:-4] = True  # stencils clear of the walls and of the walls' MYC columns
    assert np.abs(L[inner]).max() <= 1e-9 * 3.0 / h


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_quadratic_profile_second_difference_exact(axis):
    # Each phase holds its own quadratic in the coordinate across a plane
    # interface normal to `axis`, both equal to T_Gamma on the plane.  The
    # three-point second difference over unequal distances (h to a node of
    # the same phase, theta to the interface) is exact for quadratics, so
    # k_p sum L(T) is k_p T'' at every node whose stencil stays off the
    # walls: the regular nodes and the two next to the interface alike.
    n_ax = 14
    shape = [6, 6, 6]
    shape[2 - axis] = n_ax
    shape = tuple(shape)
    D = 6.37  # the plane x_axis = D (cell units): liquid below it
    xs = [np.newaxis] * 3
    xs[2 - axis] = slice(None)
    line = lambda v: np.broadcast_to(v[tuple(xs)], shape)
    c = line(np.clip(D - np.arange(n_ax), 0.0, 1.0)).copy()  # exact fractions of the cut
    h, Tg, k_l, k_g = 0.1, 2.0, 0.7, 0.03
    A_l, B_l, A_g, B_g = 3.0, 5.0, -1.5, -2.0
    x = line((np.arange(n_ax) + 0.5 - D) * h)
    T = np.where(c >= 0.5, Tg + A_l * x + B_l * x * x, Tg + A_g * x + B_g * x * x)
    g = O.Grid(shape[2], shape[1], shape[0], (1, 1, 1), h, 4.0, 1.0, Tg)
    L = diffusion_operator(g, c, T, k_l, k_g).reshape(shape)
    want = np.where(c >= 0.5, 2.0 * B_l * k_l, 2.0 * B_g * k_g)
    inner = [slice(None)] * 3
    inner[2 - axis] = slice(1, n_ax - 1)  # off the two walls across the plane
    inner = tuple(inner)
    assert np.abs(L[inner] - want[inner]).max() <= 1e-8 * np.abs(want).max()


def test_saturation_temperature_is_a_fixed_point():
    shape = (10, 10, 10)
    n, D = tilted(1)
    c = plane_fractions(shape, n, D)
    g = O.Grid(10, 10, 10, (1, 0, 1), 0.1, 4.0, 1.0, 3.0)
    e = (4.0 * c + (1 - c)) * 3.0
    e1 = diffuse(g, c, e, 0.7, 0.03, 1e-3)
    T1 = e1 / (4.0 * c + (1 - c))
    assert np.abs(T1 - 3.0).max() < 1e-12


def slab_decay(N, steps_per_unit):
    """Liquid in x < x0 = 0.75 (the interface inside a cell), a no-flux wall
    at x = 0; T - T_G = cos(pi x / (2 x0)); returns the decay at the wall
    node after time 0.05 against the exact exp(-kappa lambda t)."""
    L = 1.0
    h = L / N
    x0 = 0.75 + 0.37 * h
    xf = np.arange(N) * h
    frac = np.clip((x0 - xf) / h, 0.0, 1.0)
    c = np.broadcast_to(frac[None, None, :], (1, 1, N)).copy()
    Cp_l, k_l, Tg = 2.0, 0.5, 1.0
    g = O.Grid(N, 1, 1, (1, 0, 0), h, Cp_l, 1.0, Tg)
    xc = (np.arange(N) + 0.5) * h
    T0 = np.where(xc < x0, Tg + np.cos(math.pi * xc / (2 * x0)), Tg)
    e = (Cp_l * c + (1 - c)) * T0
    t_end = 0.05
    nsteps = int(round(t_end * steps_per_unit))
    dt = t_end / nsteps
    for _ in range(nsteps):
        e = diffuse(g, c, e, k_l, 0.01, dt)
    T = e / (Cp_l * c + (1 - c))
    kappa, lam = k_l / Cp_l, (math.pi / (2 * x0)) ** 2
    got = (T[0, 0, 0] - Tg) / (T0[0] - Tg)
    return abs(got - math.exp(-kappa * lam * t_end))


def test_slab_decay_converges():
    e1 = slab_decay(20, 400)
    e2 = slab_decay(40, 800)
    e3 = slab_decay(80, 1600)
    assert e2 < e1 / 1.7 and e3 < e2 / 1.7
    assert e3 < 2e-3


@pytest.mark.parametrize("seed", range(3))
def test_height_and_plane_distances_agree_for_planes(seed):
    shape = (12, 12, 12)
    n, D = tilted(seed + 10)
    c = plane_fractions(shape, n, D)
    g = O.Grid(12, 12, 12, (1, 1, 1), 1.0, 1.0, 1.0, 1.0)
    m, al, _ = O.reconstruct(g, c)
    checked = 0
    for P in itertools.product(range(4, 8), range(4, 8), range(4, 8)):
        liq = c[P] >= 0.5
        for axis in range(3):
            for s in (-1, 1):
                Q = list(P)
                Q[2 - axis] += s
                Q = tuple(Q)
                if (c[Q] >= 0.5) == liq:
                    continue
                th = interface_distance(g, c, m, al, P, axis, s)
                zP, yP, xP = P
                x = np.array([xP + 0.5, yP + 0.5, zP + 0.5])
                e_ax = np.zeros(3)
                e_ax[axis] = s
                exact = (D - n @ x) / (n @ e_ax)  # along the axis to the plane
                assert abs(th - min(max(exact, 1e-3), 1.0)) < 1e-12
                checked += 1
    assert checked > 10


def test_wall_temperature_gives_the_straight_steady_profile():
    N, x_if = 16, 10.3  # interface 10.3 cells from the heated wall; liquid beyond
    c = np.clip(np.arange(N) + 1.0 - x_if, 0.0, 1.0).reshape(1, 1, N)
    Tsat, Tw = 2.0, 7.0
    g = O.Grid(N, 1, 1, (1, 0, 0), 1.0, 50.0, 1.0, Tsat)
    x = np.arange(N) + 0.5
    T0 = np.where(c.ravel() >= 0.5, Tsat, Tsat + 1.0)
    e = ((50.0 * c + (1.0 - c)).ravel() * T0).reshape(1, 1, N)
    for hc in ("mixture", "phase"):
        e1 = diffuse(g, c, e, 3.0, 0.5, 1e12, wall_T={(0, -1): Tw}, heat_capacity=hc)
        T1 = (e1 / (50.0 * c + (1.0 - c))).ravel()
        gas = c.ravel() < 0.5
        want = Tw + (Tsat - Tw) * x[gas] / x_if
        assert np.abs(T1[gas] - want).max() <= 1e-9 * (Tw - Tsat)
        assert np.abs(T1[~gas] - Tsat).max() <= 1e-9 * (Tw - Tsat)


def test_phase_heat_capacity():
    rng = np.random.default_rng(12)
    g = O.Grid(6, 5, 4, (0, 1, 1), 1.0, 40.0, 1.5, 1.0)
    c = (rng.random((4, 5, 6)) < 0.5).astype(float)  # pure cells only
    T = 1.0 + rng.random(c.shape)
    e = (40.0 * c + 1.5 * (1.0 - c)) * T
    a = diffuse(g, c, e, 2.0, 0.3, 0.7, heat_capacity="mixture")
    b = diffuse(g, c, e, 2.0, 0.3, 0.7, heat_capacity="phase")
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()
    # one mixed cell, a gas node (c = 0.3) in a hot gas column next to liquid
    N = 8
    c1 = np.array([0, 0, 0, 0.3, 1, 1, 1, 1], dtype=float).reshape(1, 1, N)
    g1 = O.Grid(N, 1, 1, (1, 0, 0), 1.0, 40.0, 1.5, 1.0)
    T1 = np.array([3, 3, 3, 1.0, 1, 1, 1, 1], dtype=float).reshape(1, 1, N)
    Cp = 40.0 * c1 + 1.5 * (1.0 - c1)
    e1 = Cp * T1
    dt = 0.05
    mix = diffuse(g1, c1, e1, 2.0, 0.3, dt, heat_capacity="mixture")
    ph = diffuse(g1, c1, e1, 2.0, 0.3, dt, heat_capacity="phase")
    # the gas node of the mixed cell warms far more at its phase's heat
    # capacity than at the mixture's (C_p(0.3) = 13.05 against 1.5)
    dT_phase = (ph[0, 0, 3] - e1[0, 0, 3]) / 1.5
    dT_mix = mix[0, 0, 3] / Cp[0, 0, 3] - T1[0, 0, 3]
    assert dT_phase > 5.0 * dT_mix > 0.0
    # its energy change is the heat conducted into it over dt (backward Euler:
    # the operator at the new temperatures), at the gas heat capacity
    # (pure cells: e / C_p; the mixed node: its old T plus its energy change over C_pg)
    Tnew = (ph / Cp).ravel()
    Tnew[3] = T1.ravel()[3] + dT_phase
    L = diffusion_operator(g1, c1, Tnew.reshape(1, 1, N), 2.0, 0.3).ravel()
    assert abs((ph.ravel()[3] - e1.ravel()[3]) - dt * L[3]) <= 1e-12 * abs(dt * L[3])
