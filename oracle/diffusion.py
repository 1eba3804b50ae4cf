"""Implicit heat diffusion with the interface as a Dirichlet boundary
(Sec. 3.4.2, "Calculating the energy diffusion term": Eqs. T_diff_disc and
mod_branchesT, after Sato and Niceno): FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: plain numpy loops and one library sparse solve
(scipy.sparse.linalg.spsolve), for small grids; it shares no code with the
CUDA path.

What it computes (readings of the paper's 2D description, in 3D):
  * a node belongs to the liquid when c >= 1/2, else to the gas; each phase
    diffuses with its own conductivity, and T_Gamma = T_sat on the
    interface;
  * along each axis, the gradient towards a neighbour of the same phase is
    the plain difference over h; towards a neighbour of the other phase it
    is (T_Gamma - T) / theta (or (T - T_Gamma) / theta on the minus side),
    theta the distance from the node to the interface along that axis, and
    the axis' second difference is divided by (d_- + d_+) / 2, d = h on a
    same-phase side and theta on an interface side (Eq. T_diff_disc, which
    shows one interface side; both sides take their own theta);
  * theta is the height function in that direction: the liquid volume of the
    7 cells centred on the node along the axis, when the column ends in pure
    cells of the node's phase behind and of the other phase beyond; the
    interface then lies H - 3.5 cells ahead of a liquid node (3.5 - H for a
    gas node).  Otherwise it is the distance along the axis to the PLIC
    plane of the pair's mixed cell (the node's own when it is mixed, else
    the neighbour's; the cell's MYC normal and plane constant), and half a
    cell when both are pure or the plane is parallel to the axis -- our
    reading of the paper's "plane reconstruction in the staggered volume";
    theta is capped to [eps h, h], eps = 1e-3;
  * zero-gradient walls carry no heat flux (a ghost node at the same T);
    periodic axes wrap;
  * backward Euler: C_p(c) (T^{n+1} - T^n) / dt = k_p sum_axes L_axis(T^{n+1})
    with T^n = e / C_p(c), and e^{n+1} = C_p(c) T^{n+1}
    (heat_capacity="mixture", reading A22);
  * heat_capacity="phase" (the default, reading A24): the phase-by-phase
    solve with constant properties in each phase: every node diffuses with the
    constant C_p of its phase, C_p,node (T^{n+1} - T^n) / dt = k_p sum L,
    and the cell's energy changes by the heat conducted into it,
    e^{n+1} = e^n + C_p,node (T^{n+1} - T^n).  Pure cells are unchanged by
    the choice; in a mixed cell the node's temperature follows its phase
    instead of being held by the mixture's heat capacity (a gas node in a
    half-liquid cell has ~1600 times the gas heat capacity under
    "mixture").  With it the coupled Stefan loop reproduces the paper's
    Table stefan_errors (tests/test_oracle_stefan.py);
  * wall_T (optional): {(axis, side): T_w} makes the low (side -1) or high
    (side +1) boundary of a zero-gradient axis a wall at fixed temperature,
    the node half a cell from it: gradient (T_w - T) / (h / 2), d = h / 2
    (the heated wall of the Stefan problem, Sec. 4.3).
"""
from __future__ import annotations

import numpy as np

from . import Grid, reconstruct

THETA_EPS = 1e-3


def _cell(idx, axis, k, shape, bc):
    """Cell k steps from idx=(z, y, x) along axis (0 x, 1 y, 2 z); None off a
    zero-gradient wall."""
    z, y, x = idx
    p = [x, y, z]
    n = [shape[2], shape[1], shape[0]][axis]
    p[axis] += k
    if p[axis] < 0 or p[axis] >= n:
        if bc[axis] != 0:
            return None
        p[axis] %= n
    return (p[2], p[1], p[0])


def _clamped(idx, axis, k, shape, bc):
    """As _cell, but a zero-gradient axis clamps to the boundary cell (the
    height function's column extends by its boundary values)."""
    z, y, x = idx
    p = [x, y, z]
    n = [shape[2], shape[1], shape[0]][axis]
    p[axis] += k
    if bc[axis] != 0:
        p[axis] = min(max(p[axis], 0), n - 1)
    else:
        p[axis] %= n
    return (p[2], p[1], p[0])


def interface_distance(g: Grid, c, m, al, P, axis, s):
    """theta (cell units, capped to [eps, 1]) from node P towards its
    neighbour in direction s (+-1) along axis, the two being of different
    phases."""
    eps = float(g.par[4])
    bc = [int(b) for b in g.bc]
    shape = c.shape
    liquid_p = c[P] >= 0.5
    col = [c[_clamped(P, axis, s * k, shape, bc)] for k in range(-3, 4)]
    back, front = col[0], col[6]
    if liquid_p:
        ok = back >= 1 - eps and front <= eps
    else:
        ok = back <= eps and front >= 1 - eps
    theta = None
    if ok:
        H = sum(col)
        theta = (H - 3.5) if liquid_p else (3.5 - H)
    else:
        Q = _cell(P, axis, s, shape, bc)
        mixed = lambda q: eps < c[q] < 1 - eps
        M = P if mixed(P) else (Q if Q is not None and mixed(Q) else None)
        theta = 0.5
        if M is not None:
            mm = m[(slice(None),) + M]
            # node P in M's local coordinates, the line P + t s e_axis
            zP, yP, xP = P
            zM, yM, xM = M
            off = np.array([xP - xM, yP - yM, zP - zM], dtype=float)
            for a in range(3):  # periodic wrap of the offset
                n = [shape[2], shape[1], shape[0]][a]
                if off[a] > 1:
                    off[a] -= n
                elif off[a] < -1:
                    off[a] += n
            x0 = off + 0.5
            ma = mm[axis] * s
            if ma != 0.0:
                t = (al[M] - mm @ x0) / ma
                theta = abs(t)
    return min(max(theta, THETA_EPS), 1.0)


def diffusion_operator(g: Grid, c, T, k_l, k_g, wall_T=None):
    """k_p sum_axes L_axis(T) per cell (the explicit form of the operator)."""
    A, b = _system(g, c, k_l, k_g, wall_T)
    return A @ T.ravel() + b


def _system(g: Grid, c, k_l, k_g, wall_T=None):
    """(A, b) with k_p sum L(T) = A T + b (b: the T_Gamma terms)."""
    from scipy.sparse import lil_matrix
    h = float(g.par[0])
    Tg = float(g.par[3])
    bc = [int(bb) for bb in g.bc]
    shape = c.shape
    N = c.size
    m, al, _ = reconstruct(g, c)
    A = lil_matrix((N, N))
    b = np.zeros(N)
    flat = lambda q: (q[0] * shape[1] + q[1]) * shape[2] + q[2]
    for P in np.ndindex(shape):
        liquid_p = c[P] >= 0.5
        kp = k_l if liquid_p else k_g
        n = flat(P)
        for axis in range(3):
            # one-sided gradients g_s = coef_self T_P + coef_nb T_nb + const
            terms = {}
            dists = {}
            for s in (-1, 1):
                Q = _cell(P, axis, s, shape, bc)
                if Q is None and wall_T and (axis, s) in wall_T:
                    Tw = float(wall_T[(axis, s)])  # wall at fixed T, half a cell away
                    terms[s] = (2.0 / h, None, 0.0, Tw * 2.0 / h)
                    dists[s] = 0.5 * h
                elif Q is None:
                    terms[s] = (0.0, None, 0.0, 0.0)  # wall: no flux
                    dists[s] = h
                elif (c[Q] >= 0.5) == liquid_p:
                    terms[s] = (1.0 / h, Q, 1.0 / h, 0.0)  # (T_Q - T_P)/h, sign fixed below
                    dists[s] = h
                else:
                    th = interface_distance(g, c, m, al, P, axis, s) * h
                    terms[s] = (1.0 / th, None, 0.0, Tg / th)  # (T_G - T_P)/theta
                    dists[s] = th
            denom = 0.5 * (dists[-1] + dists[1])
            # L = (g_+ - g_-) / denom with g_+ = (X_+ - T_P)/d_+, g_- = (T_P - X_-)/d_-:
            # L = [(X_+ - T_P)/d_+ + (X_- - T_P)/d_-] / denom
            for s in (-1, 1):
                cs, Q, cq, const = terms[s]
                A[n, n] += -kp * cs / denom
                if Q is not None:
                    A[n, flat(Q)] += kp * cq / denom
                b[n] += kp * const / denom
    return A.tocsr(), b


def diffuse(g: Grid, c, e, k_l, k_g, dt, wall_T=None, heat_capacity="phase"):
    """One backward-Euler diffusion step; returns e^{n+1}."""
    from scipy.sparse import diags
    from scipy.sparse.linalg import spsolve
    c = np.ascontiguousarray(c, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    Cp = float(g.par[1]) * c + float(g.par[2]) * (1.0 - c)
    T0 = e / Cp
    if heat_capacity == "mixture":
        Cd = Cp
    elif heat_capacity == "phase":
        Cd = np.where(c >= 0.5, float(g.par[1]), float(g.par[2]))
    else:
        raise ValueError(heat_capacity)
    A, b = _system(g, c, k_l, k_g, wall_T)
    M = diags((Cd / dt).ravel()) - A
    rhs = (Cd / dt * T0).ravel() + b
    T1 = spsolve(M.tocsr(), rhs).reshape(c.shape)
    if heat_capacity == "phase":
        return e + Cd * (T1 - T0)
    return Cp * T1
