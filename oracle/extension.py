"""Velocity extension across the interface (Sec. 3.3.1, Eqs. press_inv,
the velocity correction and u_l = u^{n+1} + u~): FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: plain numpy loops and one library sparse solve
(scipy.sparse.linalg.spsolve), for small grids; only the test suite, the
package smoke check and the benchmark's CPU-baseline leg may use it.  It
shares no code with the CUDA path.

What it computes (readings of the paper's 2D description, in 3D):
  * the sub-domain: the mixed cells (eps < c < 1 - eps) and the pure gas
    cells (c <= eps) of the first two layers around them, layers counted
    across cell faces (layer 1: face neighbours of mixed cells; layer 2:
    face neighbours of layer 1);
  * its boundary: faces to pure liquid cells (c >= 1 - eps) and the walls of
    a zero-gradient axis are no-slip (u~ = 0, no flux of p~); faces to gas
    cells outside the two layers are free-flow: p~ = 0 in the outside cell;
    periodic axes wrap;
  * in every sub-domain cell P the discrete Eq. press_inv,
        sum_faces beta_f (p~_Q - p~_P) = mdot_P (1/rho_g - 1/rho_l) A_P / h,
    beta_f = (dt / rho_f) / h^2, rho_f = rho_l c_f + rho_g (1 - c_f) with
    c_f the mean of the two cells' c, and A_P the PLIC plane area of a mixed
    cell in cell units (interface area per volume A h^2 / h^3 is the
    discrete delta_Gamma); gas cells have no source;
  * on every face with a sub-domain cell on at least one side and no liquid
    cell or wall, u~ = -(dt / rho_f) (p~_R - p~_L) / h (p~ = 0 outside);
    u~ = 0 on all other faces.  Then the discrete divergence of u~ in every
    sub-domain cell is -mdot (1/rho_g - 1/rho_l) delta_Gamma, cancelling the
    source that the projection left in u^{n+1}, and u_l = u^{n+1} + u~.
A sub-domain with no free-flow face (nothing fixes p~) is rejected.
"""
from __future__ import annotations

import numpy as np

from . import Grid, plane_area, reconstruct


def _nb(idx, axis, d, shape, bc):
    """Index of the face neighbour of cell idx=(k, j, i) along axis (0 x, 1 y,
    2 z) in direction d = +-1, or None across a zero-gradient wall."""
    k, j, i = idx
    p = [i, j, k]
    n = [shape[2], shape[1], shape[0]][axis]
    p[axis] += d
    if p[axis] < 0 or p[axis] >= n:
        if bc[axis] != 0:
            return None
        p[axis] %= n
    return (p[2], p[1], p[0])


def subdomain_layers(g: Grid, c):
    """-1 outside; 0 mixed; 1, 2 the gas layers of the sub-domain."""
    eps = float(g.par[4])
    bc = [int(b) for b in g.bc]
    shape = c.shape
    mixed = (c > eps) & (c < 1 - eps)
    gas = c <= eps
    layer = np.full(shape, -1, dtype=np.int64)
    layer[mixed] = 0
    for L in (1, 2):
        new = []
        for idx in zip(*np.nonzero(layer == L - 1)):
            for axis in range(3):
                for d in (-1, 1):
                    q = _nb(idx, axis, d, shape, bc)
                    if q is not None and gas[q] and layer[q] == -1:
                        new.append(q)
        for q in new:
            layer[q] = L
    return layer


def velocity_extension(g: Grid, c, mdot, rho_l, rho_g, dt):
    """Returns (ut, vt, wt, layer, p): the face corrections u~ in the x-, y-
    and z-face layouts, the sub-domain layers and p~ (0 outside)."""
    from scipy.sparse import lil_matrix
    from scipy.sparse.linalg import spsolve

    c = np.ascontiguousarray(c, dtype=np.float64)
    mdot = np.ascontiguousarray(mdot, dtype=np.float64)
    h = float(g.par[0])
    eps = float(g.par[4])
    bc = [int(b) for b in g.bc]
    shape = c.shape
    nz, ny, nx = shape
    liquid = c >= 1 - eps
    layer = subdomain_layers(g, c)
    sub = layer >= 0
    cells = list(zip(*np.nonzero(sub)))
    index = {q: n for n, q in enumerate(cells)}
    m, al, mixed = reconstruct(g, c)

    def rho_f(P, Q):
        cf = 0.5 * (c[P] + c[Q])
        return rho_l * cf + rho_g * (1.0 - cf)

    A = lil_matrix((len(cells), len(cells)))
    rhs = np.zeros(len(cells))
    free_faces = 0
    for n, P in enumerate(cells):
        diag = 0.0
        for axis in range(3):
            for d in (-1, 1):
                Q = _nb(P, axis, d, shape, bc)
                if Q is None or liquid[Q]:
                    continue  # no-slip
                beta = dt / rho_f(P, Q) / (h * h)
                diag -= beta
                if sub[Q]:
                    A[n, index[Q]] += beta
                else:
                    free_faces += 1  # p~ = 0 in Q
        A[n, n] += diag
        if layer[P] == 0:
            area = plane_area(m[(slice(None),) + P], al[P])
            rhs[n] = mdot[P] * (1.0 / rho_g - 1.0 / rho_l) * area / h
    if cells and free_faces == 0:
        raise ValueError("velocity extension: the sub-domain has no free-flow face")
    p = np.zeros(shape)
    if cells:
        sol = spsolve(A.tocsr(), rhs)
        for n, P in enumerate(cells):
            p[P] = sol[n]

    def face_field(axis):
        fshape = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][axis]
        ut = np.zeros(fshape)
        n_ax = [nx, ny, nz][axis]
        for L in zip(*np.nonzero(np.ones(shape, bool))):
            R = _nb(L, axis, 1, shape, bc)
            if R is None:
                continue  # the wall face
            if not (sub[L] or sub[R]) or liquid[L] or liquid[R]:
                continue
            val = -(dt / rho_f(L, R)) * (p[R] - p[L]) / h
            k, j, i = L
            f = [i, j, k]
            f[axis] += 1
            ut[f[2], f[1], f[0]] = val
            if bc[axis] == 0 and f[axis] == n_ax:
                f0 = list(f)
                f0[axis] = 0
                ut[f0[2], f0[1], f0[0]] = val  # periodic: face n is face 0
        return ut

    return face_field(0), face_field(1), face_field(2), layer, p
