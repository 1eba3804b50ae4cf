"""GPU parity of the interface-Dirichlet heat diffusion (Sec. 3.4.2) through
the C ABI against the oracle (oracle/diffusion.py, a direct sparse solve).

Both sides take the same node phases, the same heights (the same sums of
the same 7 values) and the same plane distances up to the plane constants'
last bits, so the couplings agree to a few ulps; the GPU solves by Jacobi
sweeps until no T changes by more than 1e-13 of the largest T in a sweep.
T = e / C_p(c) is compared to 1e-10 of the largest T; the heights / plane
distances themselves are pinned on the oracle side.
"""
import zlib

import numpy as np
import pytest

import oracle as O
from oracle.diffusion import diffuse
from paper_2001_03477_gb300 import workloads as W
from test_oracle_mass_transfer import plane_fractions

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_03477_gb300 import build
    build.build()
    import paper_2001_03477_gb300 as P
    return P


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype=torch.float64)


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def case(name):
    """(c, T, bc, h, Cp_l, Cp_g, T_sat, k_l, k_g, dt)"""
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    if name == "plane":
        shape = (12, 12, 12)
        n = np.array([0.17, -0.11, 1.0])
        n /= np.linalg.norm(n)
        D = float(n @ np.array([6.0, 6.0, 6.23]))
        c = plane_fractions(shape, n, D)
        nz, ny, nx = shape
        Z, Y, X = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
        s = D - (n[0] * X + n[1] * Y + n[2] * Z)
        T = np.where(s > 0, 373.15 + 0.3 * s, 373.15 - 0.1 * s)
        return c, T, (1, 1, 1), 0.1, 4.0e6, 1.2e3, 373.15, 0.68, 0.025, 0.5
    if name == "droplet":
        n = 20
        h = 1.0 / n
        c = W.sphere_fractions((n, n, n), h, (0.5, 0.47, 0.53), 0.27, nsub=10)
        T = 373.15 + 2.0 * rng.random(c.shape)
        return c, T, (1, 1, 1), h, 4.0e6, 1.2e3, 373.15, 0.68, 0.025, 20.0
    if name == "ragged_periodic":
        nx, ny, nz = 23, 17, 13
        h = 1.0 / 16
        c = W.ellipsoid_fractions((nz, ny, nx), h, (0.7, 0.5, 0.4), (0.35, 0.3, 0.25),
                                  rot=np.linalg.qr(rng.normal(size=(3, 3)))[0], nsub=8)
        T = 1.0 + 0.5 * rng.random(c.shape)
        return c, T, (0, 1, 0), h, 3.0, 1.0, 1.2, 0.4, 0.05, 2e-3
    if name == "slab":
        N = 40
        h = 1.0 / N
        x0 = 0.75 + 0.37 * h
        frac = np.clip((x0 - np.arange(N) * h) / h, 0.0, 1.0)
        c = np.broadcast_to(frac[None, None, :], (1, 1, N)).copy()
        xc = (np.arange(N) + 0.5) * h
        T = np.broadcast_to(np.where(xc < x0, 1.0 + np.cos(np.pi * xc / (2 * x0)), 1.0)[None, None, :], c.shape)
        return c, T.copy(), (1, 0, 0), h, 2.0, 1.0, 1.0, 0.5, 0.01, 1.25e-3
    raise KeyError(name)


CASES = ["plane", "droplet", "ragged_periodic", "slab"]


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("hc", ["phase", "mixture"])
def test_heat_diffusion_parity(P, name, hc):
    c, T, bc, h, Cpl, Cpg, Ts, kl, kg, dt = case(name)
    nz, ny, nx = c.shape
    Cp = Cpl * c + Cpg * (1 - c)
    e = Cp * T
    og = O.Grid(nx, ny, nz, bc, h, Cpl, Cpg, Ts)
    # the slab case with its low x wall heated (the Stefan problem's wall)
    walls = {(0, -1): 1.7} if name == "slab" else None
    eo = diffuse(og, c, e, kl, kg, dt, wall_T=walls, heat_capacity=hc)
    g = P.Grid(nx, ny, nz, bc, h, Cpl, Cpg, Ts)
    ed = dev(e)
    tscale = np.abs(T).max()
    it, ch = P.vof_heat_diffusion(g, dev(c), ed, kl, kg, dt, tol=1e-13 * tscale, max_iter=200000,
                                  heat_capacity=P.VOF_CP_PHASE if hc == "phase" else P.VOF_CP_MIXTURE,
                                  wall_T=walls)
    assert it >= 1 and ch <= 1e-13 * tscale
    Tg, To = host(ed) / Cp, eo / Cp
    assert np.abs(Tg - To).max() <= 1e-10 * tscale
    # something happened (the cases are not at rest), except the steady plane
    if name != "plane":
        assert np.abs(To - T).max() > 1e-6 * tscale


def test_plane_linear_profile_stays_on_gpu(P):
    """The oracle's steady-state pin on the GPU: a temperature linear in the
    distance to a plane on each side is unchanged away from the walls."""
    c, T, bc, h, Cpl, Cpg, Ts, kl, kg, dt = case("plane")
    Cp = Cpl * c + Cpg * (1 - c)
    g = P.Grid(12, 12, 12, bc, h, Cpl, Cpg, Ts)
    ed = dev(Cp * T)
    P.vof_heat_diffusion(g, dev(c), ed, kl, kg, dt, tol=1e-11, max_iter=100000)
    Tg = host(ed) / Cp
    # the zero-gradient walls at z = 0 and z = 1.2 do not fit the linear
    # profile; the implicit step carries their change a few cells in (1e-4,
    # 1e-7, 1e-10 in the last layers, the same in the oracle)
    inner = np.zeros(c.shape, bool)
    inner[3:-3, 4:-4, 4:-4] = True
    assert np.abs(Tg - T)[inner].max() < 1e-9


def test_iteration_cap_reports_esolve(P):
    """A sweep budget too small for the tolerance ends with VOF_ESOLVE (the
    host reads it; nothing waits without a bound)."""
    c, T, bc, h, Cpl, Cpg, Ts, kl, kg, dt = case("droplet")
    nz, ny, nx = c.shape
    g = P.Grid(nx, ny, nz, bc, h, Cpl, Cpg, Ts)
    ed = dev((Cpl * c + Cpg * (1 - c)) * T)
    with pytest.raises(P.VofError) as err:
        P.vof_heat_diffusion(g, dev(c), ed, kl, kg, dt, tol=1e-300, max_iter=1)
    assert err.value.status == P.VOF_ESOLVE
