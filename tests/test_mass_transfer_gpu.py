"""GPU parity of the mass transfer rate (Sec. 3.2) through the C ABI against
the FP64 oracle, element by element on the same seeded inputs.

Both sides take the same MYC normals (bit-identical, see test_parity_gpu)
and the same unit normals n = m/|m| (one correctly rounded square root and
division each), so every choice of plane (largest xi = |n . dx|) and the
band of pure cells agree exactly.  The plane constants differ in the last
bits (FP64 Newton on the GPU, bisection in the oracle), which moves the
distances d = alpha/|m| - n . dx by ~1e-15 cells; the gradients
(T_Gamma - T)/|d| then differ by that over |d| relative, and the weighted
averages by the same relative amount (the weights 1/|dx|^2 are rounded
reciprocals on the GPU, divisions in the oracle: 1 ulp).

Tolerances: distances 1e-13 h absolute; gradients 1e-13 h / |d| + 1e-14
relative; mdot 1e-11 relative to the largest |k grad| / h_fg of the cell's
stencil (taken as the largest over the grid); the band, the cells without a
gradient and the zero pattern of mdot exactly.
"""
import zlib

import numpy as np
import pytest

import oracle as O
from paper_2001_03477_gb300 import workloads as W
from test_oracle_mass_transfer import plane_fractions, tilted_plane

pytestmark = pytest.mark.gpu

K_L, K_G, H_FG = 0.68, 0.025, 2.257e6


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
    """(nx, ny, nz, bc, h, Cp_l, Cp_g, T_sat, c, e)"""
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    if name == "plane_linear":
        shape = (14, 13, 15)
        n, D = tilted_plane(2)
        D += 0.7
        c = plane_fractions(shape, n, D)
        h, Tg, Cpl, Cpg = 0.1, 373.15, 4.0e6, 1.2e3
        nz, ny, nx = shape
        Z, Y, X = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
        s = (D - (n[0] * X + n[1] * Y + n[2] * Z)) * h
        T = np.where(s > 0, Tg + 35.0 * s, Tg + 4.0 * s)
        return nx, ny, nz, (1, 1, 1), h, Cpl, Cpg, Tg, c, (Cpl * c + Cpg * (1 - c)) * T
    if name == "ellipsoid_ragged":
        nx, ny, nz = 37, 29, 21
        h = 1.0 / 32
        c = W.ellipsoid_fractions((nz, ny, nx), h, (0.55, 0.45, 0.33), (0.3, 0.22, 0.15),
                                  rot=np.linalg.qr(rng.normal(size=(3, 3)))[0], nsub=12)
        T = 100.0 + 3.0 * rng.random((nz, ny, nx))
        Cpl, Cpg = 4.0e6, 1.2e3
        return nx, ny, nz, (1, 1, 1), h, Cpl, Cpg, 100.0, c, (Cpl * c + Cpg * (1 - c)) * T
    if name == "tiny_periodic":
        nx, ny, nz = 4, 3, 5
        c = rng.random((nz, ny, nx))
        c[c < 0.3] = 0.0
        c[c > 0.7] = 1.0
        T = 1.0 + rng.random((nz, ny, nx))
        return nx, ny, nz, (0, 0, 0), 0.25, 3.0, 1.0, 1.2, c, (3.0 * c + (1 - c)) * T
    if name == "droplet_mixed_bc":
        N = 40
        h = 1.0 / N
        c = W.sphere_fractions((N, N, N), h, (0.5 + 0.3 * h, 0.45, 0.52), 0.27, nsub=12)
        zc = (np.arange(N) + 0.5) * h
        Z, Y, X = np.meshgrid(zc, zc, zc, indexing="ij")
        r = np.sqrt((X - 0.5 - 0.3 * h) ** 2 + (Y - 0.45) ** 2 + (Z - 0.52) ** 2)
        from scipy.special import erf
        T = np.where(r < 0.27, 373.15 + 5.0 * erf((0.27 - r) / 0.05), 373.15 + 1.0 * (r - 0.27))
        Cpl, Cpg = 4.0e6, 1.2e3
        return N, N, N, (0, 1, 0), h, Cpl, Cpg, 373.15, c, (Cpl * c + Cpg * (1 - c)) * T
    raise KeyError(name)


CASES = ["plane_linear", "ellipsoid_ragged", "tiny_periodic", "droplet_mixed_bc"]


def run_both(P, name, dd_per_mdot=-0.37):
    import torch
    nx, ny, nz, bc, h, Cpl, Cpg, Tg, c, e = case(name)
    og = O.Grid(nx, ny, nz, bc, h, Cpl, Cpg, Tg)
    mo, do, go = O.mass_transfer(og, c, e, K_L, K_G, H_FG)
    g = P.Grid(nx, ny, nz, bc, h, Cpl, Cpg, Tg)
    cd, ed = dev(c), dev(e)
    md = torch.full_like(cd, 7.0)
    dg = torch.full_like(cd, 7.0)
    gn = torch.full_like(cd, 7.0)
    dd = torch.full_like(cd, 7.0)
    P.vof_mass_transfer(g, cd, ed, K_L, K_G, H_FG, md, dg, gn, dd_per_mdot, dd)
    return (mo, do, go), (host(md), host(dg), host(gn), host(dd)), h, c


def check(oracle_out, gpu_out, h, dd_per_mdot=-0.37):
    mo, do, go = oracle_out
    mg, dgg, gng, ddg = gpu_out
    # the band (pure cells within two cells of a mixed cell) and its distances
    assert np.array_equal(do >= 0, dgg >= 0)
    band = do >= 0
    assert np.all(dgg[~band] == -1.0)
    assert np.abs(dgg[band] - do[band]).max(initial=0.0) <= 1e-13 * h
    # gradients: none exactly where the oracle has none
    has = band & (go != 0.0)
    assert np.array_equal(has, band & (gng != 0.0))
    if has.any():
        rel = np.abs(gng[has] - go[has]) / np.abs(go[has])
        assert np.all(rel <= 1e-13 * h / do[has] + 1e-14)
    # mdot: the zero pattern exactly, values to the rounding of the averages
    assert np.array_equal(mo == 0.0, mg == 0.0)
    scale = max(K_L, K_G) * np.abs(go).max(initial=0.0) / H_FG
    assert np.abs(mg - mo).max() <= 1e-11 * scale + 1e-300
    assert np.array_equal(ddg, dd_per_mdot * mg)


@pytest.mark.parametrize("name", CASES)
def test_mass_transfer_parity(P, name):
    o, g_, h, c = run_both(P, name)
    check(o, g_, h)
    mixed = (c > 1e-12) & (c < 1 - 1e-12)
    assert np.all(g_[0][~mixed] == 0.0) and np.all(g_[3][~mixed] == 0.0)


def test_plane_linear_closed_form_on_gpu(P):
    """Away from the zero-gradient side walls every mixed cell of the plane
    case gives (k_g G_g + k_l G_l)/h_fg with G_l = 35, G_g = -4 (the
    oracle's closed-form pin, here on the GPU)."""
    _, (mg, *_), h, c = run_both(P, "plane_linear")
    mixed = (c > 1e-12) & (c < 1 - 1e-12)
    inner = np.zeros(c.shape, bool)
    inner[:, 5:-5, 5:-5] = True
    want = (K_G * -4.0 + K_L * 35.0) / H_FG
    assert (mixed & inner).sum() >= 4
    assert np.abs(mg[mixed & inner] - want).max() <= 1e-10 * abs(want)


def test_no_interface_gpu(P):
    import torch
    g = P.Grid(9, 7, 6, (1, 0, 1), 0.1, 2.0, 1.0, 1.0)
    c = np.zeros((6, 7, 9))
    c[:2] = 1.0
    cd = dev(c)
    md = torch.full_like(cd, 3.0)
    dg = torch.full_like(cd, 3.0)
    P.vof_mass_transfer(g, cd, cd, K_L, K_G, H_FG, md, dg)
    assert np.all(host(md) == 0.0) and np.all(host(dg) == -1.0)


def test_full_size_bubble_mass_transfer(P):
    """The benchmark workload (256^3 bubble growth): every output against
    the oracle, and the counts of mixed and band cells."""
    import torch
    wl = W.bubble_growth(n=256, nsub=8)
    nz, ny, nx = wl.shape
    og = O.Grid(nx, ny, nz, wl.bc, wl.h, wl.Cp_l, wl.Cp_g, wl.T_sat)
    mo, do, go = O.mass_transfer(og, wl.c, wl.e, K_L, K_G, H_FG)
    g = P.Grid(nx, ny, nz, wl.bc, wl.h, wl.Cp_l, wl.Cp_g, wl.T_sat)
    cd, ed = dev(wl.c), dev(wl.e)
    md, dg, gn, dd = (torch.empty_like(cd) for _ in range(4))
    ws = torch.empty(P.vof_mass_transfer_workspace_bytes(g), dtype=torch.uint8, device="cuda")
    P.vof_mass_transfer(g, cd, ed, K_L, K_G, H_FG, md, dg, gn, -0.37, dd, workspace=ws)
    check((mo, do, go), (host(md), host(dg), host(gn), host(dd)), wl.h)
    counts = P.vof_mass_transfer_work_counts(g, ws)
    mixed = (wl.c > 1e-12) & (wl.c < 1 - 1e-12)
    assert counts["mixed"] == int(mixed.sum())
    assert counts["band"] == int((do >= 0).sum())
    # superheated liquid around a vapour bubble: evaporation everywhere
    assert np.all(host(md)[mixed] > 0)
