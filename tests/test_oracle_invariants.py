"""Pins of the oracle's advection, energy and phase-change steps (CPU only).

Each test checks a property that the paper or the mathematics fixes:
  * volume conservation of the divergence-free split sweeps (Weymouth-Yue,
    cited in Sec. 3.3.1),
  * a uniform temperature stays uniform under the consistent heat-capacity
    fluxes (Sec. 3.4.1, Eq. disc_et_adv),
  * thermal energy changes only by Delta e = Delta c (C_pl - C_pg) T_Gamma
    (end of Sec. 3.4.1),
  * exact translation of planes, upwind orientation of the WENO5 face value,
  * the kinematic Stefan problem reproduces delta(t) = 2 lambda sqrt(alpha t)
    (Sec. 4.3, Eqs. stefan_delta and stefan_lamda, delta(10 s) = 1.919 mm),
  * the evaporating droplet follows R(t) = R0 - mdot t (Sec. 4.2).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2001_03477_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def grid_of(wl):
    nz, ny, nx = wl.shape
    return O.Grid(nx, ny, nz, wl.bc, wl.h, wl.Cp_l, wl.Cp_g, wl.T_sat, wl.eps)


def deformation_case(n=16, Cp_l=1000.0, Cp_g=1.0, t=0.3):
    h = 1.0 / n
    shape = (n, n, n)
    c = W.sphere_fractions(shape, h, (0.35, 0.35, 0.35), 0.15, nsub=16)
    u, v, w = W.deformation_faces(shape, h, t)
    dt = 0.25 * h / 2.0
    g = O.Grid(n, n, n, (1, 1, 1), h, Cp_l, Cp_g, 1.0)
    return g, c, u, v, w, dt


class TestConservation:
    def test_volume_uniform_translation(self):
        wl = W.translating_sphere(n=16, nsteps=4, dd=0.0, nsub=16)
        g = grid_of(wl)
        c, e = wl.c, wl.e
        for s in range(4):
            v0 = O.total(c)
            c, e, sums = O.step(g, c, e, wl.u, wl.v, wl.w, wl.dt, s)
            assert abs((sums[0] - v0) + sums[2]) / v0 < 1e-14

    def test_volume_deformation_closed_box(self):
        g, c, u, v, w, dt = deformation_case()
        e = c * 1000.0
        for s in range(3):
            v0 = O.total(c)
            c, e, sums = O.step(g, c, e, u, v, w, dt, s)
            assert abs((sums[0] - v0) + sums[2]) / v0 < 1e-14
            assert abs(sums[2]) < 1e-6  # clipping stays small at CFL 0.125

    def test_clipped_volume_is_the_volume_the_clamp_removed(self):
        # A compressive velocity (not divergence-free) drives a mixed cell
        # over 1, so the clamp of the sweep removes a known amount.  On a
        # periodic line the face fluxes telescope, so the volume after the
        # sweep is the volume before, minus the dilatation terms
        # sum c_c (a_l - a_r), minus the clipped volume the sweep reports.
        n = 8
        g = O.Grid(n, 1, 1, (0, 0, 0), 1.0, 2.0, 1.0, 0.0)
        c = np.array([1.0, 1.0, 1.0, 0.45, 0.0, 0.0, 0.0, 0.0])[None, None, :]
        e = 2.0 * c + (1.0 - c)
        a = np.zeros(n + 1)
        a[3], a[4] = 0.9, 0.1  # into cell 3 from the full cell 2, out of it
        uf = a[None, None, :]
        cc, th = O.frozen(g, c, e)
        c1, e1, clip = O.sweep(g, 0, c, e, uf, 1.0, cc, th)
        dil = float((cc[0, 0, :] * (a[:n] - a[1:])).sum())
        assert clip > 0.2  # cell 3 reaches at least 0.45 + 0.9 - 0.1
        assert c1.max() == 1.0
        assert abs(c1.sum() - (c.sum() - dil - clip)) < 1e-14

    def test_energy_conserved_with_shift(self):
        g, c, u, v, w, dt = deformation_case()
        rng = np.random.default_rng(3)
        T = 1.0 + 0.1 * rng.random(c.shape)
        e = (1000.0 * c + (1 - c)) * T
        for s in range(2):
            E0 = O.total(e)
            c, e, sums = O.step(g, c, e, u, v, w, dt, s, dd_uniform=-0.01)
            assert abs(sums[1] - (E0 + sums[5])) / E0 < 1e-13
            # the shift's energy change is its volume change times the jump
            assert abs(sums[5] - sums[3] * (1000.0 - 1.0) * 1.0) < 1e-10


class TestUniformTemperature:
    @pytest.mark.parametrize("ratio", [1000.0, 3236.3])
    def test_uniform_T_stays_uniform(self, ratio):
        g, c, u, v, w, dt = deformation_case(Cp_l=ratio, Cp_g=1.0)
        T0 = 1.0  # equals T_Gamma, so the shift adds the jump at T0 too
        e = (ratio * c + (1.0 - c)) * T0
        for s in range(3):
            c, e, sums = O.step(g, c, e, u, v, w, dt, s, dd_uniform=-0.01)
            T = e / (ratio * c + (1.0 - c))
            assert np.abs(T - T0).max() / T0 < 1e-13


class TestTranslation:
    @pytest.mark.parametrize("axis", [0, 1, 2])
    def test_plane_shifts_one_cell_in_four_sweeps(self, axis):
        n = 12
        g = O.Grid(n, n, n, (1, 1, 1), 1.0, 1.0, 1.0, 0.0)
        shape = (n, n, n)
        # oblique plane mostly normal to `axis`
        nrm = np.array([0.2, -0.15, 0.1]); nrm[axis] = -1.0
        zc = np.arange(n) + 0.5
        c = np.zeros(shape)
        m = nrm / np.abs(nrm).sum()
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    # plane through the point 5.3 along `axis` at the box centre
                    p0 = np.array([6.0, 6.0, 6.0]); p0[axis] = 5.3
                    off = m @ (p0 - np.array([i, j, k], float))
                    c[k, j, i] = O.volume(m, off)
        e = c.copy()
        uf = np.zeros(g.face_shape(axis)) + 0.25
        cc, th = O.frozen(g, c, e)
        cur, ecur = c, e
        for s in range(4):
            cur, ecur, clip = O.sweep(g, axis, cur, ecur, uf, 1.0, cc, th)
        ref = np.roll(c, 1, axis=2 - axis)
        sl = [slice(3, n - 3)] * 3
        assert np.abs(cur[tuple(sl)] - ref[tuple(sl)]).max() < 1e-14

    def test_weno_upwind_at_temperature_step(self):
        # all-liquid column, T = 1 upstream of x = 6, 0 downstream
        n = 12
        g = O.Grid(n, 1, 1, (1, 0, 0), 1.0, 2.0, 1.0, 0.0)
        c = np.ones((1, 1, n))
        T = np.where(np.arange(n) < 6, 1.0, 0.0)[None, None, :]
        e = 2.0 * T
        cc, th = O.frozen(g, c, e)
        for sgn in (1.0, -1.0):
            uf = np.zeros((1, 1, n + 1)) + 0.2 * sgn
            _, _, _, F, G = O.sweep(g, 0, c, e, uf, 1.0, cc, th, want_flux=True)
            Tf = G[0, 0, 6] / (2.0 * 0.2 * sgn)
            # the face between cells 5 (T=1) and 6 (T=0) takes the donor side
            assert abs(Tf - (1.0 if sgn > 0 else 0.0)) < 1e-6

    def test_sphere_translation_returns(self):
        # Periodic translation of the sphere R = 0.2 by u = (1, 0.5, 0.25)
        # at CFL 0.25 to t = 4, which shifts it by (4, 2, 1) periods: the
        # exact solution is the initial field.  The L1 shape error
        # sum |c(4) - c(0)| h^3 must fall by at least 2.5x per doubling of
        # the grid (measured 3.2x from 16^3 to 32^3 and 3.7x to 64^3, about
        # second order), and the volume is conserved to round-off.  A
        # mis-signed transverse slope or a donor-slab offset error stalls
        # the convergence even when it cancels over a period.
        O.set_threads(os.cpu_count() or 1)
        errs = []
        for n in (16, 32, 64):
            wl = W.translating_sphere(n=n, nsteps=0, dd=0.0, nsub=16)
            g = grid_of(wl)
            nper = int(round(4.0 / wl.dt))
            assert nper == 16 * n
            c, e, sums = O.run(g, wl.c, wl.e, wl.u, wl.v, wl.w, wl.dt, 0, nper)
            errs.append(np.abs(c - wl.c).sum() * wl.h ** 3)
            assert abs(c.sum() - wl.c.sum()) / wl.c.sum() < 1e-12
        assert errs[0] / errs[1] >= 2.5, errs
        assert errs[1] / errs[2] >= 2.5, errs
        # relative to the sphere's volume: 2 % at 64^3
        assert errs[2] / (4.0 / 3.0 * math.pi * 0.2 ** 3) < 0.03, errs


class TestEnergyConsistency:
    def test_unfused_energy_matches_fused(self):
        g, c, u, v, w, dt = deformation_case()
        rng = np.random.default_rng(5)
        T = 1.0 + 0.1 * rng.random(c.shape)
        e = (1000.0 * c + (1 - c)) * T
        cc, th = O.frozen(g, c, e)
        for axis, uf in enumerate((u, v, w)):
            c1, e1, _, F, G = O.sweep(g, axis, c, e, uf, dt, cc, th, want_flux=True)
            e2 = O.energy_consistent(g, axis, c, e, F, uf, dt, th)
            assert np.array_equal(e1, e2)

    def test_conservative_vs_nonconservative_contrast(self):
        # Sec. 3.4.1: with C_pl/C_pg ~ 3200 the consistent fluxes keep a
        # uniform T exact, while C_p(cell) * sum T_f u_f A_f (Eq.
        # disc_et_adv_noncons) would not conserve energy; here we only check
        # the conservative side: uniform T after one sweep of a sphere.
        g, c, u, v, w, dt = deformation_case(Cp_l=3236.3)
        e = 3236.3 * c + (1 - c)
        cc, th = O.frozen(g, c, e)
        c1, e1, _ = O.sweep(g, 0, c, e, u, dt, cc, th)
        T1 = e1 / (3236.3 * c1 + (1 - c1))
        assert np.abs(T1 - 1.0).max() < 1e-13


def stefan_lambda(cpg, Tsup, hfg):
    from scipy.optimize import brentq
    from scipy.special import erf
    rhs = cpg * Tsup / (hfg * math.sqrt(math.pi))
    return brentq(lambda L: L * math.exp(L * L) * erf(L) - rhs, 1e-6, 5.0, xtol=1e-15, rtol=1e-15)


class TestStefanKinematic:
    def test_lambda_reproduces_paper(self):
        gd = json.load(open(os.path.join(GOLDEN, "stefan_water.json")))
        lam = stefan_lambda(gd["cp_g"], gd["T_sup"], gd["h_fg"])
        alpha_g = gd["k_g"] / (gd["rho_g"] * gd["cp_g"])
        d10 = 2 * lam * math.sqrt(alpha_g * gd["t_end_s"])
        assert abs(d10 - gd["delta_end_m"]) / gd["delta_end_m"] < 1e-3
        d0 = 2 * lam * math.sqrt(alpha_g * gd["t0_s"])
        assert abs(d0 - gd["delta0_m"]) / gd["delta0_m"] < 1e-3

    def test_two_step_advection_tracks_stefan_front(self):
        """Planar front with vapour at the wall: Step 1 moves the liquid with
        (1 - rho_g/rho_l) d', Step 2 shifts the interface by
        -(rho_g/rho_l) d' dt / h (Eq. Delta d); the sum must follow
        delta(t) exactly for a plane."""
        gd = json.load(open(os.path.join(GOLDEN, "stefan_water.json")))
        lam = stefan_lambda(gd["cp_g"], gd["T_sup"], gd["h_fg"])
        alpha_g = gd["k_g"] / (gd["rho_g"] * gd["cp_g"])
        delta = lambda t: 2 * lam * math.sqrt(alpha_g * t)
        N = 64
        L = gd["domain_m"]
        h = L / N
        r = gd["rho_g"] / gd["rho_l"]
        g = O.Grid(N, 1, 1, (1, 0, 0), h, 1.0, 1.0, 0.0)
        x = (np.arange(N) + 0.5) * h
        d0 = delta(gd["t0_s"])
        # exact fractions of the vapour layer [0, d0]
        c = np.clip((x + 0.5 * h - d0) / h, 0.0, 1.0)[None, None, :]
        e = c.copy()
        t = gd["t0_s"]
        dt = 0.02  # coarse in time: the kinematics is exact per step
        zeros_y = np.zeros((1, 2, N)); zeros_z = np.zeros((2, 1, N))
        while t < gd["t_end_s"] - 1e-12:
            step = min(dt, gd["t_end_s"] - t)
            dd_total = delta(t + step) - delta(t)
            ul = (1 - r) * dd_total / step
            u = np.full((1, 1, N + 1), ul)
            gs = O.Grid(N, 1, 1, (1, 0, 0), h, 1.0, 1.0, 0.0)
            cc, th = O.frozen(gs, c, e)
            c, e, _ = O.sweep(gs, 0, c, e, u, step, cc, th)
            c, e, _ = O.phase_shift(gs, c, e, dd_uniform=-r * dd_total / h)
            t += step
        vapour = h * (1.0 - c).sum()
        assert abs(vapour - delta(gd["t_end_s"])) / delta(gd["t_end_s"]) < 1e-9
        assert abs(vapour - gd["delta_end_m"]) / gd["delta_end_m"] < 1e-3


class TestEvaporatingDroplet:
    @pytest.mark.parametrize("N, cos4_bound", [(32, 0.03), (64, 0.006)])
    def test_volume_follows_linear_radius(self, N, cos4_bound):
        gd = json.load(open(os.path.join(GOLDEN, "evaporating_droplet.json")))
        h = 1.0 / N
        dt = gd["dt"][str(N)]
        R0, mdot, rho = gd["R0"], gd["mdot"], gd["rho_l"]
        shape = (1, N, N)
        c = W.ellipsoid_fractions(shape, (h, h, 1.0), (0.5, 0.5, 0.5), (R0, R0, 10.0), nsub=32)
        e = c.copy()
        g = O.Grid(N, N, 1, (1, 1, 0), h, 1.0, 1.0, 0.0)
        dd = -mdot / rho * dt / h
        t = 0.0
        for s in range(int(round(2.0 / dt))):  # t = 2 s, R = 0.13
            c, e, diag = O.phase_shift(g, c, e, dd_uniform=dd)
            t += dt
        area = c.sum() * h * h
        exact = math.pi * (R0 - mdot * t) ** 2
        assert abs(area - exact) / exact < 0.01
        # circular shape (Sec. 4.2): second moments isotropic, and no
        # four-fold distortion toward the grid's axes or diagonals -- the
        # cos 4 theta moment of the liquid, relative to its r^4 moment, is
        # -0.45 for a square of the same area and shrinks with the grid here
        yy, xx = np.meshgrid((np.arange(N) + 0.5) * h - 0.5, (np.arange(N) + 0.5) * h - 0.5, indexing="ij")
        cz = c[0]
        Ixx, Iyy = (cz * xx * xx).sum(), (cz * yy * yy).sum()
        assert abs(Ixx - Iyy) / (Ixx + Iyy) < 0.02
        r2 = xx * xx + yy * yy
        cos4 = (cz * (xx ** 4 - 6.0 * xx * xx * yy * yy + yy ** 4)).sum() / (cz * r2 * r2).sum()
        assert abs(cos4) < cos4_bound


class TestShiftBookkeeping:
    def test_totals_and_bounds(self):
        # the reported volume change is the field's change; c stays in [0,1];
        # evaporation shrinks, condensation grows
        g, c, u, v, w, dt = deformation_case()
        e = c.copy()
        c2, e2, diag = O.phase_shift(g, c, e, dd_uniform=-0.3)
        assert abs((c2.sum() - c.sum()) - diag[0]) < 1e-12
        assert diag[0] < 0
        assert c2.min() >= 0.0 and c2.max() <= 1.0
        c3, e3, diag3 = O.phase_shift(g, c, e, dd_uniform=0.3)
        assert diag3[0] > 0


def band_45(N, s):
    """Exact fractions of the periodic band s <= x + y <= s + N/2 (cell
    units), liquid inside; planes built from the pinned volume function."""
    c = np.zeros((1, N, N))
    m_lo = np.array([-0.5, -0.5, 0.0])
    m_hi = np.array([0.5, 0.5, 0.0])
    for j in range(N):
        for i in range(N):
            tot = 0.0
            for shift in (-N, 0, N):
                a, b = s + shift, s + shift + N / 2
                f1 = O.volume(m_lo, (i + j - a) / 2.0)
                f2 = O.volume(m_hi, (b - (i + j)) / 2.0)
                tot += max(0.0, f1 + f2 - 1.0)
            c[0, j, i] = tot
    return c


class TestPlaneMotion:
    def test_periodic_diagonal_band_moves_exactly(self):
        # a planar interface moved by the shift crosses many cells, corners
        # included, and stays exactly planar (Sec. 3.3.2 for a plane)
        N = 32
        g = O.Grid(N, N, 1, (0, 0, 0), 1.0, 1.0, 1.0, 0.0)
        s0, dd, nst = 7.3, -0.013, 120
        c = band_45(N, s0)
        e = c.copy()
        for _ in range(nst):
            c, e, _ = O.phase_shift(g, c, e, dd_uniform=dd)
        dist = -dd * nst * math.sqrt(2.0)
        cex = np.zeros_like(c)
        m_lo = np.array([-0.5, -0.5, 0.0]); m_hi = np.array([0.5, 0.5, 0.0])
        for j in range(N):
            for i in range(N):
                tot = 0.0
                for shift in (-N, 0, N):
                    a, b = s0 + shift + dist, s0 + shift + N / 2 - dist
                    tot += max(0.0, O.volume(m_lo, (i + j - a) / 2.0) + O.volume(m_hi, (b - (i + j)) / 2.0) - 1.0)
                cex[0, j, i] = tot
        assert np.abs(c - cex).max() < 1e-12
