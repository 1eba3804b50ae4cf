"""Pins of the oracle's PLIC geometry against the mathematics (CPU only).

Volume V(m, alpha): exact rational inclusion-exclusion over the cube's
vertices (a different formula from the oracle's case split) and brute-force
sampling.  Inverse: round trips.  Slab volumes: exact inclusion-exclusion for
boxes.  Area: finite differences of V and closed forms.  MYC: exactness for
planes whose centred columns span the interface (plane test, Sec. 4.1).
WENO5: polynomial exactness (Jiang-Shu / Shu 2009).
"""
from fractions import Fraction as Fr
import itertools
import math

import numpy as np
import pytest

import oracle as O

rng = np.random.default_rng(12345)


def exact_box_volume(m, alpha, L=(1, 1, 1)):
    """Exact volume of {x in box [0,L1]x[0,L2]x[0,L3] : m.x <= alpha} for
    m_i > 0 by inclusion-exclusion over the box vertices, in rationals."""
    m = [Fr(x) for x in m]
    a = Fr(alpha)
    L = [Fr(x) for x in L]
    tot = Fr(0)
    for v in itertools.product((0, 1), repeat=3):
        s = a - sum(m[d] * (L[d] if v[d] else 0) for d in range(3))
        if s > 0:
            tot += (-1) ** sum(v) * s ** 3
    return tot / (6 * m[0] * m[1] * m[2])


def exact_unit_volume_general(m, alpha):
    """Exact unit-cube volume for any nonzero-component m (mirroring by the
    substitution x_i -> 1 - x_i for negative m_i)."""
    mp = [abs(x) for x in m]
    a = Fr(alpha) - sum(Fr(x) for x in m if x < 0)
    return exact_box_volume(mp, a)


def random_m(nonzero=True):
    m = rng.normal(size=3)
    if nonzero:
        m = np.where(np.abs(m) < 1e-3, 1e-3, m)
    return m / np.abs(m).sum()


class TestVolume:
    def test_vs_exact_rational(self):
        worst = 0.0
        for _ in range(300):
            m = random_m()
            lo = sum(x for x in m if x < 0)
            hi = sum(x for x in m if x > 0)
            a = rng.uniform(lo - 0.05, hi + 0.05)
            ex = float(exact_unit_volume_general(m, a))
            ex = min(max(ex, 0.0), 1.0)
            worst = max(worst, abs(O.volume(m, a) - ex))
        assert worst <= 2e-15, worst

    def test_thin_components_vs_exact(self):
        # tiny m1 exercises the branches that would cancel catastrophically
        worst = 0.0
        for m1 in (1e-3, 1e-6, 1e-9, 1e-12):
            for _ in range(40):
                m2 = rng.uniform(0.05, 0.5)
                m = np.array([m1, m2, 1.0])
                m /= m.sum()
                a = rng.uniform(0, 1)
                ex = float(exact_box_volume(m, a))
                ex = min(max(ex, 0.0), 1.0)
                worst = max(worst, abs(O.volume(m, a) - ex))
        assert worst <= 2e-15, worst

    def test_degenerate_limits(self):
        # 1D: V = alpha;  2D: triangle / trapezoid areas
        for a in np.linspace(0, 1, 11):
            assert abs(O.volume([0, 0, 1], a) - a) < 1e-16
            assert abs(O.volume([0, -1, 0], a - 1) - a) < 1e-15
        for _ in range(100):
            m2 = rng.uniform(0.01, 0.99)
            m = [0.0, m2, 1 - m2]
            a = rng.uniform(0, 1)
            # 2D inclusion-exclusion: (a^2 - <a-m2>^2 - <a-m3>^2 + <a-1>^2)/(2 m2 m3)
            p = lambda x: max(x, 0.0) ** 2
            ex = (p(a) - p(a - m[1]) - p(a - m[2]) + p(a - 1)) / (2 * m[1] * m[2])
            assert abs(O.volume(m, a) - ex) < 1e-13

    def test_brute_force_orientation(self):
        # catches sign/orientation mistakes: liquid is m.x <= alpha
        n = 96
        g = (np.arange(n) + 0.5) / n
        Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
        for _ in range(8):
            m = random_m(nonzero=False)
            a = rng.uniform(-0.3, 0.3)
            vb = np.mean(m[0] * X + m[1] * Y + m[2] * Z <= a)
            assert abs(O.volume(m, a) - vb) < 3.0 / n

    def test_scale_invariance(self):
        for _ in range(50):
            m = random_m()
            a = rng.uniform(-0.5, 0.5)
            assert abs(O.volume(3.7 * m, 3.7 * a) - O.volume(m, a)) < 1e-15


class TestInverse:
    @pytest.mark.parametrize("c", [1e-14, 1e-9, 1e-3, 0.3, 0.5, 0.77, 1 - 1e-9])
    def test_roundtrip_v_alpha_v(self, c):
        for _ in range(60):
            m = random_m(nonzero=False)
            a = O.alpha(m, c)
            assert abs(O.volume(m, a) - c) <= 1e-15 + 1e-15 * c

    def test_axis_aligned_and_2d(self):
        for m in ([1, 0, 0], [0, -1, 0], [0, 0, 1], [0.5, 0.5, 0], [0, -0.3, 0.7]):
            for c in (1e-9, 0.25, 0.5, 0.9):
                a = O.alpha(np.array(m, float), c)
                assert abs(O.volume(m, a) - c) < 1e-15

    def test_alpha_is_the_nearest_double(self):
        # The plane constant is the double whose volume is nearest to c: no
        # neighbouring double gives a volume closer to c.  The normals are
        # non-negative dyadic rationals summing to exactly 1, so the oracle's
        # mirroring and L1 scaling are exact and alpha is returned unscaled.
        for it in range(400):
            k = rng.integers(1, 2 ** 20, size=3).astype(float)
            if it % 4 == 0:
                k[rng.integers(0, 3)] = 0.0  # 2D normals too
            k[2] = 2.0 ** 21 - k[0] - k[1]
            m = k / 2.0 ** 21
            assert m.sum() == 1.0
            c = float(rng.choice([rng.uniform(1e-9, 1e-3), rng.uniform(0.0, 1.0), 1.0 - rng.uniform(1e-9, 1e-3)]))
            a = O.alpha(m, c)
            err = abs(O.volume(m, a) - c)
            for nb in (np.nextafter(a, -np.inf), np.nextafter(a, np.inf)):
                assert err <= abs(O.volume(m, nb) - c), (m, c, a, nb)

    def test_roundtrip_alpha_v_alpha(self):
        worst = 0.0
        for _ in range(300):
            m = random_m()
            lo = sum(x for x in m if x < 0)
            a = lo + rng.uniform(0.02, 0.98)
            v = O.volume(m, a)
            # compare only where dV/dalpha is not tiny
            if O.plane_area(m, a) < 1e-3:
                continue
            worst = max(worst, abs(O.alpha(m, v) - a))
        assert worst < 1e-12, worst


class TestSlab:
    def test_slab_vs_exact_boxes(self):
        worst = 0.0
        for _ in range(200):
            m = random_m()
            axis = int(rng.integers(3))
            lo = sum(x for x in m if x < 0)
            a = lo + rng.uniform(0.05, 0.95)
            delta = rng.uniform(0.01, 0.5)
            x0 = rng.choice([0.0, 1.0 - delta])
            # exact: mirror negative components, then slab = box(x0+delta) - box(x0)
            mp = [abs(x) for x in m]
            am = Fr(a) - sum(Fr(x) for x in m if x < 0)
            # mirroring axis `axis` maps [x0, x0+d] to [1-x0-d, 1-x0]
            xs = x0 if m[axis] >= 0 else 1.0 - x0 - delta
            Lhi = [1, 1, 1]; Llo = [1, 1, 1]
            Lhi[axis] = Fr(xs) + Fr(delta)
            Llo[axis] = Fr(xs)
            # volume of box with its low corner at the origin: shift the slab
            # to start at 0 is not needed - inclusion-exclusion of [0,Lhi]-[0,Llo]
            ex = exact_box_volume(mp, am, Lhi) - (exact_box_volume(mp, am, Llo) if xs > 0 else 0)
            got = O.slab_volume(m, a, axis, x0, delta)
            worst = max(worst, abs(got - float(ex)))
        assert worst < 2e-15, worst


class TestArea:
    def test_area_vs_derivative(self):
        for _ in range(100):
            m = random_m()
            lo = sum(x for x in m if x < 0)
            a = lo + rng.uniform(0.05, 0.95)
            hh = 1e-5
            fd = (O.volume(m, a + hh) - O.volume(m, a - hh)) / (2 * hh) * np.linalg.norm(m)
            assert abs(fd - O.plane_area(m, a)) < 1e-8

    def test_closed_forms(self):
        assert abs(O.plane_area([0, 0, 1], 0.3) - 1.0) < 1e-15
        # diagonal plane through the centre: regular hexagon of side sqrt(2)/2
        m = np.array([1, 1, 1]) / 3.0
        assert abs(O.plane_area(m, 0.5) - 3 * math.sqrt(3) / 2 * 0.5) < 1e-14  # (3 sqrt3/2) s^2
        # corner triangle x+y+z = t: equilateral with side t sqrt(2)
        t = 0.4
        assert abs(O.plane_area(m, t / 3) - math.sqrt(3) / 4 * 2 * t * t) < 1e-14


def plane_block(n, c_centre):
    m = n / np.abs(n).sum()
    off = O.alpha(m, c_centre)
    s = np.zeros((3, 3, 3))
    for dz, dy, dx in itertools.product(range(3), repeat=3):
        o = np.array([dx - 1, dy - 1, dz - 1], float)
        s[dz, dy, dx] = O.volume(m, off - m @ o)
    return s, m, off


def spans(s, d):
    cs = np.moveaxis(s, 2 - d, 0)
    for (p, q) in [(1, 1), (0, 1), (2, 1), (1, 0), (1, 2)]:
        col = cs[:, q, p]
        if not ((col[0] == 1.0 and col[2] == 0.0) or (col[0] == 0.0 and col[2] == 1.0)):
            return False
    return True


class TestNormals:
    def test_myc_exact_for_spanning_planes(self):
        nspan = 0
        for _ in range(3000):
            n = rng.normal(size=3)
            n /= np.linalg.norm(n)
            s, m, off = plane_block(n, rng.uniform(0.02, 0.98))
            d = int(np.argmax(np.abs(m)))
            if not spans(s, d):
                continue
            nspan += 1
            mm = O.myc(s)
            assert np.abs(mm - m).max() < 1e-14
            assert np.abs(O.cc_candidate(s, d) - m).max() < 1e-14
            # plane constant and the interface distance of Eq. cell_d
            a = O.alpha(mm, s[1, 1, 1])
            assert abs(a - off) < 1e-13
        assert nspan > 100

    def test_pure_neighbour_distances_plane(self):
        # Sec. 4.1: distances from pure first/second neighbours to the plane
        # of a mixed cell equal theory: d_Gamma = alpha/|m| - n.dx (Eq. dint_trans)
        for _ in range(200):
            n = rng.normal(size=3)
            n /= np.linalg.norm(n)
            s, m, off = plane_block(n, rng.uniform(0.05, 0.95))
            d = int(np.argmax(np.abs(m)))
            if not spans(s, d):
                continue
            mm = O.myc(s)
            a = O.alpha(mm, s[1, 1, 1])
            nrm = np.linalg.norm(mm)
            for off2 in itertools.product((-2, -1, 0, 1, 2), repeat=3):
                dx = np.array(off2, float) + 0.5  # node of the neighbour from the cell origin
                dG = a / nrm - (mm / nrm) @ dx
                theory = (off - m @ dx) / np.linalg.norm(m)
                assert abs(dG - theory) < 1e-13

    def test_youngs_is_the_mean_of_the_corner_gradients(self):
        # Youngs' normal is minus the mean of the gradients at the cell's
        # eight vertices, each vertex gradient the mean of the differences
        # across the 2 x 2 x 2 block of cells around that vertex; then
        # L1-normalised.  Built here from that construction for random
        # stencils (s[z, y, x], offsets -1..1).
        for _ in range(200):
            st = rng.random((3, 3, 3))
            g = np.zeros(3)
            for cz, cy, cx in itertools.product((0, 1), repeat=3):
                blk = st[cz:cz + 2, cy:cy + 2, cx:cx + 2]  # the cells around vertex (cx, cy, cz)
                g += [(blk[:, :, 1] - blk[:, :, 0]).mean(), (blk[:, 1, :] - blk[:, 0, :]).mean(),
                      (blk[1, :, :] - blk[0, :, :]).mean()]
            m = -g / np.abs(g).sum()
            assert np.abs(O.youngs(st) - m).max() < 1e-14

    def test_youngs_axis_aligned(self):
        for d in range(3):
            for sgn in (1, -1):
                n = np.zeros(3); n[d] = sgn
                s, m, _ = plane_block(n, 0.37)
                assert np.abs(O.youngs(s) - m).max() < 1e-15
                assert np.abs(O.myc(s) - m).max() < 1e-15

    def test_normal_points_liquid_to_gas(self):
        # liquid sphere: outward normal; MYC must agree in sign
        from paper_2001_03477_gb300 import workloads as W
        c = W.sphere_fractions((16, 16, 16), 1.0, (8.1, 7.9, 8.05), 4.5, nsub=24)
        for k, j, i in np.argwhere((c > 1e-12) & (c < 1 - 1e-12)):
            if min(i, j, k) < 1 or max(i, j, k) > 14:
                continue
            m = O.myc(c[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2])
            r = np.array([i + 0.5 - 8.1, j + 0.5 - 7.9, k + 0.5 - 8.05])
            assert m @ r > 0


def cell_avg_poly(coefs, j):
    """exact average of sum coefs[p] x^p over [j-1/2, j+1/2] (rationals)"""
    tot = Fr(0)
    a, b = Fr(2 * j - 1, 2), Fr(2 * j + 1, 2)
    for p, cp in enumerate(coefs):
        tot += Fr(cp) * (b ** (p + 1) - a ** (p + 1)) / (p + 1)
    return tot


def poly_at(coefs, x):
    return sum(Fr(cp) * Fr(x) ** p for p, cp in enumerate(coefs))


class TestWeno:
    def test_constant_exact(self):
        for v in (0.0, 1.0, 373.15, -2.5e-3):
            assert O.weno5([v] * 5) == v

    def test_quadratic_exact(self):
        for _ in range(50):
            coefs = [int(x) for x in rng.integers(-5, 6, size=3)]
            v = [float(cell_avg_poly(coefs, j)) for j in (-2, -1, 0, 1, 2)]
            ex = float(poly_at(coefs, Fr(1, 2)))
            assert abs(O.weno5(v) - ex) < 1e-12 * (1 + abs(ex))

    def test_linear_weights_fifth_order(self):
        # with a huge epsilon the weights are the optimal (0.1,0.6,0.3) and
        # the scheme reproduces the face value of any quartic
        for _ in range(50):
            coefs = [int(x) for x in rng.integers(-3, 4, size=5)]
            v = [float(cell_avg_poly(coefs, j)) for j in (-2, -1, 0, 1, 2)]
            ex = float(poly_at(coefs, Fr(1, 2)))
            assert abs(O.weno5(v, 1e30) - ex) < 1e-11 * (1 + abs(ex))

    def test_matches_its_construction(self):
        # WENO5 built from its definition (Jiang & Shu; Shu 2009, cited in
        # Sec. 3.4.1): p_k is the quadratic with the cell averages of stencil
        # k (cells -2..0, -1..1, 0..2 around the donor 0), q_k = p_k(1/2);
        # the linear weights d_k are the ones that make sum d_k q_k the
        # quartic's face value for every quartic; the smoothness indicator is
        # beta_k = sum over l = 1, 2 of the integral over the donor cell of
        # (d^l p_k / dx^l)^2; alpha_k = d_k / (eps + beta_k)^2.  Every piece
        # is computed generically (linear solves, polynomial derivatives and
        # integrals), none from the scheme's printed coefficients.
        P = np.polynomial.Polynomial

        def cell_avg_matrix(cells, deg):
            return np.array([[((j + 0.5) ** (p + 1) - (j - 0.5) ** (p + 1)) / (p + 1) for p in range(deg + 1)]
                             for j in cells])

        stencils = [(-2, -1, 0), (-1, 0, 1), (0, 1, 2)]
        # linear weights from the monomials x^0 .. x^4
        A5 = cell_avg_matrix((-2, -1, 0, 1, 2), 4)
        rows, rhs = [], []
        for p in range(5):
            vals = A5[:, p]  # cell averages of x^p
            rows.append([P(np.linalg.solve(cell_avg_matrix(st, 2), vals[[j + 2 for j in st]]))(0.5)
                         for st in stencils])
            rhs.append(0.5 ** p)
        d = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
        assert np.allclose(d, [0.1, 0.6, 0.3], atol=1e-14)

        def expected(v, eps=1e-6):
            q, beta = [], []
            for st in stencils:
                p = P(np.linalg.solve(cell_avg_matrix(st, 2), np.array([v[j + 2] for j in st])))
                q.append(p(0.5))
                b = 0.0
                for l in (1, 2):
                    sq = (p.deriv(l) ** 2).integ()
                    b += sq(0.5) - sq(-0.5)
                beta.append(b)
            a = d / (eps + np.array(beta)) ** 2
            return float((a * np.array(q)).sum() / a.sum())

        gen = np.random.default_rng(11)
        cases = [gen.random(5) for _ in range(200)]
        cases += [373.15 + 0.01 * gen.standard_normal(5) for _ in range(100)]
        cases += [np.sin(0.7 * np.arange(5) + gen.random() * 6) * gen.random() for _ in range(100)]
        cases += [np.where(np.arange(5) < gen.integers(1, 5), 1.0, 0.0) + 1e-3 * gen.random(5) for _ in range(50)]
        for v in cases:
            ex = expected(v)
            scale = np.abs(v).max()
            assert abs(O.weno5(list(v)) - ex) <= 1e-12 * scale, (v, O.weno5(list(v)), ex)

    def test_eno_at_step(self):
        # discontinuity downwind of the donor: the face value stays on the
        # smooth upwind side
        v = [1.0, 1.0, 1.0, 0.0, 0.0]
        assert abs(O.weno5(v) - 1.0) < 1e-6
        v = [0.0, 0.0, 1.0, 1.0, 1.0]
        assert abs(O.weno5(v) - 1.0) < 1e-6
