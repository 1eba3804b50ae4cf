"""The batched droplet workload's generator (no method arithmetic): each
subdomain is reproducible alone, and the draws follow the stated ranges."""
import numpy as np

from paper_2001_03477_gb300 import workloads as W


def test_subdomains_are_reproducible_alone():
    a = W.droplet_subdomain(7)
    W.droplet_subdomain(3)
    b = W.droplet_subdomain(7)
    assert a.shape == b.shape and np.array_equal(a.c, b.c) and a.dd_uniform == b.dd_uniform


def test_draws_follow_the_ranges():
    sizes, kinds, dds = [], [], []
    for i in range(40):
        wl = W.droplet_subdomain(i, nsub=2, n_lo=12, n_hi=20)
        n = wl.shape[0]
        sizes.append(n)
        assert 12 <= n <= 20 and wl.shape == (n, n, n) and wl.bc == (0, 0, 0)
        assert 0.0 <= wl.c.min() and wl.c.max() <= 1.0 and wl.c.sum() > 0
        speeds = np.array([wl.u[0, 0, 0], wl.v[0, 0, 0], wl.w[0, 0, 0]])
        assert np.linalg.norm(speeds) <= 1.0 + 1e-12
        if np.abs(speeds).max() > 0:
            assert abs(np.abs(speeds).max() * wl.dt / wl.h - 0.25) < 1e-12
        assert -0.02 <= wl.dd_uniform <= 0.02
        dds.append(wl.dd_uniform)
    assert len(set(sizes)) > 3 and min(dds) < 0 < max(dds)
