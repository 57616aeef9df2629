"""Pins of the oracle's filter / projection / chain rule (Sec. "Filtering and projection")."""
import math

import numpy as np
import pytest

from oracle import filter as F


def brute_filter(rho, R):
    """Eq. (FilterFunction) by explicit sums over the sphere, neighbourhoods cut at the box faces."""
    nz, ny, nx = rho.shape
    out = np.zeros_like(rho)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                num = den = 0.0
                for kk in range(nz):
                    for jj in range(ny):
                        for ii in range(nx):
                            d = math.sqrt((i - ii) ** 2 + (j - jj) ** 2 + (k - kk) ** 2)
                            if d < R:
                                num += (R - d) * rho[kk, jj, ii]
                                den += R - d
                out[k, j, i] = num / den
    return out


def test_filter_matches_brute_force_sphere_sums():
    rng = np.random.default_rng(1)
    rho = rng.uniform(size=(5, 6, 7))
    for R in (1.5, 2.2, 3.0):
        np.testing.assert_allclose(F.filter_density(rho, R), brute_filter(rho, R), rtol=1e-13, atol=1e-14)


def test_filter_keeps_constants_and_bounds():
    rho = np.full((9, 8, 10), 0.37)
    np.testing.assert_allclose(F.filter_density(rho, 3.5), 0.37, rtol=1e-14)
    rng = np.random.default_rng(2)
    r = rng.uniform(size=(9, 8, 10))
    t = F.filter_density(r, 2.5)
    assert t.min() >= r.min() - 1e-15 and t.max() <= r.max() + 1e-15      # a weighted mean


def test_projection_closed_forms():
    x = np.linspace(0, 1, 11)
    for beta in (1.0, 10.0, 52.0):
        p = F.project(x, beta, 0.5)
        assert p[0] == pytest.approx(0.0, abs=1e-15) and p[-1] == pytest.approx(1.0, rel=1e-15)
        assert p[5] == pytest.approx(0.5, rel=1e-14)                          # eta = 0.5 is the midpoint
        np.testing.assert_allclose(p + p[::-1], 1.0, rtol=1e-13)               # odd symmetry about eta
    np.testing.assert_allclose(F.project(x, 1e-6, 0.3), x, atol=1e-9)         # beta -> 0: identity
    big = F.project(np.array([0.49, 0.51]), 1e4, 0.5)
    np.testing.assert_allclose(big, [0.0, 1.0], atol=1e-12)                    # beta -> inf: step at eta
    h = 1e-6
    for b in (3.0, 20.0):
        fd = (F.project(0.4 + h, b, 0.45) - F.project(0.4 - h, b, 0.45)) / (2 * h)
        assert F.project_derivative(0.4, b, 0.45) == pytest.approx(fd, rel=1e-8)


def test_chain_rule_vs_finite_differences():
    rng = np.random.default_rng(3)
    rho = rng.uniform(size=(6, 5, 7))
    c = rng.normal(size=rho.shape)
    R, beta, eta = 2.3, 8.0, 0.5

    def objective(r):
        return float(np.sum(c * F.project(F.filter_density(r, R), beta, eta)))

    g = F.chain_rule(c, F.filter_density(rho, R), R, beta, eta)
    h = 1e-6
    for idx in [(0, 0, 0), (3, 2, 4), (5, 4, 6), (2, 1, 3)]:
        r1 = rho.copy()
        r1[idx] += h
        r2 = rho.copy()
        r2[idx] -= h
        fd = (objective(r1) - objective(r2)) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-7, abs=1e-10)
