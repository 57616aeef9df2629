"""Density filter, projection and their chain rule, plain numpy/scipy.

TEST INFRASTRUCTURE ONLY (imported by tests/ and the benchmark's CPU leg, never by the product).

Follows the paper's Sec. "Filtering and projection":
  * Eq. (FilterFunction): rho_t[n] = sum_{m in B_R(n)} w(n,m) rho[m] / sum_{m in B_R(n)} w(n,m), with the cone
    weight w = R - |r_m - r_n| over the sphere |r_m - r_n| < R (distances in voxels);
  * Eq. (Projection): rho_b = (tanh(beta eta) + tanh(beta (rho_t - eta))) / (tanh(beta eta) + tanh(beta (1 - eta)));
  * Eq. (GradientsFiltered): dF/drho[n] = sum_{m in B_R(n)} dF/drho_b[m] * drho_b/drho_t[m] * drho_t[m]/drho[n],
    with drho_t[m]/drho[n] = w(m,n) / sum_{k in B_R(m)} w(m,k).
Reading: the filter acts on the design box array; neighbourhoods are cut at the box faces (the
normalising sum only counts points inside the box).  A library correlation (scipy.ndimage.correlate,
zero outside the box) evaluates the neighbourhood sums.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import correlate


def cone_weights(R):
    """(2n+1)^3 array of w = R - |d| for |d| < R, else 0, n = ceil(R) - 1 (offsets in voxels)."""
    n = int(np.ceil(R)) - 1
    ax = np.arange(-n, n + 1, dtype=np.float64)
    dz, dy, dx = np.meshgrid(ax, ax, ax, indexing="ij")
    dist = np.sqrt(dx * dx + dy * dy + dz * dz)
    return np.where(dist < R, R - dist, 0.0)


def neighbourhood_sum(x, R):
    return correlate(np.asarray(x, dtype=np.float64), cone_weights(R), mode="constant", cval=0.0)


def filter_density(rho, R):
    """Eq. (FilterFunction)."""
    return neighbourhood_sum(rho, R) / neighbourhood_sum(np.ones_like(rho, dtype=np.float64), R)


def project(rho_t, beta, eta):
    """Eq. (Projection)."""
    rho_t = np.asarray(rho_t, dtype=np.float64)
    return (np.tanh(beta * eta) + np.tanh(beta * (rho_t - eta))) / (np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta)))


def project_derivative(rho_t, beta, eta):
    """d rho_b / d rho_t of Eq. (Projection)."""
    t = np.tanh(beta * (np.asarray(rho_t, dtype=np.float64) - eta))
    return beta * (1.0 - t * t) / (np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta)))


def chain_rule(dF_drho_b, rho_t, R, beta, eta):
    """Eq. (GradientsFiltered): dF/drho from dF/drho_b (the cone weight is symmetric)."""
    W = neighbourhood_sum(np.ones_like(rho_t, dtype=np.float64), R)
    g = np.asarray(dF_drho_b, dtype=np.float64) * project_derivative(rho_t, beta, eta) / W
    return neighbourhood_sum(g, R)
