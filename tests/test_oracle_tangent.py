"""Tangent-linear pin of the adjoint gradient (Sec. "Time-domain adjoint formulation", Eq.
(Gradient_analytic); the C-T8 check): the forward-mode derivative of the discrete scheme along a
seeded density direction equals the adjoint gradient projected on that direction, free of the
truncation and cancellation error of finite differences.  The tangent mode itself is pinned by a
central difference along the same direction.  CPU only.

Cases have fields that decay inside the window (damped metals, CPML), the condition under which the
frequency-domain adjoint is exact for the discrete objective.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import EPS0, base_desc, vacuum


def _damped_metal(seed):
    m = synth.drude_lorentz_metal(seed, 2)
    poles = []
    for comp in range(3):
        (a1, c1), (a2, c2) = m["poles"][comp]
        poles.append([(complex(-8e14, 0.0), 0.5 * c1), (complex(-1e15, a2.imag), c2)])
    m["poles"] = poles
    m["sigma"] = [-2 * EPS0 * poles[0][0][1].real] * 3
    return m


def _problem(m1, m2, gamma=0.0, lambdas=(600.0,), weights=None, src_comp=2, layout=0, steps=3000, seed=11):
    d = base_desc(20, 20, 20, dx=20e-9, n_steps=steps, cpml=5, precision=64, design=(8, 7, 6), gap=(2, 2, 2),
                  src_kind=0, src_comp=src_comp, src_pos=(10, 10, 10), lambdas_nm=lambdas, weights=weights)
    d["density_layout"] = layout
    o = oracle.Oracle(d)
    o.set_materials(vacuum(), m1, m2, gamma)
    rho = synth.uniform_rho(o.vshape, seed, 0.2, 0.8)
    o.set_density(rho)
    return o, rho


def _adjoint_vs_tangent(o, rho, seed=5):
    F0, _ = o.forward()
    o.adjoint()
    g = o.gradient()
    drho = np.random.default_rng(seed).standard_normal(rho.shape)
    F, dF = o.tangent(drho)
    assert F == F0                                   # the tangent run carries the same primal run
    return dF, float(np.sum(g * drho)), drho


def test_tangent_mode_matches_central_difference():
    o, rho = _problem(vacuum(), _damped_metal(7))
    dF, _, drho = _adjoint_vs_tangent(o, rho)
    h = 1e-5
    o.set_density(rho + h * drho)
    Fp, _ = o.forward()
    o.set_density(rho - h * drho)
    Fm, _ = o.forward()
    assert abs((Fp - Fm) / (2 * h) - dF) <= 1e-7 * abs(dF)


@pytest.mark.parametrize("case", ["metal", "three_freq_gamma_dielectric", "per_sample_layout", "non_dispersive"])
def test_adjoint_gradient_equals_tangent_linear_derivative(case):
    if case == "metal":
        o, rho = _problem(vacuum(), _damped_metal(7))
    elif case == "three_freq_gamma_dielectric":
        o, rho = _problem(synth.lorentz_dielectric(5, 1, (1.5, 1.5, 2.0)), _damped_metal(9), gamma=3e6,
                          lambdas=(500.0, 600.0, 700.0), weights=(1.0, 0.5, 2.0), src_comp=0, steps=3400)
    elif case == "per_sample_layout":
        o, rho = _problem(synth.lorentz_dielectric(5, 1, (1.5, 1.5, 2.0)), _damped_metal(9), gamma=3e6,
                          lambdas=(550.0, 650.0), src_comp=0, layout=1)
    else:
        diel = {"eps_inf": [4.0, 4.0, 4.0], "sigma": [0.0] * 3, "poles": [[], [], []]}
        o, rho = _problem(vacuum(), diel, steps=2500)
    dF, proj, _ = _adjoint_vs_tangent(o, rho)
    assert abs(dF) > 0
    # the lossless dielectric rings longest in this 5-cell CPML box: its window truncation error is
    # about 1e-5 (the same case's finite-difference check carries the same tolerance)
    tol = 1e-4 if case == "non_dispersive" else 1e-8
    assert abs(proj - dF) <= tol * abs(dF), (proj, dF)


def _paper_case(m2, n=20, steps=2000, seed=3):
    d = base_desc(n, n, n, n_steps=steps, cpml=4, precision=64, design=(8, 8, 8), gap=(2, 2, 2),
                  lambdas_nm=(600.0,), src_kind=0, src_comp=2, src_pos=(n // 2 - 5, n // 2, n // 2))
    rho = synth.uniform_rho(synth.box_shape(d["design_box"]), seed, 0.2, 0.8)
    o = oracle.Oracle(d)
    o.set_materials(vacuum(), vacuum(), m2, 0.0)
    o.set_density(rho)
    return o, rho


def _mat(eps, sig):
    m = vacuum()
    m["eps_inf"] = [eps] * 3
    m["sigma"] = [sig] * 3
    return m


@pytest.mark.parametrize("case", ["eps_inf", "sigma", "lorentz", "drude_lorentz"])
def test_paper_mode_gradient_vs_tangent_linear(case):
    """Paper mode (Eq. (Gradient_FDTD) from stored histories, the time-domain energy objective of Eq.
    (Objective_analyitically_enhancement)) projected on a seeded direction, against the exact
    forward-mode derivative of the same discrete objective.  The eps_inf and sigma terms are exact
    under either pairing of the pole term; the pole term paired with one adjoint level is exact once
    the fields and pole currents have decayed by the end of the window (the derivation's assumption;
    the metal's Drude current needs 8000 steps here, at 2000 it is 0.6% off), while the printed
    average of two levels stays off: 2e-4 for the Lorentz dielectric, 28% for the Drude-Lorentz metal."""
    m2 = {"eps_inf": _mat(4.0, 0.0), "sigma": _mat(1.0, 2e5), "lorentz": synth.lorentz_dielectric(4, 2),
          "drude_lorentz": synth.drude_lorentz_metal(3, 2)}[case]
    o, rho = _paper_case(m2, steps=8000 if case == "drude_lorentz" else 2000)
    printed, single = o.paper_gradient(1)[1], o.paper_gradient(5)[1]
    drho = np.random.default_rng(3).standard_normal(rho.shape)
    Ft, dFt = o.tangent(drho, time_domain=True)
    assert Ft > 0 and dFt != 0
    err_p = abs(np.sum(printed * drho) / dFt - 1)
    err_s = abs(np.sum(single * drho) / dFt - 1)
    if case in ("eps_inf", "sigma"):
        assert err_p <= 1e-8 and err_s <= 1e-8, (err_p, err_s)
    elif case == "lorentz":
        assert err_s <= 1e-8 and 1e-6 < err_p < 1e-2, (err_p, err_s)
    else:
        assert err_s <= 1e-8 and 0.2 < err_p < 0.35, (err_p, err_s)
