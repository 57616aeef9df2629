"""Pins of the FP64 oracle to facts other than itself (closed forms, exact discrete identities,
finite differences, reciprocity, printed numbers).  CPU only.

Every test names the passage of arXiv 2305.00234 it pins.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from synth import C0, EPS0, MU0, base_desc, vacuum

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _oracle(desc, bg=None, m1=None, m2=None, gamma=0.0, rho=None):
    import oracle
    o = oracle.Oracle(desc)
    o.set_materials(bg or vacuum(), m1 or vacuum(), m2 or vacuum(), gamma)
    if rho is not None:
        o.set_density(rho)
    return o


def _grid_coords(n):
    nz, ny, nx = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return [i.astype(float), j.astype(float), k.astype(float)]


# ----------------------------------------------------------------------------------------------
# Yee leapfrog in vacuum ("FDTD implementation and design export"): an exact discrete PEC-cavity
# eigenmode evolves as cos(w n dt) with (sin(w dt/2)/(c dt))^2 = sum_l (sin(k_l dx/2)/dx)^2.
# One test per polarisation covers every curl term of both half-steps.
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("p", [0, 1, 2])
def test_vacuum_cavity_eigenmode(p):
    nx, ny, nz = 12, 10, 14
    dx = 10e-9
    d = base_desc(nx, ny, nz, dx=dx, courant=0.9 / math.sqrt(3), n_steps=1000, cpml=0,
                  precision=64, src_amp=0.0)
    o = _oracle(d)
    N = [nx, ny, nz]
    q, r = (p + 1) % 3, (p + 2) % 3
    kq, kr = 1 * math.pi / (N[q] * dx), 2 * math.pi / (N[r] * dx)
    sq, sr = 2 * math.sin(kq * dx / 2) / dx, 2 * math.sin(kr * dx / 2) / dx
    S2 = sq * sq + sr * sr
    dt = o.dt
    w = 2 * math.asin(C0 * dt * math.sqrt(S2) / 2) / dt
    L = _grid_coords(o.n)
    Ep = np.sin(kq * L[q] * dx) * np.sin(kr * L[r] * dx)
    wh = 2 * EPS0 / dt * math.sin(w * dt / 2) ** 2
    Hq = (sr * wh / S2) * np.sin(kq * L[q] * dx) * np.cos(kr * (L[r] + 0.5) * dx)
    Hr = (-sq * wh / S2) * np.cos(kq * (L[q] + 0.5) * dx) * np.sin(kr * L[r] * dx)
    o.set_field(p, Ep)
    o.set_field(3 + q, Hq)
    o.set_field(3 + r, Hr)
    nsteps = 1000
    o.step(0, nsteps, 0)
    E = o.get_field(p)
    assert np.abs(E - math.cos(w * nsteps * dt) * Ep).max() <= 1e-12
    for c in range(3):
        if c != p:
            assert np.abs(o.get_field(c)).max() <= 1e-14


# ----------------------------------------------------------------------------------------------
# Conductivity term of Eq. (Maxwells2)a: a uniform (k = 0) field in a periodic lossy box decays
# by exactly (eps0 eps/dt - sigma/2)/(eps0 eps/dt + sigma/2) per step.
# ----------------------------------------------------------------------------------------------
def test_uniform_field_conductive_decay():
    d = base_desc(4, 4, 4, cpml=0, bc=(1, 1, 1), n_steps=10, precision=64, src_amp=0.0)
    bg = {"eps_inf": [2.0, 3.0, 4.0], "sigma": [1e6, 2e6, 5e5], "poles": [[], [], []]}
    o = _oracle(d, bg=bg)
    dt = o.dt
    init = [1.0, -2.0, 0.5]
    for c in range(3):
        o.set_field(c, np.full(o.n, init[c]))
    o.step(0, 200, 0)
    for c in range(3):
        e, s = bg["eps_inf"][c], bg["sigma"][c]
        ratio = (EPS0 * e / dt - s / 2) / (EPS0 * e / dt + s / 2)
        np.testing.assert_allclose(o.get_field(c), init[c] * ratio ** 200, rtol=1e-12, atol=0)
        assert np.abs(o.get_field(3 + c)).max() == 0.0


# ----------------------------------------------------------------------------------------------
# Lossy cavity: a PEC-cavity mode in a conductive medium follows the two-variable mode recurrence
# (mode amplitude e, curl amplitude w); its per-step energy ratio is (D-)/(D+) and the continuous
# decay rate of the E part is sigma/(eps0 eps).
# ----------------------------------------------------------------------------------------------
def test_lossy_cavity_mode_decay():
    nx, ny, nz = 10, 12, 6
    dx = 10e-9
    bg = {"eps_inf": [1.5] * 3, "sigma": [3e4] * 3, "poles": [[], [], []]}
    d = base_desc(nx, ny, nz, dx=dx, cpml=0, n_steps=10, precision=64, src_amp=0.0)
    o = _oracle(d, bg=bg)
    dt = o.dt
    kx, ky = math.pi / (nx * dx), math.pi / (ny * dx)
    sx, sy = 2 * math.sin(kx * dx / 2) / dx, 2 * math.sin(ky * dx / 2) / dx
    L = _grid_coords(o.n)
    pat = np.sin(kx * L[0] * dx) * np.sin(ky * L[1] * dx)
    o.set_field(2, pat)
    nsteps = 600
    o.step(0, nsteps, 0)
    eps, sig = 1.5 * EPS0, 3e4
    Dp, Dm = eps / dt + sig / 2, eps / dt - sig / 2
    e, w = 1.0, 0.0
    amps = []
    for _ in range(nsteps):
        w = w - dt / MU0 * (sx * sx + sy * sy) * e
        e = (Dm * e + w) / Dp
        amps.append(e)
    Ez = o.get_field(2)
    np.testing.assert_allclose(Ez, amps[-1] * pat, rtol=0, atol=1e-12 * np.abs(pat).max())
    # characteristic roots of the recurrence: |lambda|^2 = Dm/Dp  (energy ratio per step)
    lam = np.roots([Dp, -(2 * eps / dt - dt / MU0 * (sx * sx + sy * sy)), Dm])
    assert abs(abs(lam[0]) ** 2 - Dm / Dp) < 1e-13
    assert abs(-math.log(Dm / Dp) / dt - sig / eps) / (sig / eps) < (sig * dt / eps) ** 2


# ----------------------------------------------------------------------------------------------
# CCPR pole recursion (Eq. (Maxwells2)b, Eq. (CCPRModel)).  An E sample driven by a pulse in its
# curl: (1) the recovered transfer function equals 1/Y(z) of the discrete recursion exactly;
# (2) Y(z)/(j w eps0) recovers the paper's continuous CCPR permittivity with its Table 1
# parameters to O((w dt)^2).
# ----------------------------------------------------------------------------------------------
def _ccpr_eps(mat, comp, w):
    e = mat["eps_inf"][comp] + mat["sigma"][comp] / (1j * w * EPS0)
    for a, c in mat["poles"][comp]:
        e += c / (1j * w - a) + np.conj(c) / (1j * w - np.conj(a))
    return e


def _discrete_Y(m1, m2, comp, rho, gamma, dt, z):
    eps = (1 - rho) * m1["eps_inf"][comp] + rho * m2["eps_inf"][comp]
    sig = (1 - rho) * m1["sigma"][comp] + rho * m2["sigma"][comp] + rho * (1 - rho) * gamma
    Y = EPS0 * eps * (z - 1) + sig * dt * (z + 1) / 2
    for kap, mat in ((1 - rho, m1), (rho, m2)):
        for a, c in mat["poles"][comp]:
            al = np.exp(a * dt)
            be = EPS0 * c * (al - 1) / (2 * a)
            h = be * (z + 1) / (z - al) + np.conj(be) * (z + 1) / (z - np.conj(al))
            Y += kap * (z - 1) * h
    return Y / dt


def _recovered_eps(o, mat, comp, courant_scale, lams):
    """Drive one sample with a zero-mean pulse in its curl; return (|Ehat Y/S - 1|, eps_rec) per
    wavelength.  The drive sits at half steps, so its transform carries z^{-1/2}."""
    dt = o.dt
    M = int(60000 * courant_scale)
    t = (np.arange(M) + 0.5) * dt
    tau, t0 = 0.3e-15, 1.5e-15
    g = np.exp(-((t - t0) ** 2) / (2 * tau * tau))
    curl = np.diff(g, prepend=0.0)       # drive^{n+1/2}: sums to g[-1] = 0, so no static remainder
    e = o.sample_response(comp, 1.0, curl)                                # E^{n+1}, n = 0..M-1
    assert abs(e[-1]) < 1e-12 * np.abs(e).max()
    out = []
    n = np.arange(M)
    for lam_nm in lams:
        w = 2 * math.pi * C0 / (lam_nm * 1e-9)
        z = np.exp(1j * w * dt)
        S = np.sum(curl * z ** (-n * 1.0))
        Ehat = np.sum(e * z ** (-(n + 1.0)))
        Y = _discrete_Y(vacuum(), mat, comp, 1.0, 0.0, dt, z)
        out.append((abs(Ehat * Y / S - 1), z ** -0.5 * S / (Ehat * 1j * w * EPS0), w))
    return out


@pytest.mark.parametrize("name,comp", [("Au", 0), ("Al", 1), ("Si", 2)])
def test_ccpr_recovered_from_pulse(name, comp):
    mat = synth.table_material(name)
    lams = (350.0, 500.0, 600.0, 1000.0)
    errs = []
    for scale in (1, 2):
        d = base_desc(8, 8, 8, dx=2e-9, courant=0.5 / scale, precision=64, design=(2, 2, 2), cpml=0)
        o = _oracle(d, m1=vacuum(), m2=mat)
        res = _recovered_eps(o, mat, comp, scale, lams)
        row = []
        for (disc, eps_rec, w) in res:
            assert disc < 1e-9                       # exactly the discrete transfer 1/Y(z)
            eps_ccpr = _ccpr_eps(mat, comp, w)
            scale_terms = abs(mat["eps_inf"][comp]) + abs(mat["sigma"][comp] / (w * EPS0)) + sum(
                abs(c / (1j * w - a)) + abs(np.conj(c) / (1j * w - np.conj(a)))
                for a, c in mat["poles"][comp])
            err = abs(eps_rec - eps_ccpr)
            assert err < (w * o.dt) ** 2 * scale_terms   # Eq. (CCPRModel) to O((w dt)^2)
            row.append(err)
        errs.append(row)
    for e1, e2 in zip(*errs):                          # halving dt quarters the error
        assert 3.5 < e1 / e2 < 4.5


def test_blended_sample_is_discrete_Y_of_interpolated_model():
    """Eqs. (eps_mixed), (sigma_mixed), (Poles_mixed): both materials' poles kept, weighted by
    1-rho and rho; sigma gets rho(1-rho)gamma."""
    m1, m2 = synth.table_material("Si"), synth.table_material("Au")
    d = base_desc(8, 8, 8, dx=2e-9, courant=0.5, precision=64, design=(2, 2, 2), cpml=0)
    gamma = 2e6
    o = _oracle(d, m1=m1, m2=m2, gamma=gamma)
    dt = o.dt
    M = 60000
    curl = np.zeros(M)
    curl[0], curl[1] = 1.0, -1.0          # zero-sum drive: no static field left in Si (sigma = 0)
    for rho in (0.0, 0.37, 1.0):
        e = o.sample_response(2, rho, curl)
        for lam_nm in (450.0, 700.0):
            z = np.exp(1j * 2 * math.pi * C0 / (lam_nm * 1e-9) * dt)
            Ehat = np.sum(e * z ** (-(np.arange(M) + 1.0)))
            assert abs(Ehat * _discrete_Y(m1, m2, 2, rho, gamma, dt, z) / (1 - 1 / z) - 1) < 1e-9


# ----------------------------------------------------------------------------------------------
# Density endpoints (Eqs. (eps_mixed)-(Poles_mixed)): rho = 0 with (X, Y) and rho = 1 with (Y, X)
# are the same pure-X run, bit for bit; the gradients are exact negatives.
# ----------------------------------------------------------------------------------------------
def test_density_endpoints_bitwise():
    X = synth.drude_lorentz_metal(3, 2)
    Y = synth.lorentz_dielectric(4, 2, eps_inf=(2.0, 2.5, 3.0))
    d = base_desc(14, 14, 14, dx=10e-9, n_steps=300, cpml=4, precision=64, design=(6, 6, 6),
                  gap=(2, 2, 2), src_pos=(7, 7, 7))
    shape = synth.box_shape(d["design_box"])
    a = _oracle(d, m1=X, m2=Y, rho=np.zeros(shape))
    b = _oracle(d, m1=Y, m2=X, rho=np.ones(shape))
    Fa, ga = a.forward()
    Fb, gb = b.forward()
    assert Fa == Fb
    for c in range(6):
        assert np.array_equal(a.get_field(c), b.get_field(c))
    assert np.array_equal(a.get_dft(), b.get_dft())
    a.adjoint()
    b.adjoint()
    Ga, Gb = a.gradient(), b.gradient()
    np.testing.assert_allclose(Ga, -Gb, rtol=1e-11, atol=1e-11 * np.abs(Ga).max())


# ----------------------------------------------------------------------------------------------
# Adjoint gradient vs central finite differences of the oracle's own discrete objective
# (Sec. "Time-domain adjoint formulation", Eq. (Gradient_analytic)).  Small CPML-bounded grids
# whose fields decay inside the window, so the frequency-domain adjoint is exact up to the tail.
# ----------------------------------------------------------------------------------------------
def _damped_metal(seed):
    m = synth.drude_lorentz_metal(seed, 2)
    poles = []
    for comp in range(3):
        (a1, c1), (a2, c2) = m["poles"][comp]
        poles.append([(complex(-8e14, 0.0), 0.5 * c1), (complex(-1e15, a2.imag), c2)])
    m["poles"] = poles
    m["sigma"] = [-2 * EPS0 * poles[0][0][1].real] * 3
    return m


def _fd_case(m2, m1=None, gamma=0.0, lambdas=(600.0,), weights=None, steps=3000, src_comp=2):
    d = base_desc(20, 20, 20, dx=20e-9, n_steps=steps, cpml=5, precision=64, design=(8, 8, 8),
                  gap=(2, 2, 2), src_kind=0, src_comp=src_comp, src_pos=(10, 10, 10),
                  lambdas_nm=lambdas, weights=weights)
    rho = synth.uniform_rho(synth.box_shape(d["design_box"]), 11, 0.2, 0.8)
    return d, rho, _oracle(d, m1=m1 or vacuum(), m2=m2, gamma=gamma, rho=rho)


def _check_fd(o, rho, voxels, h=1e-4, rtol=2e-5):
    o.set_density(rho)
    o.forward()
    o.adjoint()
    g = o.gradient()
    scale = np.abs(g).max()
    for v in voxels:
        r1 = rho.copy()
        r1[v] += h
        o.set_density(r1)
        Fp, _ = o.forward()
        r1[v] -= 2 * h
        o.set_density(r1)
        Fm, _ = o.forward()
        fd = (Fp - Fm) / (2 * h)
        assert abs(g[v] - fd) <= rtol * max(abs(fd), 1e-3 * scale), (v, g[v], fd)
    return g


FD_VOXELS = [(6, 5, 4), (2, 2, 0), (4, 4, 7), (1, 6, 3)]


def test_gradient_vs_finite_differences_dispersive_metal():
    d, rho, o = _fd_case(_damped_metal(7))
    _check_fd(o, rho, FD_VOXELS)


def test_gradient_vs_finite_differences_three_frequencies_and_gamma():
    """Several objective frequencies in one adjoint run (2F basis pulses) and the
    rho(1-rho) gamma damping of Eq. (sigma_mixed)."""
    d, rho, o = _fd_case(_damped_metal(9), m1=synth.lorentz_dielectric(5, 1, (1.5, 1.5, 2.0)),
                         gamma=3e6, lambdas=(500.0, 600.0, 700.0), weights=(1.0, 0.5, 2.0),
                         steps=3400, src_comp=0)
    _check_fd(o, rho, FD_VOXELS[:3], rtol=5e-5)


def test_nondispersive_special_case():
    """With all pole and conductivity terms zero only the eps_inf term remains (Sec. "Time-domain
    adjoint formulation", the remark after Eq. (Gradient_analytic)); identical materials give a
    zero gradient."""
    diel = {"eps_inf": [4.0, 4.0, 4.0], "sigma": [0.0] * 3, "poles": [[], [], []]}
    d, rho, o = _fd_case(diel, steps=2500)
    g = _check_fd(o, rho, FD_VOXELS[:2], rtol=1e-4)
    o2 = _oracle(d, m1=_damped_metal(7), m2=_damped_metal(7), rho=rho)
    o2.forward()
    o2.adjoint()
    ref = np.abs(g).max()
    assert np.abs(o2.gradient()).max() <= 1e-12 * ref


# ----------------------------------------------------------------------------------------------
# Reciprocity of the discrete Yee + CPML + CCPR operator (needed by the adjoint run, SI Eq.
# (AdjointSystem)): dipole at A observed at B equals dipole at B observed at A, step by step.
# ----------------------------------------------------------------------------------------------
def test_reciprocity_dipole_swap():
    m2 = synth.drude_lorentz_metal(21, 2)
    base = dict(dx=10e-9, n_steps=400, cpml=4, precision=64, design=(8, 8, 8), gap=(2, 2, 2))
    A, ca = (5, 6, 7), 0
    B, cb = (9, 8, 6), 2
    da = base_desc(16, 16, 16, src_kind=0, src_comp=ca, src_pos=A, **base)
    db = base_desc(16, 16, 16, src_kind=0, src_comp=cb, src_pos=B, **base)
    rho = synth.uniform_rho(synth.box_shape(da["design_box"]), 5)
    oa = _oracle(da, m2=m2, rho=rho)
    ob = _oracle(db, m2=m2, rho=rho)
    oa.forward()
    ob.forward()
    lo = da["design_box"][0::2]
    Ga = oa.get_dft()[0, cb][B[2] - lo[2], B[1] - lo[1], B[0] - lo[0]]
    Gb = ob.get_dft()[0, ca][A[2] - lo[2], A[1] - lo[1], A[0] - lo[0]]
    assert abs(Ga - Gb) <= 1e-10 * abs(Ga)


# ----------------------------------------------------------------------------------------------
# One-sided TF/SF plane wave: in vacuum with periodic y/z walls the scattered-field region stays
# empty (the 1-D incident line has the 3-D grid's exact dispersion along x).
# ----------------------------------------------------------------------------------------------
def test_tfsf_no_leakage():
    # the +x end is a PEC wall far enough away that its echo cannot reach the plane in the window
    M = 1500
    d = base_desc(480, 2, 2, dx=5e-9, n_steps=M, cpml=(10, 0, 0, 0, 0, 0), bc=(0, 1, 1),
                  precision=64, src_kind=1, src_pos=(14, 0, 0))
    o = _oracle(d)
    peak_tf = 0.0
    peak_sf = 0.0
    for n in range(0, M, 50):
        o.step(n, 50, 1)
        Ez = o.get_field(2)
        peak_tf = max(peak_tf, np.abs(Ez[:, :, 14:400]).max())
        peak_sf = max(peak_sf, np.abs(Ez[:, :, 10:14]).max())
    assert peak_tf > 0.5
    assert peak_sf <= 1e-12 * peak_tf


# ----------------------------------------------------------------------------------------------
# A source waveform passed as samples (src_wave, p(s dt/2)) drives the same run as the built-in
# pulse it samples, for both source kinds; the paper's truncated-sinc pulse has the spectrum the
# setup section describes (carrier 576.5 THz, ~50% band at half maximum inside 350-1000 nm).
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [0, 1])
def test_src_wave_samples_equal_builtin_pulse(kind):
    M = 300
    d = base_desc(24, 20, 20, n_steps=M, cpml=4, precision=64, src_kind=kind, src_pos=(7, 10, 10))
    dt = d["courant"] * d["dx"] / C0
    tau = math.sqrt(2.0 * math.log(2.0)) / (math.pi * d["src_fwhm_hz"])
    t = np.arange(2 * M + 1) * dt / 2.0 - 4.0 * tau
    d2 = dict(d, src_wave=np.exp(-t * t / (2.0 * tau * tau)) * np.sin(2.0 * math.pi * d["src_f0"] * t))
    fields = []
    for dd in (d, d2):
        o = _oracle(dd)
        o.step(0, M, 1)
        fields.append([o.get_field(c) for c in range(6)])
        o.close()
    scale = max(np.max(np.abs(a)) for a in fields[0])
    assert scale > 0
    for a, b in zip(*fields):
        assert np.max(np.abs(a - b)) <= 1e-12 * scale


def test_paper_pulse_spectrum():
    dt = 0.5 * 2e-9 / C0
    wv = synth.sinc_hann_wave(18000, dt)[::2]
    sp = np.abs(np.fft.rfft(wv, 1 << 17))
    fr = np.fft.rfftfreq(1 << 17, dt)
    band = fr[sp >= sp.max() / 2]
    assert abs(0.5 * (band.min() + band.max()) - 576.5e12) < 0.01 * 576.5e12
    assert 0.45 < (band.max() - band.min()) / 576.5e12 < 0.55
    assert band.min() > C0 / 1000e-9 and band.max() < C0 / 350e-9


# ----------------------------------------------------------------------------------------------
# Normal-incidence reflection from a dispersive half-space (Table 1 gold): the measured
# reflection equals the exact discrete interface formula, and the continuous Fresnel coefficient
# (1-n)/(1+n) with n = sqrt(eps_CCPR) to the grid's discretisation error.
# ----------------------------------------------------------------------------------------------
def test_dispersive_half_space_reflection():
    nx, cp, i0, probe, m = 140, 20, 26, 23, 60
    M = 4000
    d = base_desc(nx, 2, 2, dx=5e-9, n_steps=M, cpml=(cp, cp, 0, 0, 0, 0), bc=(0, 1, 1),
                  precision=64, src_kind=1, src_pos=(i0, 0, 0))
    d["design_box"] = [m, nx - cp, 0, 2, 0, 2]
    au = synth.table_material("Au")
    o = _oracle(d, m2=au, rho=np.ones((2, 2, nx - cp - m)))
    dt, dx = o.dt, d["dx"]
    ts = np.zeros(M)
    for n in range(M):
        o.step(n, 1, 1)
        ts[n] = o.get_field(2)[0, 0, probe]
    einc = o.get_source(1)
    nn = np.arange(M)
    for lam_nm in (500.0, 600.0, 700.0):
        w = 2 * math.pi * C0 / (lam_nm * 1e-9)
        z = np.exp(1j * w * dt)
        Es = np.sum(ts * z ** (-(nn + 1.0)))
        Ei = np.sum(einc * z ** (-nn * 1.0))
        # discrete wave factors u = e^{-j k dx} from Y dx / g = u + 1/u - 2, g = dt/(mu0 dx (1 - 1/z))
        def u_of(Y):
            s = Y * MU0 * dx * dx * (1 - 1 / z) / dt
            r = np.roots([1.0, -(2.0 + s), 1.0])
            return r
        r1 = u_of(_discrete_Y(vacuum(), vacuum(), 2, 0.0, 0.0, dt, z))
        u1 = r1[np.argmin(r1.imag)]                   # forward wave: Im u < 0
        r2 = u_of(_discrete_Y(vacuum(), au, 2, 1.0, 0.0, dt, z))
        u2 = r2[np.argmin(np.abs(r2))]                # decaying into the metal
        ratio_meas = Es / Ei * u1 ** (probe + i0 - 2 * m)
        ratio_exact = (u2 - u1) / (u1 * (1 - u1 * u2))
        assert abs(ratio_meas - ratio_exact) < 2e-5
        nref = np.sqrt(_ccpr_eps(au, 2, w))
        fres = (1 - nref) / (1 + nref)
        # continuous Fresnel with the interface half a cell before the first metal node, to
        # second order in the cell size
        assert abs(ratio_exact * u1 - fres) < 2 * (w * dx / C0) ** 2


# ----------------------------------------------------------------------------------------------
# CPML ("surrounded by CPML layers", Methods): a dipole in a small CPML-bounded box sees the same
# field as in a box large enough that nothing returns within the window.
# ----------------------------------------------------------------------------------------------
def test_cpml_absorbs():
    """3-D: a dipole pulse in a 40^3 box with a 12-cell CPML against the same pulse in a 140^3 box without
    one, at a probe 3 cells from the source, over the 190 steps before the large box's PEC walls can echo
    back (round trip 140 cells at c dt / dx = 0.57 cells per step): what the CPML reflects, including its
    edges and corners at grazing incidence, stays below 2e-4 of the peak (measured 2.6e-5)."""
    M = 190

    def probe(n, cp):
        c = n // 2
        d = base_desc(n, n, n, dx=10e-9, n_steps=M, cpml=cp, precision=64, src_pos=(c, c, c))
        dt = d["courant"] * d["dx"] / C0
        d.update(src_fwhm_hz=2.0e15, src_t0=40 * dt)
        o = _oracle(d)
        ts = []
        for n0 in range(0, M, 2):
            o.step(n0, 2, 1)
            ts.append(o.get_field(2)[c, c, c + 3])
        o.close()
        return np.array(ts)

    small, big = probe(40, 12), probe(140, 0)
    assert np.abs(big).max() > 0
    assert np.abs(small - big).max() <= 2e-4 * np.abs(big).max()


def test_cpml_normal_incidence_reflection():
    """1-D: the TF/SF plane wave in a box periodic in y and z (so the fields are uniform there) hits the
    +x CPML at normal incidence; the field the CPML sends back into the scattered-field region, 3 cells
    before the plane, against the incident field 3 cells after it.  A graded CFS-CPML of 12 or 16 cells
    reflects below 1e-4 (measured 1.6e-5 and 6.8e-6), and the thicker layer reflects less.  A half-cell
    shift of the grading between the E and H positions reflects 6-8% here, a profile graded from the
    wrong side about 75%."""
    M = 1600
    r = {}
    for cp in (12, 16):
        i0 = cp + 20
        d = base_desc(2 * cp + 40, 4, 4, dx=10e-9, n_steps=M, cpml=(cp, cp, 0, 0, 0, 0), precision=64,
                      bc=(0, 1, 1), src_kind=1, src_pos=(i0, 0, 0))
        o = _oracle(d)
        refl, inc = [], []
        for n0 in range(M):
            o.step(n0, 1, 1)
            E = o.get_field(2)
            refl.append(E[2, 2, i0 - 3])
            inc.append(E[2, 2, i0 + 3])
        o.close()
        r[cp] = np.abs(refl).max() / np.abs(inc).max()
        assert 0 < r[cp] < 1e-4, (cp, r[cp])
    assert r[16] < r[12]


# ----------------------------------------------------------------------------------------------
# Adjoint source construction: the injected waveform's transform at every objective frequency
# equals w_f conj(Ehat_g(w_f)) at every gap sample (time reversal = conjugation, SI Eq.
# (AdjointSystem)a).
# ----------------------------------------------------------------------------------------------
def test_adjoint_source_spectrum():
    d = base_desc(16, 16, 16, dx=10e-9, n_steps=800, cpml=4, precision=64, design=(8, 8, 8),
                  gap=(2, 2, 2), src_pos=(8, 8, 8), lambdas_nm=(500.0, 600.0, 700.0),
                  weights=(1.0, 0.3, 2.0))
    rho = synth.uniform_rho(synth.box_shape(d["design_box"]), 3)
    o = _oracle(d, m2=synth.drude_lorentz_metal(2, 2), rho=rho)
    F, gap = o.forward()
    o.adjoint()
    S = o.get_source(3)                         # (3*ngap, M): drive S_g^{n+1/2}
    n = np.arange(d["n_steps"])
    gflat = gap.reshape(3, 3, -1)              # (F, comp, gap voxel)
    for f, fr in enumerate(d["freqs_hz"]):
        z = np.exp(1j * 2 * math.pi * fr * o.dt)
        spec = S @ (z ** (-n * 1.0))
        target = d["freq_weights"][f] * np.conj(gflat[f].reshape(-1))
        np.testing.assert_allclose(spec, target, rtol=1e-9, atol=1e-9 * np.abs(target).max())
    assert F == pytest.approx(sum(d["freq_weights"][f] * np.sum(np.abs(gflat[f]) ** 2)
                                  for f in range(3)), rel=1e-12)


# ----------------------------------------------------------------------------------------------
# Printed numbers (Methods, "Technical details of the optimization"): dt = 8.34e-3 fs at 5 nm and
# 3.34e-3 fs at 2 nm with 10000 / 18000 steps = 83.40 / 60.12 fs; both are dt = dx/(2 c0).
# ----------------------------------------------------------------------------------------------
def test_paper_time_steps():
    with open(os.path.join(GOLDEN, "paper_numbers.json")) as f:
        g = json.load(f)
    for row in g["time_discretisation"]:
        d = base_desc(8, 8, 8, dx=row["dx_m"], courant=0.5, cpml=0, precision=64)
        o = _oracle(d)
        assert o.dt == pytest.approx(row["dt_s"], rel=6e-3)
        assert o.dt * row["n_steps"] == pytest.approx(row["T_s"], rel=6e-3)
    au = g["au_drude"]
    assert -2 * EPS0 * au["c1_per_s"] == pytest.approx(au["sigma_S_per_m"], rel=5e-3)


# ----------------------------------------------------------------------------------------------
# Integer maps (voxel ownership, design/gap membership, PEC and CPML flags) against counts that
# follow from the definitions.
# ----------------------------------------------------------------------------------------------
def test_index_map_counts():
    d = base_desc(20, 18, 16, n_steps=10, cpml=(3, 4, 2, 5, 4, 3), precision=64,
                  design=(8, 6, 6), gap=(2, 2, 2), src_pos=(10, 9, 8))
    o = _oracle(d, m2=synth.drude_lorentz_metal(1, 1))
    m0 = o.get_index_map(0)
    nx, ny, nz = 20, 18, 16
    cls = m0 & 3
    assert (cls == 1).sum() == 3 * (8 * 6 * 6 - 8)
    assert (cls == 2).sum() == 3 * 8
    pec = (m0 >> 2) & 1
    # E_x fixed where j == 0 or k == 0, etc.
    assert pec[0].sum() == nx * (ny * nz - (ny - 1) * (nz - 1))
    assert pec[1].sum() == ny * (nx * nz - (nx - 1) * (nz - 1))
    assert pec[2].sum() == nz * (nx * ny - (nx - 1) * (ny - 1))
    assert ((m0 >> 5) & 1).sum() == 1 and (m0[2, 8, 9, 10] >> 5) & 1
    # E_x's first derivative axis is y: CPML at integer y positions j < 2 or j > 18 - 5
    flag = (m0[0] >> 3) & 1
    expect = ((np.arange(ny) < 2) | (np.arange(ny) > ny - 5))[None, :, None]
    assert np.array_equal(flag, np.broadcast_to(expect, flag.shape).astype(flag.dtype))
    # H_y's second derivative axis is x: half-integer positions i + 1/2 < 3 or > 20 - 4
    hflag = (o.get_index_map(1)[1] >> 4) & 1
    i = np.arange(nx) + 0.5
    expect = ((i < 3) | (i > nx - 4))[None, None, :]
    assert np.array_equal(hflag, np.broadcast_to(expect, hflag.shape).astype(hflag.dtype))
    dm = o.get_index_map(2)
    assert (dm >= 0).sum() == 8 * 6 * 6 and dm.max() == 8 * 6 * 6 - 1
    gm = o.get_index_map(3)
    assert sorted(gm[gm >= 0].tolist()) == list(range(8))
