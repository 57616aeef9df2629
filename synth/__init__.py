"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the oracle.

This module only *draws* inputs: density fields, CCPR pole/residue sets and
grid descriptions shaped like the paper's gap-antenna problems (Sec. 2 and
Sec. 4.3 of arXiv 2305.00234).  It holds none of the method's arithmetic: no
permittivity evaluation, no update coefficients, no time stepping, no DFT.

Conventions of the drawn values:
  * materials are dicts ``{"eps_inf": [3], "sigma": [3], "poles": [[(a, c), ...] x3]}``
    with complex ``a`` (rad/s, Re a < 0) and ``c`` (1/s) per Cartesian component, in the
    e^{j omega t} convention of the CCPR model (Eq. 1).  Each (a, c) stands for one
    complex-conjugate pair.
  * grid descriptions are dicts whose keys mirror ``fdtd_grid_desc`` of the C-ABI.
  * density arrays are float64, shape (dnz, dny, dnx) (x fastest), values in [0, 1].
"""
from __future__ import annotations

import math

import numpy as np

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)

SEED_BASE = 2305


# ----------------------------------------------------------------------------------------------
# Materials
# ----------------------------------------------------------------------------------------------

def vacuum():
    return {"eps_inf": [1.0, 1.0, 1.0], "sigma": [0.0, 0.0, 0.0], "poles": [[], [], []]}


def _isotropic(eps_inf, sigma, poles):
    return {"eps_inf": [float(eps_inf)] * 3, "sigma": [float(sigma)] * 3,
            "poles": [list(poles), list(poles), list(poles)]}


def _lorentz_pair(rng, re_rng=(1e14, 3e15), im_rng=(3e15, 7e15), d_eps=(0.3, 3.0)):
    """One passive Lorentz oscillator d_eps*w0^2/(w0^2 + j w G - w^2) written as a CCPR pair.

    The drawn half-width g = G/2 and resonance nu give the pole a = -g + j nu; the residue of a
    Lorentz term at that pole is purely imaginary, c = -j d_eps w0^2 / (2 nu) with
    w0^2 = nu^2 + g^2, so the pair is passive by construction.
    """
    g = rng.uniform(*re_rng)
    nu = rng.uniform(*im_rng)
    de = rng.uniform(*d_eps)
    w0sq = nu * nu + g * g
    a = complex(-g, nu)
    c = complex(0.0, -de * w0sq / (2.0 * nu))
    return a, c


def drude_lorentz_metal(seed, n_pairs, eps_inf=1.0):
    """Drude-like metal in the visible range: one real Drude pole plus (n_pairs-1) Lorentz pairs.

    The Drude part is sigma/(j w eps0) + 2 c1/(j w - a1) with a1 = -Gamma, c1 = -wp^2/(2 Gamma)
    and sigma = eps0 wp^2/Gamma (so sigma = -2 eps0 c1, the relation the paper's Au column obeys).
    Ranges bracket the paper's fitted metals (Table 1): a1 in -[1e14, 6e14], c1 in about -[1e17, 1e18].
    """
    rng = np.random.default_rng(seed)
    wp = rng.uniform(1.0e16, 1.4e16)
    gam = rng.uniform(1.0e14, 6.0e14)
    sigma = EPS0 * wp * wp / gam
    poles = [(complex(-gam, 0.0), complex(-wp * wp / (2.0 * gam), 0.0))]
    for _ in range(n_pairs - 1):
        poles.append(_lorentz_pair(rng))
    return _isotropic(eps_inf, sigma, poles)


def lorentz_dielectric(seed, n_pairs, eps_inf=(11.7, 11.7, 12.1)):
    """Lossy Lorentz dielectric with diagonal anisotropic eps_inf (same poles on every axis)."""
    rng = np.random.default_rng(seed)
    poles = [_lorentz_pair(rng, re_rng=(1e14, 1e15), im_rng=(5e15, 8e15), d_eps=(0.2, 1.0))
             for _ in range(n_pairs)]
    return {"eps_inf": [float(e) for e in eps_inf], "sigma": [0.0, 0.0, 0.0],
            "poles": [list(poles), list(poles), list(poles)]}


# CCPR parameters printed in the paper's Table 1 (Sec. 1).  Column 1 is headed "Ag" while the text
# names Al; it is kept as printed.  TiO2 is uniaxial: the ordinary column on x and y, the
# extraordinary one on z (Sec. 3 aligns eps_e with the z-polarised excitation).
def table_material(name):
    j = 1j
    if name == "Al":
        return _isotropic(3.07, 1.49e7, [(-1.89e14 + 0 * j, -1.00e18 + 0 * j),
                                         (-5.46e14 - 6.37e15 * j, 1.30e15 + 1.54e15 * j),
                                         (-5.68e14 - 3.43e14 * j, 1.61e17 + 1.00e12 * j)])
    if name == "Au":
        return _isotropic(2.31, 1.21e7, [(-1.28e14 + 0 * j, -6.85e17 + 0 * j),
                                         (-6.36e14 - 3.89e15 * j, 2.06e15 + 8.70e14 * j),
                                         (-2.96e15 - 6.12e15 * j, 1.60e13 + 1.47e16 * j)])
    if name == "Si":
        return _isotropic(1.0, 0.0, [(-8.00e14 + 6.39e15 * j, 7.31e14 - 2.89e16 * j),
                                     (-2.32e14 + 5.12e15 * j, 4.68e15 - 4.55e15 * j)])
    if name == "TiO2":
        po = [(0.0 - 6.65e15 * j, 0.0 + 1.01e16 * j)]
        pe = [(0.0 - 6.49e15 * j, 0.0 + 1.29e16 * j)]
        return {"eps_inf": [2.87, 2.87, 3.26], "sigma": [0.0, 0.0, 0.0], "poles": [po, po, pe]}
    raise KeyError(name)


def n_poles(mat):
    return [len(p) for p in mat["poles"]]


# ----------------------------------------------------------------------------------------------
# Density fields
# ----------------------------------------------------------------------------------------------

def uniform_rho(shape, seed, lo=0.0, hi=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape).astype(np.float64)


def smooth_rho(shape, seed, sigma_vox=3.0):
    """U[0,1] noise -> Gaussian filter (sigma in voxels, truncated at 3 sigma, edge-replicate)
    -> min-max rescaled to [0, 1]."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, size=shape)
    y = gaussian_filter(x, sigma=sigma_vox, mode="nearest", truncate=3.0)
    lo, hi = float(y.min()), float(y.max())
    return ((y - lo) / (hi - lo)).astype(np.float64)


# ----------------------------------------------------------------------------------------------
# Grid descriptions
# ----------------------------------------------------------------------------------------------

def centred_box(n, d):
    """Half-open [lo, hi) per axis of an edge-d box centred in an n-cell axis, as 6 ints."""
    out = []
    for nn, dd in zip(n, d):
        lo = (nn - dd) // 2
        out += [lo, lo + dd]
    return out


def base_desc(nx, ny, nz, *, dx=5e-9, courant=0.99 / math.sqrt(3.0), n_steps=1000, cpml=8,
              precision=32, design=None, gap=None, lambdas_nm=(600.0,), weights=None,
              src_kind=0, src_comp=2, src_pos=None, src_amp=1.0, bc=(0, 0, 0)):
    n = (nx, ny, nz)
    cp = [cpml] * 6 if np.isscalar(cpml) else list(cpml)
    design_box = centred_box(n, design) if design is not None else [0] * 6
    gap_box = centred_box(n, gap) if gap is not None else [0] * 6
    f0 = C0 / 600e-9
    fwhm = C0 / 500e-9 - C0 / 700e-9
    freqs = [C0 / (l * 1e-9) for l in lambdas_nm]
    w = list(weights) if weights is not None else [1.0] * len(freqs)
    if src_pos is None:
        src_pos = [nx // 2, ny // 2, nz // 2]
    return {"nx": nx, "ny": ny, "nz": nz, "dx": dx, "courant": courant, "n_steps": n_steps,
            "cpml": cp, "cpml_m": 3.0, "cpml_sigma_scale": 1.0, "cpml_kappa_max": 1.0,
            "cpml_a_max": 0.05, "bc": list(bc), "precision": precision,
            "design_box": design_box, "gap_box": gap_box,
            "freqs_hz": freqs, "freq_weights": w,
            "src_kind": src_kind, "src_comp": src_comp, "src_pos": list(src_pos),
            "src_f0": f0, "src_fwhm_hz": fwhm, "src_t0": 0.0, "src_amp": src_amp, "adj_tau": 0.0,
            "src_wave": None, "density_layout": 0}


def sinc_hann_wave(n_steps, dt, f_c=576.5e12, rel_bw=0.5, lobes=3):
    """The paper's excitation (Sec. "Optimization setup", Fig. "Signal"): a sinc envelope truncated to
    `lobes` zero crossings either side of its peak, times a Hanning window over the same span,
    modulating a carrier f_c (576.5 THz, the centre of the 350-1000 nm window).  The sinc's spectrum
    is a rectangle of full width rel_bw * f_c (~50% at half maximum).  Sampled at t = s dt / 2,
    s = 0 .. 2 n_steps, the half-step grid the solvers read (src_wave)."""
    B = rel_bw * f_c
    half = lobes / B                      # sinc(B x) vanishes at x = k / B
    x = np.arange(2 * n_steps + 1) * (dt / 2.0) - half
    win = np.where(np.abs(x) <= half, 0.5 * (1.0 + np.cos(np.pi * x / half)), 0.0)
    return np.sinc(B * x) * win * np.sin(2.0 * np.pi * f_c * x)


def paper_workload(material="Au", seed=None, n_freq=8, n_steps=None, pad=15, cpml=20, design=(25, 100, 100),
                   gap=(25, 6, 6), precision=32, gamma=5e4, density_layout=1):
    """The paper's own optimisation setup (Sec. "Optimization setup" and "Technical details"):
    Omega_d 100 x 25 x 100 and Omega_g 6 x 25 x 6 Yee cells, z-polarised plane wave along y carrying
    the truncated-sinc pulse, 20-cell CPML, dx = 2 nm (Al, Au) or 5 nm (Si, TiO2), dt = dx / (2 c0),
    18000 (metals) or 10000 (dielectrics) steps, air | Table-1 material.  Here x and y are exchanged
    (the plane wave travels along +x through the TF/SF plane; every Table-1 material has equal x and y
    components), `pad` air cells separate the design box from the CPML (the paper gives none), and
    the time-domain energy objective is represented by n_freq frequencies evenly spaced over
    350-1000 nm with equal weights (a uniform quadrature of its spectrum by Parseval).  As in the
    paper: the damping gamma = 5e4 of Eq. (sigma_mixed) for every material, and one density per E
    sample (density_layout 1, the N~_k count of Sec. "FDTD implementation and design export"), drawn
    from one smooth field on the design box grown by one cell so that the three components' samples
    of a voxel see neighbouring values."""
    idx = {"Al": 11, "Au": 12, "Si": 13, "TiO2": 14}[material]
    seed = SEED_BASE + idx if seed is None else seed
    metal = material in ("Al", "Au")
    dx = 2e-9 if metal else 5e-9
    M = n_steps if n_steps is not None else (18000 if metal else 10000)
    nx = 2 * (cpml + pad) + design[0]
    nx += (-nx) % 4                       # x rows of a multiple of 16 bytes (fused interior kernel)
    ny = 2 * (cpml + pad) + design[1]
    nz = 2 * (cpml + pad) + design[2]
    f = np.linspace(C0 / 1000e-9, C0 / 350e-9, n_freq)
    d = base_desc(nx, ny, nz, dx=dx, courant=0.5, n_steps=M, cpml=cpml, precision=precision, design=design,
                  gap=gap, lambdas_nm=tuple(C0 / f * 1e9), src_kind=1, src_pos=(cpml + 2, 0, 0))
    dt = 0.5 * dx / C0
    d["src_wave"] = sinc_hann_wave(M, dt)
    d["density_layout"] = density_layout
    nz_, ny_, nx_ = box_shape(d["design_box"])
    if density_layout == 1:   # E_x, E_y, E_z sample sets: (z, y, x) extents grown by one off their own axis
        field = smooth_rho((nz_ + 1, ny_ + 1, nx_ + 1), seed + 1000, 3.0)
        rho = np.concatenate([field[:nz_ + 1, :ny_ + 1, :nx_].ravel(), field[:nz_ + 1, :ny_, :nx_ + 1].ravel(),
                              field[:nz_, :ny_ + 1, :nx_ + 1].ravel()])
    else:
        rho = smooth_rho((nz_, ny_, nx_), seed + 1000, 3.0)
    return dict(desc=d, bg=vacuum(), m1=vacuum(), m2=table_material(material), gamma=gamma, rho=rho, seed=seed)


def box_shape(box):
    """(dnz, dny, dnx) of a half-open 6-int box."""
    return (box[5] - box[4], box[3] - box[2], box[1] - box[0])


def workload(name, seed=None):
    """The five paper-shaped workloads.  Returns dict(desc, bg, m1, m2, gamma, rho, seed)."""
    idx = {"c1": 1, "c2": 2, "c3": 3, "c4": 4}[name]
    seed = SEED_BASE + idx if seed is None else seed
    if name == "c1":
        # 32^3, dx = 5 nm, 8-cell CPML, 1000 steps, FP64; z-dipole at E_z(16,16,16+1/2);
        # 16^3 design [8,24)^3, 2^3 gap [15,17)^3, U[0,1] density, vacuum | 2-pair Drude metal.
        d = base_desc(32, 32, 32, n_steps=1000, cpml=8, precision=64, design=(16, 16, 16),
                      gap=(2, 2, 2), src_kind=0, src_comp=2, src_pos=(16, 16, 16))
        m2 = drude_lorentz_metal(seed, 2)
        rho = uniform_rho(box_shape(d["design_box"]), seed + 1000)
        return dict(desc=d, bg=vacuum(), m1=vacuum(), m2=m2, gamma=0.0, rho=rho, seed=seed)
    if name == "c2":
        # 256^3, 12-cell CPML, 4000 steps, FP32; 128^3 design, smooth density; air | 3-pair
        # metal; F = 3 (500/600/700 nm); TF/SF plane wave along +x two cells inside the CPML.
        d = base_desc(256, 256, 256, n_steps=4000, cpml=12, precision=32, design=(128, 128, 128),
                      gap=(2, 2, 2), lambdas_nm=(500.0, 600.0, 700.0), src_kind=1,
                      src_pos=(14, 0, 0))
        m2 = drude_lorentz_metal(seed, 3)
        rho = smooth_rho(box_shape(d["design_box"]), seed + 1000, 3.0)
        return dict(desc=d, bg=vacuum(), m1=vacuum(), m2=m2, gamma=0.0, rho=rho, seed=seed)
    if name == "c3":
        d = base_desc(512, 512, 384, n_steps=6000, cpml=16, precision=32,
                      design=(256, 256, 192), gap=(2, 2, 2), lambdas_nm=(500.0, 600.0, 700.0),
                      src_kind=1, src_pos=(18, 0, 0))
        m1 = lorentz_dielectric(seed + 7, 2)
        m2 = drude_lorentz_metal(seed, 4)
        rho = smooth_rho(box_shape(d["design_box"]), seed + 1000, 3.0)
        return dict(desc=d, bg=vacuum(), m1=m1, m2=m2, gamma=0.0, rho=rho, seed=seed)
    if name == "c4":
        d = base_desc(64, 64, 64, n_steps=2000, cpml=8, precision=32, design=(32, 32, 32),
                      gap=(2, 2, 2), src_kind=0, src_comp=2, src_pos=(32, 32, 32))
        m2 = drude_lorentz_metal(seed, 2)
        rho = uniform_rho(box_shape(d["design_box"]), seed + 1000, 0.2, 0.8)
        return dict(desc=d, bg=vacuum(), m1=vacuum(), m2=m2, gamma=0.0, rho=rho, seed=seed)
    raise KeyError(name)


def scaled_workload(name, n, n_steps, seed=None):
    """The same workload recipe on an n^3 grid (design = n/2 per axis, CPML scaled down)."""
    w = workload(name, seed)
    d = w["desc"]
    cp = max(4, min(d["cpml"][0], n // 8))
    nd = n // 2
    src_pos = (cp + 2, 0, 0) if d["src_kind"] == 1 else (n // 2, n // 2, n // 2)
    lam = tuple(C0 / f * 1e9 for f in d["freqs_hz"])
    d2 = base_desc(n, n, n, dx=d["dx"], courant=d["courant"], n_steps=n_steps, cpml=cp,
                   precision=d["precision"], design=(nd, nd, nd), gap=(2, 2, 2), lambdas_nm=lam,
                   src_kind=d["src_kind"], src_comp=d["src_comp"], src_pos=src_pos)
    shape = box_shape(d2["design_box"])
    rng_seed = w["seed"] + 1000
    if name in ("c2", "c3"):
        rho = smooth_rho(shape, rng_seed, 3.0)
    elif name == "c4":
        rho = uniform_rho(shape, rng_seed, 0.2, 0.8)
    else:
        rho = uniform_rho(shape, rng_seed)
    return dict(desc=d2, bg=w["bg"], m1=w["m1"], m2=w["m2"], gamma=w["gamma"], rho=rho,
                seed=w["seed"])


def serving_stream(seed=SEED_BASE + 5, n_requests=200, rate_hz=20.0,
                   sizes=(48, 64, 96, 128, 192), steps=(1500, 4000), pairs=(1, 4)):
    """Poisson stream of gradient requests (serving workload).  Each request: cubic grid n^3,
    n_steps, m2 with P pole pairs (m1 vacuum), design edge U[0.4, 0.6]*n per axis (centred),
    8-cell CPML, z-dipole at the centre, 2^3 gap, 600 nm objective, seeded U[0,1] density."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        n = int(rng.choice(sizes))
        m = int(rng.integers(steps[0], steps[1] + 1))
        p = int(rng.integers(pairs[0], pairs[1] + 1))
        ded = [max(4, int(round(rng.uniform(0.4, 0.6) * n))) for _ in range(3)]
        d = base_desc(n, n, n, n_steps=m, cpml=8, precision=32, design=tuple(ded), gap=(2, 2, 2),
                      src_kind=0, src_comp=2, src_pos=(n // 2, n // 2, n // 2))
        m2 = drude_lorentz_metal(seed * 1000 + r, p)
        rho = uniform_rho(box_shape(d["design_box"]), seed * 1000 + r + 7)
        out.append(dict(t_arrival=t, desc=d, bg=vacuum(), m1=vacuum(), m2=m2, gamma=0.0,
                        rho=rho, id=r))
    return out
