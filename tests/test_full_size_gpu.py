"""Configs 2 and 3 and the paper's own workload at their full sizes, in the launch configuration the
benchmark times (fused interior kernel, shell kernels, design-E kernel, 16-step CUDA graphs),
checked against the oracle.

Config 2: 256^3 grid, 12-cell CPML, 128^3 design box, smooth seeded density, air | 3-pair metal, FP32
fields with FP64 DFTs.  Config 3: 512 x 512 x 384 grid, 16-cell CPML, 256 x 256 x 192 design box,
anisotropic 2-pair Lorentz dielectric | 4-pair metal (six poles per component: the 8-pole design
kernel).  Config 2 and 3 are checked on sampled outputs:

A Yee step reaches one cell further, so after N steps every field is zero farther than N cells from
the sources.  With a point dipole inside the design box and N = 24 steps, every nonzero value of the
forward run (and of the adjoint run, driven at the gap next to it) lies inside a 101^3 box around the
dipole, and the oracle run on that box alone, walled by PEC that the fields never reach, computes the
same values; the GPU fields outside it must be exactly zero.  The pulse is short (it rises within the
window) and the objective has one frequency, so that the adjoint basis stays well conditioned over 24
steps.

The paper's workload (96 x 170 x 170 cells, 20-cell CPML, Table-1 Au with gamma = 5e4, one density per E
sample, the sinc x Hanning plane wave) is small enough for the oracle to run the whole grid: it is
checked everywhere, over 300 steps in which the plane wave crosses the design box.
"""
import numpy as np
import pytest

import synth
from parity_util import TOL, box_rim, check_array, field_regions, rel
from synth import C0

pytestmark = pytest.mark.gpu

N = 24
DIPOLE = (120, 128, 128)
R = 2 * N + 2


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_00234_gb300 import build
    build.build()
    import paper_2305_00234_gb300 as lib
    lib.load_library()
    return lib


def _workload(name="c2", dipole=DIPOLE):
    w = synth.workload(name)
    d = dict(w["desc"])
    dt = d["courant"] * d["dx"] / C0
    d.update(n_steps=N, src_kind=0, src_comp=2, src_pos=list(dipole), freqs_hz=[C0 / 600e-9],
             freq_weights=[1.0], src_fwhm_hz=2.0e15, src_t0=12 * dt, adj_tau=4 * dt, src_wave=None)
    w["desc"] = d
    return w


def _crop(w, dipole=DIPOLE):
    """The oracle's box: R cells around the dipole, no CPML, design box and gap shifted into it."""
    d = dict(w["desc"])
    lo = [c - R for c in dipole]
    n = 2 * R + 1
    db, gb = d["design_box"], d["gap_box"]
    cdb, cgb = [], []
    for a in range(3):
        cdb += [max(db[2 * a], lo[a]) - lo[a], min(db[2 * a + 1], lo[a] + n) - lo[a]]
        cgb += [gb[2 * a] - lo[a], gb[2 * a + 1] - lo[a]]
        assert db[2 * a] <= lo[a] + n and gb[2 * a] >= lo[a] + N + 2 and gb[2 * a + 1] <= lo[a] + n - N - 2
    d.update(nx=n, ny=n, nz=n, cpml=[0] * 6, design_box=cdb, gap_box=cgb, src_pos=[R, R, R])
    for a in range(3):      # the CPML lies beyond the light cone
        assert w["desc"]["cpml"][2 * a] < lo[a] and lo[a] + n <= w["desc"]["n" + "xyz"[a]] - w["desc"]["cpml"][2 * a + 1]
    # density on the crop's design box, (z, y, x) offsets into the full design box
    sl = tuple(slice(cdb[2 * a] + lo[a] - db[2 * a], cdb[2 * a + 1] + lo[a] - db[2 * a]) for a in (2, 1, 0))
    return dict(w, desc=d, rho=np.ascontiguousarray(w["rho"][sl])), lo, sl


def test_config2_full_size_against_the_oracle_on_the_light_cone(gpu):
    import oracle
    w = _workload()
    p = gpu.Problem(w["desc"], w["bg"], w["m1"], w["m2"], w["gamma"])
    assert p.timings()["fused_step"] == 1               # the benchmark's interior + shell split
    p.set_density(w["rho"])
    F, _ = p.forward()
    fields = [p.field(c) for c in range(6)]
    dft = p.dft()
    p.adjoint()
    adft = p.dft(True)
    grad = p.gradient()
    p.close()

    wc, lo, sl = _crop(w)
    o = oracle.problem(wc)
    Fo, _ = o.forward()
    ofields = [o.get_field(c) for c in range(6)]
    odft = o.get_dft()
    o.adjoint()
    oadft = o.get_dft(True)
    ograd = o.gradient()
    o.close()

    n = 2 * R + 1
    box = (slice(lo[2], lo[2] + n), slice(lo[1], lo[1] + n), slice(lo[0], lo[0] + n))
    for name, s in (("E", slice(0, 3)), ("H", slice(3, 6))):
        g = np.stack([f[box] for f in fields[s]])
        assert np.abs(g).max() > 0
        assert rel(g, np.stack(ofields[s])) <= 1e-4, name
        for f in fields[s]:                             # nothing beyond the light cone
            f[box] = 0.0
            assert not f.any(), name
    assert abs(F - Fo) <= 1e-4 * abs(Fo) and Fo > 0
    assert rel(dft[(slice(None), slice(None)) + sl], odft) <= 1e-4
    assert rel(adft[(slice(None), slice(None)) + sl], oadft) <= 1e-4
    assert rel(grad[sl], ograd) <= 1e-4
    grad[sl] = 0.0
    assert not grad.any()


def test_config2_full_size_plane_wave_against_the_oracle(gpu):
    """The benchmark's own source at full size: the one-sided TF/SF plane at x = 14 (inside the x-wall
    shell box) launching the plane wave along x.  The field is uniform in y and z, so the oracle runs
    the full x extent (with the same 12-cell x CPML) on a y-z window of 101 x 101 cells, walled by PEC;
    after N steps the window's inner 53 x 53 columns, farther than N + 1 cells from those walls, match
    the full grid."""
    import oracle
    w = synth.workload("c2")
    d = dict(w["desc"])
    dt = d["courant"] * d["dx"] / C0
    d.update(n_steps=N, src_fwhm_hz=2.0e15, src_t0=12 * dt, adj_tau=4 * dt, freqs_hz=[C0 / 600e-9],
             freq_weights=[1.0])
    w = dict(w, desc=d)
    p = gpu.Problem(d, w["bg"], w["m1"], w["m2"], w["gamma"])
    assert p.timings()["fused_step"] == 1
    p.set_density(w["rho"])
    p.forward()
    fields = [p.field(c) for c in range(6)]
    p.close()

    n = 2 * R + 1
    c0 = 128 - R                                        # window origin in y and z
    dc = dict(d, ny=n, nz=n, cpml=[12, 12, 0, 0, 0, 0], design_box=[0] * 6, gap_box=[0] * 6)
    o = oracle.Oracle(dc)
    o.set_materials(w["bg"], w["m1"], w["m2"], w["gamma"])
    o.forward()
    ofields = [o.get_field(c) for c in range(6)]
    o.close()
    inner = slice(N + 2, n - N - 2)
    g = np.stack([f[c0 + N + 2:c0 + n - N - 2, c0 + N + 2:c0 + n - N - 2, :] for f in fields])
    ref = np.stack([f[inner, inner, :] for f in ofields])
    assert np.abs(g[2]).max() > 0                       # E_z carries the wave
    for name, s in (("E", slice(0, 3)), ("H", slice(3, 6))):
        assert rel(g[s], ref[s]) <= 1e-4, name


def test_config3_full_size_against_the_oracle_on_the_light_cone(gpu):
    """Config 3 at full size (512 x 512 x 384, 16-cell CPML, 256 x 256 x 192 design box, anisotropic 2-pair
    Lorentz dielectric | 4-pair metal: six poles per component, the 8-pole design kernel): a dipole inside
    the design box, N steps, every nonzero value on the GPU inside the light-cone box the oracle runs.
    The fields come back on the device (fdtd_get_field with a device buffer) and are checked there."""
    import torch

    import oracle
    dip = (250, 256, 192)
    w = _workload("c3", dip)
    w["gamma"] = 3e6                                  # the damping term of Eq. (sigma_mixed) as well
    assert sum(len(p) for p in (w["m1"]["poles"][0], w["m2"]["poles"][0])) == 6
    d = w["desc"]
    shape = (d["nz"], d["ny"], d["nx"])
    p = gpu.Problem(d, w["bg"], w["m1"], w["m2"], w["gamma"], stream=torch.cuda.current_stream().cuda_stream)
    assert p.timings()["fused_step"] == 1
    p.set_density(w["rho"])
    F, _ = p.forward()
    n = 2 * R + 1
    lo = [c - R for c in dip]
    box = (slice(lo[2], lo[2] + n), slice(lo[1], lo[1] + n), slice(lo[0], lo[0] + n))
    fields = []
    buf = torch.empty(int(np.prod(shape)), dtype=torch.float64, device="cuda")
    for c in range(6):
        p.field(c, out=buf)
        f = buf.view(shape)
        fields.append(f[box].cpu().numpy())
        f[box] = 0.0                                  # nothing beyond the light cone
        assert float(f.abs().max()) == 0.0, c
    dft = p.dft()
    p.adjoint()
    adft = p.dft(True)
    grad = p.gradient()
    p.close()

    wc, lo2, sl = _crop(w, dip)
    assert lo2 == lo
    o = oracle.problem(wc)
    Fo, _ = o.forward()
    ofields = [o.get_field(c) for c in range(6)]
    odft = o.get_dft()
    o.adjoint()
    oadft = o.get_dft(True)
    ograd = o.gradient()
    o.close()

    tol = TOL[32]
    regions = field_regions(wc["desc"])
    for name, s_ in (("E", slice(0, 3)), ("H", slice(3, 6))):
        g = np.stack(fields[s_])
        assert np.abs(g).max() > 0
        check_array(name, g, np.stack(ofields[s_]), tol, regions)
    assert abs(F - Fo) <= tol * abs(Fo) and Fo > 0
    check_array("forward DFT", dft[(slice(None), slice(None)) + sl], odft, tol)
    check_array("adjoint DFT", adft[(slice(None), slice(None)) + sl], oadft, tol)
    check_array("gradient", grad[sl], ograd, tol)
    for a in (dft, adft):
        a[(slice(None), slice(None)) + sl] = 0.0
        assert not a.any()
    grad[sl] = 0.0
    assert not grad.any()


def test_paper_workload_full_size_against_the_oracle(gpu):
    """The paper's setup at full size (96 x 170 x 170 cells: design 25 x 100 x 100, gap 25 x 6 x 6, 20-cell
    CPML, 15 air cells, dt = dx / (2 c0), Table-1 Au with gamma = 5e4, one density per E sample), 300
    steps of the sinc x Hanning plane wave taken from its main lobe on (the run starts at the pulse's
    centre), one objective frequency; the oracle runs the same whole grid.  Fields, both DFTs over the
    working box, the objective, the per-sample gradient and the integer maps are compared everywhere."""
    import oracle
    w = synth.paper_workload("Au")
    d = dict(w["desc"])
    assert (d["nx"], d["ny"], d["nz"]) == (96, 170, 170) and d["density_layout"] == 1 and w["gamma"] == 5e4
    M = 300
    dt = d["courant"] * d["dx"] / C0
    centre = int(round(2 * 3.0 / (0.5 * 576.5e12) / dt))      # half-step sample of the sinc's peak
    wave = synth.sinc_hann_wave(centre // 2 + M + 1, dt)
    d.update(n_steps=M, src_wave=wave[centre:centre + 2 * M + 1], freqs_hz=[C0 / 350e-9], freq_weights=[1.0],
             adj_tau=40 * dt)
    w = dict(w, desc=d)
    p = gpu.Problem(d, w["bg"], w["m1"], w["m2"], w["gamma"])
    assert p.timings()["fused_step"] == 1
    p.set_density(w["rho"])
    F, gap = p.forward()
    fields = [p.field(c) for c in range(6)]
    dft = p.dft()
    maps = [p.index_map(q) for q in range(4)]
    p.adjoint()
    adft = p.dft(True)
    grad = p.gradient()
    p.close()

    o = oracle.problem(w)
    Fo, gapo = o.forward()
    ofields = [o.get_field(c) for c in range(6)]
    odft = o.get_dft()
    omaps = [o.get_index_map(q) for q in range(4)]
    o.adjoint()
    oadft = o.get_dft(True)
    ograd = o.gradient()
    o.close()

    tol = TOL[32]
    for q in range(4):
        assert np.array_equal(maps[q], omaps[q]), q
    regions = field_regions(d)
    for name, s_ in (("E", slice(0, 3)), ("H", slice(3, 6))):
        g = np.stack(fields[s_])
        assert np.abs(g[:, :, :, 40:]).max() > 1e-3 * np.abs(g).max()      # the wave reached the design box
        check_array(name, g, np.stack(ofields[s_]), tol, regions)
    assert abs(F - Fo) <= tol * abs(Fo) and Fo > 0
    rim = [("design-box rim", box_rim(odft.shape[2:]))]
    check_array("gap DFT", gap, gapo, tol)
    check_array("forward DFT", dft, odft, tol, rim)
    check_array("adjoint DFT", adft, oadft, tol, rim)
    check_array("gradient", grad, ograd, tol)
    assert grad.shape == w["rho"].shape and np.all(grad[ograd == 0.0] == 0.0)
