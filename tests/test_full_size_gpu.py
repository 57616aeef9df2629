"""Config 2 at its full size (256^3 grid, 12-cell CPML, 128^3 design box, smooth seeded density, air |
3-pair metal, FP32 fields with FP64 DFTs) in the launch configuration the benchmark times (fused
interior kernel, shell kernels, design-E kernel, 16-step CUDA graphs), checked against the oracle on
sampled outputs.

A Yee step reaches one cell further, so after N steps every field is zero farther than N cells from
the sources.  With a point dipole inside the design box and N = 24 steps, every nonzero value of the
forward run (and of the adjoint run, driven at the gap next to it) lies inside a 101^3 box around the
dipole, and the oracle run on that box alone, walled by PEC that the fields never reach, computes the
same values; the GPU fields outside it must be exactly zero.  The pulse is short (it rises within the
window) and the objective has one frequency, so that the adjoint basis stays well conditioned over 24
steps.
"""
import numpy as np
import pytest

import synth
from synth import C0

pytestmark = pytest.mark.gpu

N = 24
DIPOLE = (120, 128, 128)
R = 2 * N + 2


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


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


def _workload():
    w = synth.workload("c2")
    d = dict(w["desc"])
    dt = d["courant"] * d["dx"] / C0
    d.update(n_steps=N, src_kind=0, src_comp=2, src_pos=list(DIPOLE), freqs_hz=[C0 / 600e-9],
             freq_weights=[1.0], src_fwhm_hz=2.0e15, src_t0=12 * dt, adj_tau=4 * dt, src_wave=None)
    w["desc"] = d
    return w


def _crop(w):
    """The oracle's box: R cells around the dipole, no CPML, design box and gap shifted into it."""
    d = dict(w["desc"])
    lo = [c - R for c in DIPOLE]
    n = 2 * R + 1
    db, gb = d["design_box"], d["gap_box"]
    cdb, cgb = [], []
    for a in range(3):
        cdb += [max(db[2 * a], lo[a]) - lo[a], min(db[2 * a + 1], lo[a] + n) - lo[a]]
        cgb += [gb[2 * a] - lo[a], gb[2 * a + 1] - lo[a]]
        assert db[2 * a] <= lo[a] + n and gb[2 * a] >= lo[a] + N + 2 and gb[2 * a + 1] <= lo[a] + n - N - 2
    d.update(nx=n, ny=n, nz=n, cpml=[0] * 6, design_box=cdb, gap_box=cgb, src_pos=[R, R, R])
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
