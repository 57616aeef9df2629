"""GPU (CUDA C-ABI) vs FP64 oracle, element by element, on seeded inputs.

Tolerances: relative L2 <= 1e-4 for the FP32 build, <= 1e-10 for the FP64 build (fields, DFTs,
objective, gradient); integer maps bit-exact.
"""
import math

import numpy as np
import pytest

import synth
from parity_util import TOL, box_rim, check_array, field_regions, rel
from synth import base_desc, vacuum

pytestmark = pytest.mark.gpu


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


def run_oracle(w, adjoint=True):
    import oracle
    o = oracle.problem(w)
    F, gap = o.forward()
    out = {"F": F, "gap": gap, "fields": [o.get_field(c) for c in range(6)], "dft": o.get_dft(),
           "maps": [o.get_index_map(q) for q in range(4)], "desc": w["desc"]}
    if adjoint:
        o.adjoint()
        out["adft"] = o.get_dft(True)
        out["grad"] = o.gradient()
    o.close()
    return out


def run_gpu(lib, w, adjoint=True, rho=None):
    p = lib.Problem(w["desc"], w["bg"], w["m1"], w["m2"], w.get("gamma", 0.0))
    p.set_density(w["rho"] if rho is None else rho)
    F, gap = p.forward()
    out = {"F": F, "gap": gap, "fields": [p.field(c) for c in range(6)], "dft": p.dft(),
           "maps": [p.index_map(q) for q in range(4)], "p": p}
    if adjoint:
        p.adjoint()
        out["adft"] = p.dft(True)
        out["grad"] = p.gradient()
    return out


def compare(g, o, prec, adjoint=True, per_voxel=True):
    """Integer maps bitwise; fields, DFTs, objective and gradient by whole-array relative L2, largest
    local error and per-region errors (parity_util.check_array)."""
    tol = TOL[prec]
    for q in range(4):
        assert np.array_equal(g["maps"][q], o["maps"][q]), f"index map {q}"
    regions = field_regions(o["desc"])
    # E and H compared as vector fields (a component can vanish by symmetry, e.g. H_z of a z-dipole)
    for name, sl in (("E", slice(0, 3)), ("H", slice(3, 6))):
        if g["fields"][sl.start] is not None:
            check_array(name, np.stack(g["fields"][sl]), np.stack(o["fields"][sl]), tol, regions)
    rim = [("design-box rim", box_rim(o["dft"].shape[2:]))]
    check_array("forward DFT", g["dft"], o["dft"], tol, rim)
    check_array("gap DFT", g["gap"], o["gap"], tol)
    assert abs(g["F"] - o["F"]) <= tol * abs(o["F"])
    if adjoint:
        check_array("adjoint DFT", g["adft"], o["adft"], tol, rim)
        check_array("gradient", g["grad"], o["grad"], tol, rim if per_voxel else ())
        if per_voxel:
            gap_design_idx = o["maps"][2][o["maps"][3] >= 0]
            assert np.all(g["grad"].ravel()[gap_design_idx] == 0.0)


def ragged_tfsf(prec, steps=500, seed=11):
    """C2-shaped case on a ragged 44x40x36 grid: TF/SF plane wave, 3 frequencies, smooth density,
    air | 3-pair metal (several (32, 8) tiles plus partial ones)."""
    d = base_desc(44, 40, 36, n_steps=steps, cpml=(6, 5, 4, 6, 5, 4), precision=prec,
                  design=(20, 18, 16), gap=(2, 2, 2), lambdas_nm=(500.0, 600.0, 700.0),
                  weights=(1.0, 0.7, 1.3), src_kind=1, src_pos=(8, 0, 0))
    rho = synth.smooth_rho(synth.box_shape(d["design_box"]), seed, 2.0)
    return dict(desc=d, bg=vacuum(), m1=vacuum(), m2=synth.drude_lorentz_metal(seed, 3), gamma=0.0, rho=rho)


def two_dispersive(prec, steps=400, seed=5, gamma=2e6):
    """C3-shaped case: anisotropic 2-pair Lorentz dielectric | 4-pair metal, gamma damping."""
    d = base_desc(40, 36, 34, n_steps=steps, cpml=5, precision=prec, design=(18, 16, 14),
                  gap=(2, 2, 2), lambdas_nm=(500.0, 600.0, 700.0), src_kind=0, src_comp=0,
                  src_pos=(20, 18, 17))
    rho = synth.uniform_rho(synth.box_shape(d["design_box"]), seed)
    m1 = synth.lorentz_dielectric(seed + 1, 2, eps_inf=(11.7, 11.7, 12.1))
    return dict(desc=d, bg=vacuum(), m1=m1, m2=synth.drude_lorentz_metal(seed, 4), gamma=gamma, rho=rho)


@pytest.mark.parametrize("src", ["tfsf", "dipole_shell", "dipole_interior"])
@pytest.mark.parametrize("prec,nx,fused", [(32, 52, 1), (32, 45, 0), (64, 46, 1), (64, 45, 0), (32, 72, 1), (64, 72, 1)])
def test_step_paths(gpu, prec, nx, fused, src):
    """Both background-step layouts: an interior box for the fused TMA kernel (x rows a multiple of
    16 bytes) plus the shell kernels around it, and the shell kernels over the whole grid.  Grids
    ragged in all three tile axes, CPML of unequal thickness, a 3-pair metal whose design box
    straddles the interior box, and the TF/SF plane inside the interior box or a dipole in the shell or
    in the interior box.  nx = 72: the interior box ends in a partial tile column (26 of 32 cells) and,
    like nx = 52, a partial tile row (14 of 16 rows)."""
    kw = {"tfsf": dict(src_kind=1, src_pos=(9, 0, 0)),
          "dipole_shell": dict(src_kind=0, src_comp=1, src_pos=(8, 33, 6)),
          "dipole_interior": dict(src_kind=0, src_comp=2, src_pos=(12, 8, 8))}[src]
    d = base_desc(nx, 42, 37, n_steps=420, cpml=(6, 5, 4, 7, 5, 3), precision=prec,
                  design=(22, 18, 15), gap=(2, 2, 2), lambdas_nm=(500.0, 650.0), **kw)
    rho = synth.smooth_rho(synth.box_shape(d["design_box"]), 23, 2.0)
    w = dict(desc=d, bg=vacuum(), m1=vacuum(), m2=synth.drude_lorentz_metal(23, 3), gamma=1e6, rho=rho)
    g = run_gpu(gpu, w)
    t = g["p"].timings()
    assert t["fused_step"] == fused
    assert t["pdl_graphs"] == 1                    # phases linked by programmatic dependent launch edges
    compare(g, run_oracle(w), prec)


@pytest.mark.parametrize("material", ["Si", "Au"])
def test_paper_workload_reduced(gpu, material):
    """The paper's own setup (z-polarised plane wave carrying the truncated sinc x Hanning pulse,
    Table-1 material in air, dt = dx/(2 c0), gamma = 5e4, one density per E sample, design box thin
    along the propagation axis, gap spanning it) on a reduced grid with an interior box: design 24 x 32 x 32, gap 24 x 4 x 4, 8-cell CPML,
    2400 steps, 4 objective frequencies over 350-1000 nm."""
    w = synth.paper_workload(material, design=(24, 32, 32), gap=(24, 4, 4), pad=10, cpml=8, n_steps=2400,
                             n_freq=4)
    w["desc"]["adj_tau"] = 1.0e-15
    assert w["desc"]["density_layout"] == 1 and w["gamma"] == 5e4    # the paper's layout and damping
    g = run_gpu(gpu, w)
    assert g["p"].timings()["fused_step"] == 1
    compare(g, run_oracle(w), 32, per_voxel=False)


@pytest.mark.parametrize("prec", [64, 32])
def test_config1_full(gpu, prec):
    """Config 1 at its full size: 32^3 FP64, 1000 steps, dipole, 2-pair metal, 16^3 design."""
    w = synth.workload("c1")
    w["desc"]["precision"] = prec
    compare(run_gpu(gpu, w), run_oracle(w), prec)


@pytest.mark.parametrize("prec", [32, 64])
def test_ragged_tfsf_three_frequencies(gpu, prec):
    w = ragged_tfsf(prec)
    compare(run_gpu(gpu, w), run_oracle(w), prec)


@pytest.mark.parametrize("prec", [32, 64])
def test_two_dispersive_materials_gamma(gpu, prec):
    w = two_dispersive(prec)
    compare(run_gpu(gpu, w), run_oracle(w), prec)


def test_config4_shape(gpu):
    w = synth.scaled_workload("c4", 40, 600)
    compare(run_gpu(gpu, w), run_oracle(w), 32)


@pytest.mark.parametrize("m1,m2,prec", [("Si", "Au", 32), ("TiO2", "Au", 32), ("TiO2", "Al", 64)])
def test_paper_table_materials(gpu, m1, m2, prec):
    """Table 1 fits (Al/Au/Si/TiO2; TiO2 anisotropic with lossless poles) as design materials.
    The printed first column (Al, headed Ag) has sigma + 2 eps0 c1 < 0, a negative instantaneous
    conductivity that makes the FP32 update stiff; it is checked in the FP64 build."""
    d = base_desc(36, 36, 36, dx=2e-9, courant=0.5, n_steps=600, cpml=6, precision=prec,
                  design=(16, 16, 16), gap=(2, 2, 2), lambdas_nm=(450.0, 700.0), src_pos=(18, 18, 18))
    w = dict(desc=d, bg=vacuum(), m1=synth.table_material(m1), m2=synth.table_material(m2), gamma=5e4,
             rho=synth.uniform_rho((16, 16, 16), 3))
    compare(run_gpu(gpu, w), run_oracle(w), prec)


@pytest.mark.parametrize("value", [0.0, 1.0])
def test_density_endpoints(gpu, value):
    w = two_dispersive(32, steps=300)
    w["rho"] = np.full(synth.box_shape(w["desc"]["design_box"]), value)
    compare(run_gpu(gpu, w), run_oracle(w), 32)


def test_many_poles_and_frequencies(gpu):
    """16 poles on a component (the maximum) and 8 objective frequencies (the maximum), evenly
    spaced 350-850 THz with a window long enough to separate them (adjoint basis cond ~ 8)."""
    lam = tuple(synth.C0 / np.linspace(350e12, 850e12, 8) * 1e9)
    d = base_desc(24, 24, 24, n_steps=2000, cpml=4, precision=32, design=(10, 10, 10), gap=(2, 2, 2),
                  lambdas_nm=lam, src_pos=(12, 12, 12))
    d["adj_tau"] = 3e-15
    m1 = synth.lorentz_dielectric(8, 8, eps_inf=(2.0, 2.5, 3.0))
    m2 = synth.drude_lorentz_metal(9, 8)
    w = dict(desc=d, bg=vacuum(), m1=m1, m2=m2, gamma=1e6, rho=synth.uniform_rho((10, 10, 10), 2))
    # after 2000 steps the fields have decayed to a small tail, so the field check is made on a
    # 500-step run; DFTs, objective and gradient come from the full run
    g, o = run_gpu(gpu, w), run_oracle(w)
    g["fields"], o["fields"] = [None] * 6, [None] * 6
    ws = dict(w, desc=dict(d, n_steps=500))
    g["fields"] = run_gpu(gpu, ws, adjoint=False)["fields"]
    o["fields"] = run_oracle(ws, adjoint=False)["fields"]
    compare(g, o, 32)


def test_small_grid_and_single_voxel_design(gpu):
    d = base_desc(8, 9, 10, n_steps=200, cpml=2, precision=64, design=(1, 1, 1), gap=None,
                  src_pos=(4, 4, 5))
    w = dict(desc=d, bg=vacuum(), m1=vacuum(), m2=synth.drude_lorentz_metal(1, 2), gamma=0.0,
             rho=np.array([[[0.4]]]))
    compare(run_gpu(gpu, w, adjoint=False), run_oracle(w, adjoint=False), 64, adjoint=False)


def test_gap_fills_design_box(gpu):
    """All design voxels are gap: no blended voxel, gradient identically zero."""
    d = base_desc(16, 16, 16, n_steps=200, cpml=3, precision=32, design=(2, 2, 2), gap=(2, 2, 2),
                  src_pos=(8, 8, 8))
    w = dict(desc=d, bg=vacuum(), m1=vacuum(), m2=synth.drude_lorentz_metal(1, 2), gamma=0.0,
             rho=np.full((2, 2, 2), 0.5))
    g, o = run_gpu(gpu, w), run_oracle(w)
    compare(g, o, 32)
    assert np.all(g["grad"] == 0.0)


def test_device_density_and_device_gradient(gpu):
    torch = pytest.importorskip("torch")
    w = ragged_tfsf(32, steps=300)
    o = run_oracle(w)
    for dt in (torch.float32, torch.float64):
        rho_t = torch.tensor(w["rho"], dtype=dt, device="cuda")
        p = gpu.Problem(w["desc"], w["bg"], w["m1"], w["m2"], 0.0,
                        stream=torch.cuda.current_stream().cuda_stream)
        p.set_density(rho_t)
        F, _ = p.forward()
        p.adjoint()
        g = torch.zeros(p.dshape, dtype=dt, device="cuda")
        p.gradient(g)
        torch.cuda.synchronize()
        assert rel(g.double().cpu().numpy(), o["grad"]) <= 1e-4
        assert abs(F - o["F"]) <= 1e-4 * o["F"]
        p.close()


def test_repeat_runs_are_deterministic(gpu):
    w = ragged_tfsf(32, steps=300)
    p = gpu.problem(w)
    F1, g1 = p.forward()
    p.adjoint()
    G1 = p.gradient()
    n1 = p.gradient_norm2()
    F2, g2 = p.forward()
    p.adjoint()
    G2 = p.gradient()
    assert F1 == F2 and np.array_equal(g1, g2) and np.array_equal(G1, G2)
    assert n1 == pytest.approx(float(np.sum(G1 * G1)), rel=1e-12)


def test_errors_and_call_order(gpu):
    from paper_2305_00234_gb300 import FdtdError
    w = ragged_tfsf(32, steps=400)
    p = gpu.Problem(w["desc"], w["bg"], w["m1"], w["m2"])
    with pytest.raises(FdtdError) as e:
        p.forward()
    assert e.value.status == 4                       # density not set
    bad = w["rho"].copy()
    bad[0, 0, 0] = 1.5
    with pytest.raises(FdtdError) as e:
        p.set_density(bad)
    assert e.value.status == 1
    bad[0, 0, 0] = np.nan
    with pytest.raises(FdtdError):
        p.set_density(bad)
    torch = pytest.importorskip("torch")
    with pytest.raises(FdtdError) as e:
        p.set_density(torch.tensor(bad, device="cuda"))
    assert e.value.status == 1
    with pytest.raises(FdtdError):
        p.set_density(w["rho"][:-1])
    p.set_density(w["rho"])
    with pytest.raises(FdtdError) as e:
        p.adjoint()
    assert e.value.status == 4
    p.forward()
    p.adjoint()
    p.gradient()
    p.close()
    # too many poles on one component
    with pytest.raises(FdtdError):
        gpu.Problem(w["desc"], vacuum(), synth.lorentz_dielectric(1, 9), synth.drude_lorentz_metal(1, 8))
    # dispersive background is rejected
    with pytest.raises(FdtdError):
        gpu.Problem(w["desc"], synth.drude_lorentz_metal(1, 1), vacuum(), vacuum())


def test_ill_conditioned_adjoint_basis_is_refused(gpu):
    """8 frequencies 50 nm apart cannot be separated in a 300-step window: FDTD_ERR_ARG, not noise."""
    from paper_2305_00234_gb300 import FdtdError
    d = base_desc(24, 24, 24, n_steps=300, cpml=4, precision=32, design=(10, 10, 10), gap=(2, 2, 2),
                  lambdas_nm=tuple(np.linspace(450, 800, 8)), src_pos=(12, 12, 12))
    p = gpu.Problem(d, vacuum(), vacuum(), synth.drude_lorentz_metal(9, 2))
    p.set_density(synth.uniform_rho((10, 10, 10), 2))
    p.forward()
    with pytest.raises(FdtdError) as e:
        p.adjoint()
    assert e.value.status == 1 and "ill-conditioned" in str(e.value)
    p.close()


def test_unstable_run_is_reported(gpu):
    from paper_2305_00234_gb300 import FdtdError
    w = ragged_tfsf(32, steps=200)
    w["desc"]["src_amp"] = 1e36                        # overflows FP32 in the first steps
    p = gpu.problem(w)
    with pytest.raises(FdtdError) as e:
        p.forward()
    assert e.value.status == 5
    with pytest.raises(FdtdError):
        p.forward()                                   # the handle is dead
    p.close()


def test_cancel_flag_resets_per_call(gpu):
    w = ragged_tfsf(32, steps=100)
    p = gpu.problem(w)
    gpu.fdtd_cancel(p.h)          # a cancel before the call does not stick to the next run
    F, _ = p.forward()
    assert F > 0
    p.close()


@pytest.mark.parametrize("src", ["tfsf_odd", "tfsf_even", "dipole_shell_odd", "dipole_shell_even", "per_sample"])
def test_paired_shell_paths(gpu, src):
    """The paired FP32 shell kernels (two x-adjacent cells per thread): x CPML of even thickness on an even
    grid, so that the shell boxes' x bounds are even; the design box's x bounds odd (pairs straddle the
    working box in the shell E kernel), the TF/SF plane on either cell of a pair, a dipole in the shell on
    either cell of a pair, and the per-sample density layout (working box grown by one on +x)."""
    kw = {"tfsf_odd": dict(src_kind=1, src_pos=(9, 0, 0)), "tfsf_even": dict(src_kind=1, src_pos=(10, 0, 0)),
          "dipole_shell_odd": dict(src_kind=0, src_comp=2, src_pos=(43, 20, 6)),
          "dipole_shell_even": dict(src_kind=0, src_comp=1, src_pos=(4, 33, 18)),
          "per_sample": dict(src_kind=1, src_pos=(9, 0, 0))}[src]
    d = base_desc(52, 42, 37, n_steps=420, cpml=(6, 4, 4, 7, 5, 3), precision=32,
                  design=(21, 18, 15), gap=(2, 2, 2), lambdas_nm=(500.0, 650.0), **kw)
    assert d["design_box"][0] % 2 == 1
    rho = synth.smooth_rho(synth.box_shape(d["design_box"]), 23, 2.0)
    w = dict(desc=d, bg=vacuum(), m1=vacuum(), m2=synth.drude_lorentz_metal(23, 3), gamma=1e6, rho=rho)
    per_voxel = src != "per_sample"
    if not per_voxel:
        w = per_sample(w, 31)
    g = run_gpu(gpu, w)
    t = g["p"].timings()
    assert t["fused_step"] == 1 and t["paired_shell"] == 1
    assert t["paired_design"] == 0                 # odd working-box x origin: the one-sample design kernel
    compare(g, run_oracle(w), 32, per_voxel=per_voxel)


@pytest.mark.parametrize("case", ["gap_odd", "gap_even", "tfsf_in_design_odd", "tfsf_in_design_even",
                                  "poles8", "no_poles", "per_sample"])
def test_paired_design_paths(gpu, case):
    """The paired FP32 design-E kernel (two x-adjacent samples per thread): an even grid with the design
    box's x origin and extent even; the gap box (the adjoint run's sources) and the forward dipole on
    either sample of a pair, the TF/SF plane through the design box on either sample of a pair, 6 and
    0 poles a component, and the per-sample density layout (working box grown by one on +x, E_x samples
    of its last x column outside their sample box)."""
    gap = (4, 2, 2) if case == "gap_even" else (2, 2, 2)
    kw = {"gap_odd": dict(src_kind=0, src_comp=2, src_pos=(27, 21, 18)),
          "gap_even": dict(src_kind=0, src_comp=0, src_pos=(25, 21, 18)),
          "tfsf_in_design_odd": dict(src_kind=1, src_pos=(23, 0, 0)),
          "tfsf_in_design_even": dict(src_kind=1, src_pos=(30, 0, 0))}.get(case, dict(src_kind=1, src_pos=(9, 0, 0)))
    design = (23, 18, 15) if case == "per_sample" else (24, 18, 15)
    d = base_desc(56, 42, 37, n_steps=420, cpml=(6, 4, 4, 7, 5, 3), precision=32,
                  design=design, gap=gap, lambdas_nm=(500.0, 650.0), **kw)
    rho = synth.smooth_rho(synth.box_shape(d["design_box"]), 41, 2.0)
    m1, m2 = vacuum(), synth.drude_lorentz_metal(41, 3)
    if case == "poles8":
        m1 = synth.lorentz_dielectric(42, 2, eps_inf=(11.7, 11.7, 12.1))
        m2 = synth.drude_lorentz_metal(41, 4)
    if case == "no_poles":
        m2 = dict(vacuum(), eps_inf=[4.0, 4.5, 5.0], sigma=[2e5, 2e5, 2e5])
    w = dict(desc=d, bg=vacuum(), m1=m1, m2=m2, gamma=1e6, rho=rho)
    if case == "per_sample":
        w = per_sample(w, 43)
    db, gb = w["desc"]["design_box"], w["desc"]["gap_box"]
    assert db[0] % 2 == 0 and (db[1] - db[0] + (case == "per_sample")) % 2 == 0
    assert gb[0] % 2 == (case != "gap_even")
    g = run_gpu(gpu, w)
    t = g["p"].timings()
    assert t["paired_design"] == 1 and t["fused_step"] == 1
    compare(g, run_oracle(w), 32, per_voxel=case != "per_sample")


def per_sample(w, seed):
    """The same case with one density per E sample (density_layout 1): a seeded vector of
    N~ = sum_k prod_l (N_l + 1 - delta_kl) values (Sec. "FDTD implementation and design export")."""
    w = dict(w, desc=dict(w["desc"], density_layout=1))
    db = w["desc"]["design_box"]
    N = (db[1] - db[0], db[3] - db[2], db[5] - db[4])
    n = sum(int(np.prod([N[l] + 1 - (k == l) for l in range(3)])) for k in range(3))
    w["rho"] = synth.uniform_rho((n,), seed)
    return w


@pytest.mark.parametrize("prec,nx,fused", [(32, 52, 1), (64, 45, 0)])
def test_per_sample_density(gpu, prec, nx, fused):
    """density_layout 1 on a ragged grid, Lorentz dielectric | metal with gamma damping: the
    working box (design box grown on its +x/+y/+z faces) straddles the interior box of the fused
    step; fields, DFTs over the working box, objective and the per-sample gradient against the
    oracle, gap samples exactly zero."""
    d = base_desc(nx, 42, 37, n_steps=420, cpml=(6, 5, 4, 7, 5, 3), precision=prec,
                  design=(21, 17, 15), gap=(2, 2, 2), lambdas_nm=(500.0, 650.0), src_kind=0,
                  src_comp=1, src_pos=(12, 8, 8))
    m1 = synth.lorentz_dielectric(3, 2, eps_inf=(11.7, 11.7, 12.1))
    w = per_sample(dict(desc=d, bg=vacuum(), m1=m1, m2=synth.drude_lorentz_metal(23, 3), gamma=5e4), 29)
    g, o = run_gpu(gpu, w), run_oracle(w)
    assert g["p"].timings()["fused_step"] == fused
    assert g["grad"].shape == o["grad"].shape == w["rho"].shape
    compare(g, o, prec, per_voxel=False)
    assert (o["grad"] == 0.0).sum() == 3 * 8 and np.all(g["grad"][o["grad"] == 0.0] == 0.0)
    g["p"].close()
    if prec == 32:   # device-resident density and gradient
        torch = pytest.importorskip("torch")
        from paper_2305_00234_gb300 import FdtdError
        p = gpu.Problem(w["desc"], w["bg"], w["m1"], w["m2"], w["gamma"],
                        stream=torch.cuda.current_stream().cuda_stream)
        with pytest.raises(FdtdError):
            p.set_density(w["rho"][:-1])
        p.set_density(torch.tensor(w["rho"], dtype=torch.float32, device="cuda"))
        with pytest.raises(FdtdError) as e:     # paper mode takes one density per voxel
            p.paper_forward()
        assert e.value.status == 1
        F, _ = p.forward()
        p.adjoint()
        gt = torch.zeros(p.dshape, dtype=torch.float32, device="cuda")
        p.gradient(gt)
        torch.cuda.synchronize()
        assert rel(gt.double().cpu().numpy(), o["grad"]) <= 1e-4
        assert abs(F - o["F"]) <= 1e-4 * o["F"]
        p.close()
