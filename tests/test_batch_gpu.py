"""Batched runs: several gradient evaluations of different grids advanced together by the persistent
kernel (fdtd_batch_*), against the oracle and the plain per-handle path; a result is bitwise the same
alone and in any mix; a dependency wait that runs out is reported, not hung."""
import numpy as np
import pytest

import synth
from parity_util import TOL, box_rim, check_array
from synth import base_desc, vacuum

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_00234_gb300 import build
    build.build()
    import paper_2305_00234_gb300 as lib
    return lib


def cases():
    """Three requests of different shapes: the config-2 recipe on 40^3 (TF/SF plane, 3 frequencies,
    3-pair metal), a ragged 44 x 38 x 35 grid with a dipole, an anisotropic Lorentz dielectric | 4-pair
    metal and gamma damping, and a serving-stream request (48^3, dipole at the centre, 2-pair metal)."""
    a = synth.scaled_workload("c2", 40, 420)
    d = base_desc(44, 38, 35, n_steps=300, cpml=(6, 5, 4, 6, 5, 4), precision=32, design=(18, 16, 14),
                  gap=(2, 2, 2), lambdas_nm=(500.0, 650.0), src_kind=0, src_comp=0, src_pos=(21, 19, 17))
    b = dict(desc=d, bg=vacuum(), m1=synth.lorentz_dielectric(6, 2, eps_inf=(11.7, 11.7, 12.1)),
             m2=synth.drude_lorentz_metal(5, 4), gamma=2e6, rho=synth.uniform_rho(synth.box_shape(d["design_box"]), 5))
    it = synth.serving_stream(seed=31, n_requests=1, sizes=(48,), steps=(280, 280), pairs=(2, 2))[0]
    c = dict(desc=it["desc"], bg=it["bg"], m1=it["m1"], m2=it["m2"], gamma=0.0, rho=it["rho"])
    return [a, b, c]


def run_batched(lib, ws, chunk, stagger=False):
    """Forward and adjoint runs of every workload through one batch; `stagger` submits the later
    requests after the first launches (continuous batching).  Returns [(F, gap, dft, adft, grad)]."""
    probs = [lib.problem(w) for w in ws]
    out = [None] * len(ws)
    with lib.Batch() as b:
        pending = list(range(len(ws)))
        first = pending.pop(0)
        b.submit(probs[first])
        if not stagger:
            while pending:
                b.submit(probs[pending.pop(0)])
        launches = 0
        while b.info()["runs"] or pending:
            for p, st in b.run(chunk):
                assert st == 0
                i = probs.index(p)
                if out[i] is None:                       # forward ended: its adjoint next
                    F, gap = p.objective()
                    out[i] = [F, gap, p.dft()]
                    b.submit(p, adjoint=True)
                else:
                    out[i] += [p.dft(True), p.gradient()]
            launches += 1
            if pending and launches % 2 == 1:
                b.submit(probs[pending.pop(0)])
        assert b.info()["launches"] == launches
    for p in probs:
        p.close()
    return out


def test_batched_runs_match_the_oracle_and_the_plain_path(lib):
    import oracle
    ws = cases()
    got = run_batched(lib, ws, chunk=64)
    tol = TOL[32]
    for w, (F, gap, dft, adft, grad) in zip(ws, got):
        o = oracle.problem(w)
        Fo, gapo = o.forward()
        odft = o.get_dft()
        o.adjoint()
        oadft = o.get_dft(True)
        ograd = o.gradient()
        o.close()
        rim = [("design-box rim", box_rim(odft.shape[2:]))]
        assert abs(F - Fo) <= tol * abs(Fo)
        check_array("gap DFT", gap, gapo, tol)
        check_array("forward DFT", dft, odft, tol, rim)
        check_array("adjoint DFT", adft, oadft, tol, rim)
        check_array("gradient", grad, ograd, tol, rim)
        p = lib.problem(w)                              # the plain path on the same request
        Fp, _ = p.forward()
        p.adjoint()
        gp = p.gradient()
        p.close()
        assert abs(F - Fp) <= 1e-5 * abs(Fp)
        assert np.linalg.norm(grad - gp) <= 1e-5 * np.linalg.norm(gp)


def test_result_is_the_same_alone_and_in_any_mix(lib):
    ws = cases()
    alone = [run_batched(lib, [w], chunk=48)[0] for w in ws]
    mixed = run_batched(lib, ws, chunk=32, stagger=True)
    mixed2 = run_batched(lib, ws[::-1], chunk=100)[::-1]
    for a, m, m2 in zip(alone, mixed, mixed2):
        for x, y, z in zip(a, m, m2):
            assert np.array_equal(x, y) and np.array_equal(x, z)


def test_wait_that_runs_out_is_reported_and_the_device_stays_usable(lib):
    from paper_2305_00234_gb300 import FdtdError
    w = cases()[2]
    p = lib.problem(w)
    with lib.Batch() as b:
        b.set_wait_limit(2_000_000, gate=True)          # 2 ms, first item waits on a flag nothing sets
        b.submit(p)
        with pytest.raises(FdtdError) as e:
            b.run(64)
        assert e.value.status == 6
        with pytest.raises(FdtdError) as e:
            b.run(64)                                   # the batch is dead
        assert e.value.status == 4
    with pytest.raises(FdtdError) as e:
        p.forward()                                     # so is the handle
    assert e.value.status == 4
    p.close()
    ref = run_batched(lib, [w], chunk=64)[0]            # a new batch on the same device works
    q = lib.problem(w)
    Fq, _ = q.forward()
    q.close()
    assert abs(ref[0] - Fq) <= 1e-5 * abs(Fq)


def test_batch_call_order_and_limits(lib):
    from paper_2305_00234_gb300 import FdtdError
    ws = cases()
    with lib.Batch() as b:
        p = lib.problem(ws[2])
        with pytest.raises(FdtdError) as e:
            b.submit(p, adjoint=True)                   # adjoint before any forward
        assert e.value.status == 4
        b.submit(p)
        with pytest.raises(FdtdError) as e:
            b.submit(p)                                 # already running in the batch
        assert e.value.status == 4
        with pytest.raises(FdtdError) as e:
            p.forward()                                 # the handle is busy until its run ends
        assert e.value.status == 4
        d64 = dict(ws[2]["desc"], precision=64)
        q = lib.Problem(d64, ws[2]["bg"], ws[2]["m1"], ws[2]["m2"])
        q.set_density(ws[2]["rho"])
        with pytest.raises(FdtdError) as e:
            b.submit(q)                                 # FP32 handles only
        assert e.value.status == 1
        q.close()
        p.close()                                       # destroying a member removes its run
        assert b.info()["runs"] == 0
        assert b.run(16) == []
