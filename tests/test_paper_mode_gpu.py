"""GPU paper mode (fdtd_paper_forward / fdtd_paper_gradient: the time-domain energy objective and
Eq. (Gradient_FDTD) by checkpoint-recompute) against the oracle's paper mode on the same inputs.

Tolerances as for the frequency-domain path: relative L2 <= 1e-4 (FP32), <= 1e-10 (FP64).  The
checkpoint interval is a memory / recompute trade only: different intervals give the same gradient.
"""
import numpy as np
import pytest

import synth
from synth import base_desc, vacuum

pytestmark = pytest.mark.gpu

TOL = {32: 1e-4, 64: 1e-10}


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_00234_gb300 import build
    build.build()
    import paper_2305_00234_gb300 as lib
    lib.load_library()
    return lib


def _case(prec, metal=True, steps=1200):
    # 52 x 48 x 44 with a 4-cell CPML has an interior box for the fused kernel (FP32 and FP64)
    d = base_desc(52, 48, 44, n_steps=steps, cpml=4, precision=prec, design=(16, 16, 16), gap=(2, 2, 2),
                  lambdas_nm=(600.0,), src_kind=0, src_comp=2, src_pos=(14, 24, 22))
    rho = synth.uniform_rho(synth.box_shape(d["design_box"]), 17, 0.2, 0.8)
    m2 = synth.drude_lorentz_metal(17, 2) if metal else synth.lorentz_dielectric(18, 2)
    return dict(desc=d, bg=vacuum(), m1=vacuum(), m2=m2, gamma=2e5, rho=rho)


def _oracle(w):
    import oracle
    o = oracle.problem(w)
    F, g0 = o.paper_gradient(1)     # printed pole term
    _, g1 = o.paper_gradient(5)     # pole term on one adjoint level
    o.close()
    return F, g0, g1


@pytest.mark.parametrize("prec,metal", [(32, True), (64, True), (32, False)])
def test_paper_mode_matches_oracle(lib, prec, metal):
    w = _case(prec, metal)
    Fo, go0, go1 = _oracle(w)
    p = lib.problem(w)
    assert p.timings()["fused_step"] == 1
    F = p.paper_forward(checkpoint_steps=170)          # 1200 = 7 x 170 + 10: a short last segment
    g0 = p.paper_gradient(pole_pairing=0)
    g1 = p.paper_gradient(pole_pairing=1)
    assert abs(F - Fo) <= TOL[prec] * abs(Fo)
    assert rel(g0, go0) <= TOL[prec], rel(g0, go0)
    assert rel(g1, go1) <= TOL[prec], rel(g1, go1)
    gap = np.zeros(g0.shape, bool)
    db, gb = w["desc"]["design_box"], w["desc"]["gap_box"]
    gap[gb[4] - db[4]:gb[5] - db[4], gb[2] - db[2]:gb[3] - db[2], gb[0] - db[0]:gb[1] - db[0]] = True
    assert np.all(g0[gap] == 0.0) and np.all(g1[gap] == 0.0)
    # another checkpoint interval (the default) gives the same gradient
    F2 = p.paper_forward()
    g2 = p.paper_gradient(pole_pairing=0)
    assert F2 == F
    assert rel(g2, g0) <= 1e-12
    p.close()


def test_paper_mode_call_order(lib):
    from paper_2305_00234_gb300 import _native as N
    w = _case(32, steps=300)
    p = lib.problem(w)
    with pytest.raises(N.FdtdError):
        p.paper_gradient()                              # before the paper forward
    p.paper_forward(64)
    p.set_density(w["rho"])
    with pytest.raises(N.FdtdError):
        p.paper_gradient()                              # the density changed since
    p.close()
