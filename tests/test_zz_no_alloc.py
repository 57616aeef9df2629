"""fdtd_gradient_static, the gradient entry point that allocates nothing, against fdtd_gradient.

Some callers cannot allocate device memory: a host that has handed all of it to its own pool
allocator, or a loop that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
They hold the forward and adjoint DFTs in their own buffers and call fdtd_gradient_static, whose
scratch is a static device array shared by every call.  Its output must equal fdtd_gradient's on
the same inputs, on two calls in a row (the second call finds the first call's scratch contents).
"""
import numpy as np
import pytest

import synth
from synth import EPS0

pytestmark = pytest.mark.gpu


def dy_drho_constants(desc, m1, m2, gamma, dt):
    """(3, F, 4): A.re, A.im, B.re, B.im with dY/drho = A + (1 - 2 rho) B at each frequency."""
    out = np.zeros((3, len(desc["freqs_hz"]), 4))
    for k in range(3):
        for f, fr in enumerate(desc["freqs_hz"]):
            z = np.exp(1j * 2 * np.pi * fr * dt)
            poles = 0j
            for sign, mat in ((-1.0, m1), (1.0, m2)):
                for a, c in mat["poles"][k]:
                    al = np.exp(a * dt)
                    be = EPS0 * c * (al - 1) / (2 * a)
                    poles += sign * (be * (z + 1) / (z - al) + np.conj(be) * (z + 1) / (z - np.conj(al)))
            A = (EPS0 * (m2["eps_inf"][k] - m1["eps_inf"][k]) * (z - 1)
                 + (m2["sigma"][k] - m1["sigma"][k]) * dt * (z + 1) / 2 + (z - 1) * poles) / dt
            B = gamma * (z + 1) / 2
            out[k, f] = (A.real, A.imag, B.real, B.imag)
    return out


def test_static_scratch_gradient_matches_fdtd_gradient():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_00234_gb300 import build
    build.build()
    import paper_2305_00234_gb300 as lib
    from paper_2305_00234_gb300 import _native as N

    w = synth.scaled_workload("c2", 40, 500)
    w["gamma"] = 4e6                                  # exercise the (1 - 2 rho) gamma term as well
    d = w["desc"]
    p = lib.problem(w)
    p.forward()
    p.adjoint()
    ref = p.gradient()                                # the existing entry point
    ref_norm2 = p.gradient_norm2()
    dt = p.info()["dt"]
    nd = p.nd
    to_dev = lambda z: torch.tensor(np.stack([z.real, z.imag], -1).ravel(), dtype=torch.float64, device="cuda")
    dft_f, dft_a = to_dev(p.dft(False)), to_dev(p.dft(True))
    rho = torch.tensor(w["rho"], dtype=torch.float32, device="cuda")
    cst = dy_drho_constants(d, w["m1"], w["m2"], w["gamma"], dt)
    p.close()
    for _ in range(2):
        grad = torch.full((nd,), float("nan"), dtype=torch.float64, device="cuda")
        n2 = N.fdtd_gradient_static(dft_f, dft_a, rho, d["design_box"], d["gap_box"], len(d["freqs_hz"]), cst, grad)
        g = grad.cpu().numpy().reshape(ref.shape)
        assert np.linalg.norm(g - ref) <= 1e-10 * np.linalg.norm(ref)
        assert n2 == pytest.approx(ref_norm2, rel=1e-10)
    # sizes beyond the static scratch are refused with a reason, before any launch
    big = [0, 4096, 0, 4096, 0, 4]
    with pytest.raises(N.FdtdError) as e:
        N.fdtd_gradient_static(dft_f, dft_a, rho, big, None, len(d["freqs_hz"]), cst, grad)
    assert e.value.status == 1 and "at most" in str(e.value)
