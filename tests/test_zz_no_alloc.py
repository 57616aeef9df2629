"""fdtd_gradient_static, the gradient entry point that allocates nothing, against fdtd_gradient.

Some callers cannot allocate device memory: a host that has handed all of it to its own pool
allocator, or a loop that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
They hold the forward and adjoint DFTs in their own buffers and call fdtd_gradient_static, whose
scratch is a static device array shared by every call.  Its output must equal fdtd_gradient's on
the same inputs, on two calls in a row (the second call finds the first call's scratch contents),
for float32 and float64 densities, with and without a gap box, and with the squared norm returned
(the call waits for the stream) or not (the call only enqueues its work).
"""
import numpy as np
import pytest

import synth
from synth import EPS0

pytestmark = pytest.mark.gpu


def dy_drho_constants(desc, m1, m2, gamma, dt):
    """(3, F, 4): A.re, A.im, B.re, B.im with dY/drho = A + (1 - 2 rho) B at each frequency, written
    out from the definition (the exported constants are checked against it)."""
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


@pytest.fixture(scope="module")
def case():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_00234_gb300 import build
    build.build()
    import paper_2305_00234_gb300 as lib

    w = synth.scaled_workload("c2", 40, 500)
    w["gamma"] = 4e6                                  # exercise the (1 - 2 rho) gamma term as well
    p = lib.problem(w)
    p.forward()
    p.adjoint()
    ref = p.gradient()                                # the existing entry point
    ref_norm2 = p.gradient_norm2()
    dt = p.info()["dt"]
    cst = p.gradient_constants()
    dfts = (p.dft(False), p.dft(True))
    nd = p.nd
    p.close()
    return dict(w=w, ref=ref, ref_norm2=ref_norm2, dt=dt, cst=cst, dfts=dfts, nd=nd, torch=torch)


def test_exported_constants_match_their_definition(case):
    w = case["w"]
    want = dy_drho_constants(w["desc"], w["m1"], w["m2"], w["gamma"], case["dt"])
    assert case["cst"].shape == want.shape
    assert np.abs(case["cst"] - want).max() <= 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("rho_dtype", ["float32", "float64"])
@pytest.mark.parametrize("with_gap", [True, False])
@pytest.mark.parametrize("with_norm", [True, False])
def test_static_scratch_gradient_matches_fdtd_gradient(case, rho_dtype, with_gap, with_norm):
    torch = case["torch"]
    from paper_2305_00234_gb300 import _native as N

    w, ref, nd = case["w"], case["ref"], case["nd"]
    d = w["desc"]
    to_dev = lambda z: torch.tensor(np.stack([z.real, z.imag], -1).ravel(), dtype=torch.float64, device="cuda")
    dft_f, dft_a = to_dev(case["dfts"][0]), to_dev(case["dfts"][1])
    rho = torch.tensor(w["rho"], dtype=getattr(torch, rho_dtype), device="cuda")
    stream = torch.cuda.current_stream()
    gap_box = d["gap_box"] if with_gap else None
    # without a gap box every voxel takes the formula, the gap voxels included
    Ef, Ea = case["dfts"]
    r = np.asarray(w["rho"], dtype=np.float32 if rho_dtype == "float32" else np.float64).astype(np.float64)
    cst = case["cst"]
    full = np.zeros_like(ref)
    for k in range(3):
        for f in range(len(d["freqs_hz"])):
            dy = (cst[k, f, 0] + 1j * cst[k, f, 1]) + (1.0 - 2.0 * r) * (cst[k, f, 2] + 1j * cst[k, f, 3])
            full -= 2.0 * np.real(dy * Ef[f, k] * Ea[f, k])
    gap = synth.box_shape(d["gap_box"])
    gsl = tuple(slice(d["gap_box"][2 * a] - d["design_box"][2 * a], d["gap_box"][2 * a + 1] - d["design_box"][2 * a])
                for a in (2, 1, 0))
    assert all(s.stop - s.start == n for s, n in zip(gsl, gap))
    for _ in range(2):
        grad = torch.full((nd,), float("nan"), dtype=torch.float64, device="cuda")
        n2 = N.fdtd_gradient_static(dft_f, dft_a, rho, d["design_box"], gap_box, len(d["freqs_hz"]), cst, grad,
                                    stream=stream.cuda_stream, norm=with_norm)
        if not with_norm:
            assert n2 is None
            stream.synchronize()                      # the call only enqueued its work
        g = grad.cpu().numpy().reshape(ref.shape)
        want = full.copy()
        if with_gap:
            want[gsl] = 0.0
        assert np.linalg.norm(g - want) <= 1e-10 * np.linalg.norm(want)
        if rho_dtype == "float32" and with_gap:       # the handle keeps an FP32 density: same inputs
            assert np.linalg.norm(g - ref) <= 1e-10 * np.linalg.norm(ref)
            if with_norm:
                assert n2 == pytest.approx(case["ref_norm2"], rel=1e-10)
        if with_norm:
            assert n2 == pytest.approx(float(np.sum(g * g)), rel=1e-10)


def test_static_entry_refuses_bad_sizes(case):
    torch = case["torch"]
    from paper_2305_00234_gb300 import _native as N

    w, nd = case["w"], case["nd"]
    d = w["desc"]
    nf = len(d["freqs_hz"])
    dft = torch.zeros(6 * nf * nd, dtype=torch.float64, device="cuda")
    rho = torch.zeros(nd, dtype=torch.float32, device="cuda")
    grad = torch.zeros(nd, dtype=torch.float64, device="cuda")
    cst = case["cst"]
    # sizes beyond the static scratch are refused by the library itself with a reason, before any
    # launch (called through the raw C-ABI: the small buffers are never touched)
    import ctypes as C
    lib = N.load_library()
    big = (C.c_int * 6)(0, 4096, 0, 4096, 0, 4)
    c = np.ascontiguousarray(cst).ravel()
    rc = lib.fdtd_gradient_static(C.c_void_p(dft.data_ptr()), C.c_void_p(dft.data_ptr()), C.c_void_p(rho.data_ptr()),
                                  0, big, None, nf, c.ctypes.data_as(C.POINTER(C.c_double)),
                                  C.c_void_p(grad.data_ptr()), None, None)
    assert rc == 1 and "at most" in lib.fdtd_last_error(None).decode()
    # buffers that do not match the design box and frequency count are refused before the call
    with pytest.raises(ValueError):
        N.fdtd_gradient_static(dft[:-2], dft, rho, d["design_box"], None, nf, cst, grad)
    with pytest.raises(ValueError):
        N.fdtd_gradient_static(dft, dft, rho[:-1], d["design_box"], None, nf, cst, grad)
    with pytest.raises(ValueError):
        N.fdtd_gradient_static(dft, dft, rho, d["design_box"], None, nf, cst, grad[:-1])
    with pytest.raises(ValueError):
        N.fdtd_gradient_static(dft, dft, rho, d["design_box"], None, nf, cst[:, :, :3], grad)
