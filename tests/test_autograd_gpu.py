"""torch.autograd wrapper on config 4 (64^3, 2000 steps, 2 pole pairs, 32^3 design, rho in
[0.2, 0.8]): gradient against the oracle's adjoint gradient and central finite differences;
DFT-checkpoint memory against a full time history."""
import numpy as np
import pytest

import synth

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


def test_autograd_config4_fp64_vs_oracle_and_fd(lib):
    import torch

    import oracle
    w = synth.workload("c4")
    d = dict(w["desc"], precision=64)
    p = lib.Problem(d, w["bg"], w["m1"], w["m2"], w["gamma"])
    rho = torch.tensor(w["rho"], dtype=torch.float64, device="cuda", requires_grad=True)
    F = lib.objective(rho, p)
    F.backward()
    g = rho.grad.detach().cpu().numpy()
    o = oracle.problem(dict(w, desc=d))
    Fo, _ = o.forward()
    o.adjoint()
    go = o.gradient()
    o.close()
    assert abs(F.item() - Fo) <= 1e-10 * abs(Fo)
    assert np.linalg.norm(g - go) <= 1e-10 * np.linalg.norm(go)
    # central finite differences, step 1e-4, FP64 GPU build, 64 random voxels
    rng = np.random.default_rng(2309)
    vox = [tuple(int(x) for x in rng.integers(0, 32, size=3)) for _ in range(64)]
    gap = [tuple(range(d["gap_box"][2 * a] - d["design_box"][2 * a], d["gap_box"][2 * a + 1] - d["design_box"][2 * a]))
           for a in (2, 1, 0)]
    vox = [v for v in vox if not all(v[a] in gap[a] for a in range(3))]
    fd = []
    base = w["rho"].copy()
    for v in vox:
        r = base.copy()
        r[v] += 1e-4
        p.set_density(r)
        Fp, _ = p.forward()
        r[v] -= 2e-4
        p.set_density(r)
        Fm, _ = p.forward()
        fd.append((Fp - Fm) / 2e-4)
    fd = np.array(fd)
    ga = np.array([g[v] for v in vox])
    err = np.abs(ga - fd) / np.abs(fd).max()
    # the frequency-domain adjoint is exact for decayed fields; 2000 steps leave a small tail (measured on a
    # GB300: the median voxel within 1e-5 of the largest derivative, the worst within 10%)
    assert np.median(err) < 1e-4, (np.median(err), err.max())
    assert err.max() < 0.2, (np.median(err), err.max())
    assert np.corrcoef(ga, fd)[0, 1] > 0.999
    dft, hist = lib.checkpoint_bytes(p)
    assert dft * 100 < hist
    p.close()


def test_autograd_fp32_gradient_dtype(lib):
    import torch
    w = synth.scaled_workload("c4", 32, 400)
    p = lib.Problem(w["desc"], w["bg"], w["m1"], w["m2"], w["gamma"])
    rho = torch.tensor(w["rho"], dtype=torch.float32, device="cuda", requires_grad=True)
    (2.0 * lib.objective(rho, p)).backward()
    p2 = lib.problem(w)
    p2.forward()
    p2.adjoint()
    g2 = p2.gradient()
    assert rho.grad.dtype == torch.float32
    assert np.allclose(rho.grad.cpu().numpy(), 2.0 * g2, rtol=1e-5, atol=1e-6 * np.abs(g2).max())
    p.close()
    p2.close()


def test_backward_after_another_forward_on_the_same_problem_is_refused(lib):
    """A Problem holds one density and one forward DFT: a second forward before the first node's
    backward would silently give both nodes the gradient at the second density, so it raises."""
    import torch
    w = synth.scaled_workload("c4", 32, 200)
    p = lib.Problem(w["desc"], w["bg"], w["m1"], w["m2"], w["gamma"])
    r1 = torch.tensor(w["rho"], dtype=torch.float32, device="cuda", requires_grad=True)
    r2 = torch.tensor(0.5 * w["rho"], dtype=torch.float32, device="cuda", requires_grad=True)
    F1 = lib.objective(r1, p)
    F2 = lib.objective(r2, p)
    with pytest.raises(RuntimeError, match="another forward"):
        (F1 + F2).backward()
    # one node at a time works
    F1 = lib.objective(r1, p)
    F1.backward()
    assert torch.isfinite(r1.grad).all()
    p.close()
