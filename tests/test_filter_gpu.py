"""Density filter, projection and chain rule on the GPU (Sec. "Filtering and projection") against
the oracle's numpy/scipy version, element by element (FP32 sums of up to ~7200 taps: 1e-5)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_00234_gb300 import build
    build.build()
    from paper_2305_00234_gb300 import _native
    return _native


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("shape,R,beta,eta", [((13, 17, 20), 1.5, 10.0, 0.5), ((24, 20, 28), 3.0, 1e-4, 0.5),
                                              ((30, 26, 33), 12.0, 52.0, 0.5), ((9, 40, 11), 5.5, 8.0, 0.3)])
def test_filter_project_and_chain_rule(N, shape, R, beta, eta):
    import torch

    from oracle import filter as OF
    rng = np.random.default_rng(int(R * 10))
    rho = rng.uniform(size=shape)
    g_b = rng.normal(size=shape)
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    r, rt, rb = dev(rho), torch.empty(shape, dtype=torch.float32, device="cuda"), torch.empty(shape, dtype=torch.float32, device="cuda")
    N.fdtd_filter_project(r, rt, rb, R, beta, eta)
    grad = torch.empty(shape, dtype=torch.float32, device="cuda")
    N.fdtd_filter_project_grad(rt, dev(g_b), grad, R, beta, eta)
    torch.cuda.synchronize()
    rt_o = OF.filter_density(rho.astype(np.float32).astype(np.float64), R)
    assert rel(rt.cpu().numpy(), rt_o) <= 1e-5
    # the projection of the GPU's own filtered field (a steep projection amplifies the filter's
    # FP32 rounding, which the line above already bounds)
    assert rel(rb.cpu().numpy(), OF.project(rt.cpu().numpy().astype(np.float64), beta, eta)) <= 1e-5
    go = OF.chain_rule(g_b.astype(np.float32).astype(np.float64), rt.cpu().numpy().astype(np.float64), R, beta, eta)
    assert rel(grad.cpu().numpy(), go) <= 1e-5


def test_filter_argument_errors(N):
    import torch
    x = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(N.FdtdError):
        N.fdtd_filter_project(x, x.clone(), x.clone(), 13.0, 1.0, 0.5)     # radius above the limit
    with pytest.raises(N.FdtdError):
        N.fdtd_filter_project(x, x.clone(), x.clone(), 2.0, -1.0, 0.5)
