"""Serving loop: continuous batching with admission by device footprint; every result is the
same alone and in the mix."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_00234_gb300 import build
    build.build()
    from paper_2305_00234_gb300 import serve
    return serve


def small_stream(n=6, seed=7):
    items = synth.serving_stream(seed=seed, n_requests=n, sizes=(48, 56, 64), steps=(300, 500),
                                 pairs=(1, 3))
    return items


def test_alone_and_in_the_mix_are_bitwise_equal(srv):
    items = small_stream()
    alone = [srv.evaluate(r) for r in srv.from_stream(items)]
    with srv.GradientServer(max_slots=4) as server:
        futs = [server.submit(r) for r in srv.from_stream(items)]
        mixed = [f.result() for f in futs]
    assert server.peak_active >= 2            # the requests overlapped on the device
    for (F, g), r in zip(alone, mixed):
        assert F == r.F
        assert np.array_equal(g, r.grad)


def test_admission_by_footprint_and_failure_isolation(srv):
    items = small_stream(5, seed=11)
    reqs = srv.from_stream(items)
    fps = [r.footprint() for r in reqs]
    budget = 2 * max(fps) + 1                 # at most two of the largest fit at a time
    bad = srv.from_stream(small_stream(1, seed=3))[0]
    bad.desc = dict(bad.desc, design_box=[0, 10, 0, 10, 0, 10])    # reaches into the CPML
    too_big = srv.from_stream(synth.serving_stream(seed=5, n_requests=1, sizes=(192,)))[0]
    with srv.GradientServer(max_slots=8, hbm_budget=budget) as server:
        futs = [server.submit(r) for r in reqs]
        f_bad = server.submit(bad)
        f_big = server.submit(too_big)
        res = [f.result() for f in futs]
    assert server.peak_in_use <= budget
    assert server.peak_active < len(reqs)     # admission held some requests back
    with pytest.raises(Exception):
        f_bad.result()
    with pytest.raises(Exception) as e:
        f_big.result()
    assert "budget" in str(e.value)
    assert all(r.F > 0 for r in res)
