"""Serving loop: continuous batching with admission by device footprint, the batch lane (persistent kernel
over a device work queue) and the plain lane (per-request streams); every result is the same alone and in
the mix."""
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


def small_stream(n=6, seed=7, sizes=(48, 56, 64)):
    return synth.serving_stream(seed=seed, n_requests=n, sizes=sizes, steps=(300, 500), pairs=(1, 3))


@pytest.mark.parametrize("batch_max_cells", [None, 0, 52 ** 3])
def test_alone_and_in_the_mix_are_bitwise_equal(srv, batch_max_cells):
    """batch_max_cells None: every request in the batch lane; 0: every request in the plain lane; 52^3:
    both lanes at once.  Alone = the same server admitting one request at a time."""
    items = small_stream()
    with srv.GradientServer(max_slots=1, batch_max_cells=batch_max_cells, chunk_steps=64) as server:
        alone = [server.submit(r).result() for r in srv.from_stream(items)]
    with srv.GradientServer(max_slots=6, batch_max_cells=batch_max_cells, chunk_steps=48) as server:
        futs = [server.submit(r) for r in srv.from_stream(items)]
        mixed = [f.result() for f in futs]
    assert server.peak_active >= 2            # the requests overlapped on the device
    lanes = {r.lane for r in mixed}
    assert lanes == {None: {"batch"}, 0: {"plain"}}.get(batch_max_cells, {"batch", "plain"})
    for a, m, it in zip(alone, mixed, items):
        assert a.F == m.F and a.lane == m.lane
        assert np.array_equal(a.grad, m.grad)
    # either lane gives the plain path's result to FP32 rounding
    for m, r in zip(mixed, srv.from_stream(items)):
        F, g = srv.evaluate(r)
        assert abs(m.F - F) <= 1e-5 * abs(F)
        assert np.linalg.norm(m.grad - g) <= 1e-5 * np.linalg.norm(g)


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


def test_requests_arriving_during_a_launch_join_the_next_one(srv):
    """Continuous batching: requests submitted while the batch lane is running enter its later launches
    (the batch held more runs at once than were submitted before the first launch)."""
    items = small_stream(6, seed=19, sizes=(48,))
    reqs = srv.from_stream(items)
    with srv.GradientServer(max_slots=8, batch_max_cells=None, chunk_steps=32) as server:
        futs = [server.submit(reqs[0])]
        import time
        time.sleep(0.05)
        futs += [server.submit(r) for r in reqs[1:]]
        res = [f.result() for f in futs]
    assert all(r.lane == "batch" for r in res)
    assert server.peak_batched >= 2 and server.launches >= 2


def test_large_grids_run_one_at_a_time_and_small_ones_overtake(srv):
    """exclusive_cells: two large requests never overlap on the device, and a small request submitted after
    the second large one starts before it (it may pass a request that waits for a running large grid)."""
    big = srv.from_stream(synth.serving_stream(seed=23, n_requests=2, sizes=(64,), steps=(400, 401), pairs=(2, 2)))
    small = srv.from_stream(synth.serving_stream(seed=29, n_requests=1, sizes=(32,), steps=(300, 301), pairs=(1, 1)))
    with srv.GradientServer(max_slots=4, batch_max_cells=0, exclusive_cells=64 ** 3) as server:
        futs = [server.submit(r) for r in big + small]
        b1, b2, s1 = [f.result() for f in futs]
    assert b2.t_admit >= b1.t_done or b1.t_admit >= b2.t_done
    first, second = (b1, b2) if b1.t_admit <= b2.t_admit else (b2, b1)
    assert s1.t_admit < second.t_admit
    assert {b1.lane, b2.lane, s1.lane} == {"plain"}
