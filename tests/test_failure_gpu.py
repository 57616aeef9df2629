"""Failure detection on the GPU without a fault: a bounded device wait that runs out.

fdtd_inject_wait_timeout makes one block of the interior step kernel wait, with a short limit, on an
mbarrier that no copy completes.  The wait gives up, the block records it in the handle's device
flags, waits for its own copies in flight and returns; the run reports FDTD_ERR_TIMEOUT, the handle
is dead, and the device context stays usable for a new handle."""
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


def test_wait_that_runs_out_reports_timeout_and_leaves_the_context_usable(lib):
    from paper_2305_00234_gb300 import FdtdError
    w = synth.scaled_workload("c2", 48, 64)
    ref = lib.problem(w)
    assert ref.timings()["fused_step"] == 1
    F_ref, _ = ref.forward()
    ref.close()

    p = lib.problem(w)
    p.inject_wait_timeout(2_000_000)                  # 2 ms
    with pytest.raises(FdtdError) as e:
        p.forward()
    assert e.value.status == 6                        # FDTD_ERR_TIMEOUT
    assert "time limit" in str(e.value)
    with pytest.raises(FdtdError) as e:
        p.forward()                                   # the handle is dead
    assert e.value.status == 4
    p.close()

    q = lib.problem(w)                                # same device, new handle: same result as before
    F, _ = q.forward()
    q.close()
    assert F == F_ref


def test_hook_off_and_refused_without_an_interior_box(lib):
    from paper_2305_00234_gb300 import FdtdError
    w = synth.scaled_workload("c2", 48, 64)
    p = lib.problem(w)
    p.inject_wait_timeout(2_000_000)
    p.inject_wait_timeout(0)                          # off again
    F, _ = p.forward()
    assert np.isfinite(F) and F > 0
    p.close()
    small = synth.base_desc(12, 12, 12, n_steps=20, cpml=2, design=(4, 4, 4), gap=(2, 2, 2))
    q = lib.Problem(small, synth.vacuum(), synth.vacuum(), synth.drude_lorentz_metal(1, 1))
    assert q.timings()["fused_step"] == 0
    with pytest.raises(FdtdError) as e:
        q.inject_wait_timeout(1_000_000)
    assert e.value.status == 1
    q.close()
