"""The C-ABI library loads and exports every symbol include/*.h declares; host-only validation
(fdtd_footprint_bytes touches no GPU).  CPU only."""
import glob
import os
import re

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_00234_gb300 import build
    build.build()
    from paper_2305_00234_gb300 import _native
    return _native.load_library()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(fdtd_[a-z_0-9]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_every_symbol():
    from paper_2305_00234_gb300 import _native
    assert set(_native.EXPORTS) == declared_functions()


def test_footprint_and_validation_on_host(lib):
    from paper_2305_00234_gb300 import _native as N
    w = synth.workload("c2")
    b = N.fdtd_footprint_bytes(w["desc"], [3, 3, 3])
    ncell = 256 ** 3
    # fields 48 B (two buffers) + CPML slabs ~6.8 B + design state (rho, Q, two FP64 DFTs, 16-step E ring)
    # ~71 B per cell
    assert 115 * ncell < b < 135 * ncell
    bad = dict(w["desc"])
    bad["design_box"] = [4, 200, 64, 192, 64, 192]     # reaches into the CPML
    with pytest.raises(N.FdtdError) as e:
        N.fdtd_footprint_bytes(bad, [3, 3, 3])
    assert e.value.status == 1
    bad = dict(w["desc"])
    bad["courant"] = 0.6                               # above 1/sqrt(3)
    with pytest.raises(N.FdtdError):
        N.fdtd_footprint_bytes(bad, [3, 3, 3])
    bad = dict(w["desc"])
    bad["gap_box"] = [10, 12, 10, 12, 10, 12]          # outside the design box
    with pytest.raises(N.FdtdError):
        N.fdtd_footprint_bytes(bad, [3, 3, 3])


def test_product_package_does_not_touch_the_oracle():
    """The product path never imports or loads the oracle."""
    for f in glob.glob(os.path.join(ROOT, "paper_2305_00234_gb300", "**", "*.py"), recursive=True):
        src = open(f).read()
        assert "oracle" not in src, f
    for f in glob.glob(os.path.join(ROOT, "paper_2305_00234_gb300", "csrc", "*")):
        assert "oracle" not in open(f).read(), f
