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


def test_per_sample_layout_validation_on_host(lib):
    """density_layout 1 grows the working box by one cell on the +x/+y/+z sides: a design box that
    ends at the CPML is valid per voxel but not per sample; layouts other than 0 and 1 are refused."""
    from paper_2305_00234_gb300 import _native as N
    d = synth.base_desc(64, 64, 64, n_steps=10, cpml=8, design=(20, 20, 20), gap=(2, 2, 2))
    d["design_box"] = [36, 56, 22, 42, 22, 42]         # x1 = 56 = nx - cpml
    d["gap_box"] = [40, 42, 30, 32, 30, 32]
    b0 = N.fdtd_footprint_bytes(d, [2, 2, 2])
    with pytest.raises(N.FdtdError) as e:
        N.fdtd_footprint_bytes(dict(d, density_layout=1), [2, 2, 2])
    assert e.value.status == 1
    with pytest.raises(N.FdtdError):
        N.fdtd_footprint_bytes(dict(d, density_layout=2), [2, 2, 2])
    d["design_box"] = [30, 50, 22, 42, 22, 42]
    assert N.fdtd_footprint_bytes(dict(d, density_layout=1), [2, 2, 2]) > N.fdtd_footprint_bytes(d, [2, 2, 2]) > 0
    assert b0 > 0


@pytest.mark.parametrize("box", [[30, 50, 22, 42, 22, 42], [10, 11, 12, 20, 5, 9], [0, 0, 0, 0, 0, 0]])
def test_binding_shapes_match_the_oracle(box):
    """The binding's density / gradient and DFT shapes for both layouts equal the oracle's."""
    import oracle
    from paper_2305_00234_gb300.problem import box_shape, sample_shapes, working_box
    import numpy as np
    d = synth.base_desc(64, 64, 64, n_steps=4, cpml=4, precision=64)
    d["design_box"] = box
    for layout in (0, 1):
        d["density_layout"] = layout
        o = oracle.Oracle(d)
        w = box_shape(working_box(box, layout))
        if box_shape(box)[0] == 0:
            assert o.vshape == (0, 0, 0)
        else:
            assert o.wshape == w
            n = sum(int(np.prod(s)) for s in sample_shapes(box)) if layout else int(np.prod(box_shape(box)))
            assert int(np.prod(o.vshape)) == n
        o.close()
