"""Handle-owning wrapper over the C-ABI calls (shapes and dtypes only; no arithmetic)."""
from __future__ import annotations

import numpy as np

from . import _native as N


def box_shape(box):
    """(dnz, dny, dnx) of a half-open {i0,i1,j0,j1,k0,k1} box (zeros if empty)."""
    if box[1] <= box[0] or box[3] <= box[2] or box[5] <= box[4]:
        return (0, 0, 0)
    return (box[5] - box[4], box[3] - box[2], box[1] - box[0])


def sample_shapes(box):
    """(z, y, x) extents of the E_x, E_y, E_z sample sets of a design box under density layout 1:
    component k spans the box's voxels extended by one on the +l faces, l != k."""
    nz, ny, nx = box_shape(box)
    if nz == 0:
        return [(0, 0, 0)] * 3
    return [(nz + 1, ny + 1, nx), (nz + 1, ny, nx + 1), (nz, ny + 1, nx + 1)]


def working_box(box, layout):
    """Box the solver keeps design state on (DFTs): the design box, grown by one cell on its +x,
    +y, +z sides under density layout 1."""
    if layout != 1 or box_shape(box)[0] == 0:
        return list(box)
    return [box[0], box[1] + 1, box[2], box[3] + 1, box[4], box[5] + 1]


class Problem:
    """One gradient problem on the current CUDA device.

    desc: grid description dict (keys of ``fdtd_grid_desc``); bg/m1/m2: material dicts
    ``{"eps_inf": [3], "sigma": [3], "poles": [[(a, c), ...] x 3]}``; stream: a cudaStream_t
    handle as int (e.g. ``torch.cuda.current_stream().cuda_stream``) or None.
    """

    def __init__(self, desc, bg, m1, m2, gamma=0.0, stream=None):
        self.desc = dict(desc)
        self.h = N.fdtd_create_grid(desc, stream)
        try:
            N.fdtd_set_materials(self.h, bg, m1, m2, gamma)
        except Exception:
            self.close()
            raise
        self.n = (int(desc["nz"]), int(desc["ny"]), int(desc["nx"]))
        self.layout = int(desc.get("density_layout", 0))
        self.wshape = box_shape(working_box(desc["design_box"], self.layout))
        if self.layout == 1:   # design variables: the three components' samples, concatenated
            self.dshape = (sum(int(np.prod(s)) for s in sample_shapes(desc["design_box"])),)
        else:
            self.dshape = box_shape(desc["design_box"])
        self.gshape = box_shape(desc["gap_box"])
        self.nf = len(desc["freqs_hz"])
        self.nd = int(np.prod(self.wshape))
        self.nvar = int(np.prod(self.dshape))
        self.ngap = int(np.prod(self.gshape))
        self.poles_total = [len(m1["poles"][k]) + len(m2["poles"][k]) for k in range(3)]
        # bumped by every call that replaces the density or the forward result the handle holds
        self.version = 0

    def close(self):
        if getattr(self, "h", None):
            N.fdtd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_density(self, rho):
        self.version += 1
        N.fdtd_set_density(self.h, rho)

    def forward(self):
        self.version += 1
        ng = 2 * self.nf * 3 * self.ngap
        F, g = N.fdtd_forward(self.h, ng)
        return F, (g[0::2] + 1j * g[1::2]).reshape((self.nf, 3) + self.gshape)

    def adjoint(self):
        N.fdtd_adjoint(self.h)

    def gradient(self, out=None):
        if out is None:
            out = np.zeros(self.dshape, dtype=np.float64)
        N.fdtd_gradient(self.h, out)
        return out

    def paper_forward(self, checkpoint_steps=0):
        """Time-domain energy objective of the paper (fdtd_paper_forward)."""
        return N.fdtd_paper_forward(self.h, checkpoint_steps)

    def paper_gradient(self, out=None, pole_pairing=0):
        """The paper's history gradient by checkpoint-recompute (fdtd_paper_gradient)."""
        if out is None:
            out = np.zeros(self.dshape, dtype=np.float64)
        N.fdtd_paper_gradient(self.h, out, pole_pairing)
        return out

    def objective(self):
        """(F, gap DFT) of the last forward run, batched or not."""
        F, g = N.fdtd_get_objective(self.h, 2 * self.nf * 3 * self.ngap)
        return F, (g[0::2] + 1j * g[1::2]).reshape((self.nf, 3) + self.gshape)

    def gradient_norm2(self):
        return N.fdtd_gradient_norm(self.h)

    def field(self, which, out=None):
        """Field `which` (0..5 = Ex..Hz) as FP64 (nz, ny, nx); `out`: a float64 CUDA tensor of that
        many elements receives it on the device (ordered on the handle's stream)."""
        a = N.fdtd_get_field(self.h, which, int(np.prod(self.n)), out)
        return a.reshape(self.n) if out is None else out

    def dft(self, adjoint=False, out=None):
        """DFT over the working box, complex (F, 3, dnz, dny, dnx); `out`: a float64 CUDA tensor of
        2 F 3 nd elements receives the interleaved (re, im) values on the device instead."""
        a = N.fdtd_get_dft(self.h, adjoint, 2 * self.nf * 3 * self.nd, out)
        if out is not None:
            return out
        return (a[0::2] + 1j * a[1::2]).reshape((self.nf, 3) + self.wshape)

    def gradient_constants(self):
        """(3, F, 4): A.re, A.im, B.re, B.im of dY/drho = A + (1 - 2 rho) B (fdtd_gradient_static's dy_drho)."""
        return N.fdtd_get_gradient_constants(self.h, self.nf)

    def inject_wait_timeout(self, timeout_ns):
        """Failure-path test hook (fdtd_inject_wait_timeout)."""
        N.fdtd_inject_wait_timeout(self.h, timeout_ns)

    def index_map(self, which):
        shape = ((3,) + self.n) if which <= 1 else self.n
        return N.fdtd_get_index_map(self.h, which, int(np.prod(shape))).reshape(shape)

    def set_profiling(self, on=True):
        N.fdtd_set_profiling(self.h, on)

    def timings(self):
        return N.fdtd_get_timings(self.h)

    def reset_timings(self):
        N.fdtd_reset_timings(self.h)

    def info(self):
        return N.fdtd_get_info(self.h)


class Batch:
    """Runs of several Problems advanced together by the persistent kernel (fdtd_batch_*)."""

    def __init__(self, stream=None):
        self.b = N.fdtd_batch_create(stream)
        self.members = {}                       # handle value -> Problem

    def submit(self, problem, adjoint=False):
        """Start the problem's forward (or adjoint) run in the batch."""
        if not adjoint:
            problem.version += 1                # replaces the forward result the handle holds
        N.fdtd_batch_submit(self.b, problem.h, adjoint)
        self.members[problem.h.value] = problem

    def run(self, max_steps):
        """One launch; [(problem, status), ...] of the runs that ended (status 0 = ok)."""
        out = []
        for hv, st in N.fdtd_batch_run(self.b, max_steps):
            out.append((self.members.pop(hv), st))
        return out

    def set_wait_limit(self, wait_ns, gate=False):
        N.fdtd_batch_set_wait_limit(self.b, wait_ns, gate)

    def set_blocks(self, blocks):
        """Blocks of the persistent launches (0: as many as fit on the device)."""
        N.fdtd_batch_set_blocks(self.b, blocks)

    def info(self):
        return N.fdtd_batch_info(self.b)

    def close(self):
        if getattr(self, "b", None):
            N.fdtd_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def problem(w, stream=None):
    """Problem for a workload dict (desc, bg, m1, m2, gamma, rho) with the density set."""
    p = Problem(w["desc"], w["bg"], w["m1"], w["m2"], w.get("gamma", 0.0), stream)
    if w.get("rho") is not None:
        p.set_density(w["rho"])
    return p
