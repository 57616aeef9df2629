"""ctypes binding of ``libfdtdccpr.so`` (C-ABI in include/fdtd_ccpr.h).

Argument marshalling only: every step of the gradient evaluation runs in the library's CUDA
kernels.  If the library has not been built this module raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libfdtdccpr.so")

FDTD_OK = 0
STATUS = {0: "FDTD_OK", 1: "FDTD_ERR_ARG", 2: "FDTD_ERR_OOM", 3: "FDTD_ERR_CUDA", 4: "FDTD_ERR_STATE",
          5: "FDTD_ERR_UNSTABLE", 6: "FDTD_ERR_TIMEOUT", 7: "FDTD_ERR_CANCELLED"}

EXPORTS = ("fdtd_create_grid", "fdtd_footprint_bytes", "fdtd_set_materials", "fdtd_set_density",
           "fdtd_forward", "fdtd_adjoint", "fdtd_gradient", "fdtd_gradient_norm", "fdtd_get_field",
           "fdtd_get_dft", "fdtd_get_index_map", "fdtd_set_profiling", "fdtd_get_timings",
           "fdtd_reset_timings", "fdtd_get_info", "fdtd_cancel", "fdtd_last_error", "fdtd_destroy",
           "fdtd_gradient_static", "fdtd_filter_project", "fdtd_filter_project_grad", "fdtd_paper_forward",
           "fdtd_paper_gradient", "fdtd_get_gradient_constants", "fdtd_inject_wait_timeout", "fdtd_batch_create",
           "fdtd_batch_submit", "fdtd_batch_run", "fdtd_batch_set_wait_limit", "fdtd_batch_set_blocks", "fdtd_batch_info",
           "fdtd_batch_destroy",
           "fdtd_get_objective")


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("courant", C.c_double), ("n_steps", C.c_int),
                ("cpml", C.c_int * 6),
                ("cpml_m", C.c_double), ("cpml_sigma_scale", C.c_double),
                ("cpml_kappa_max", C.c_double), ("cpml_a_max", C.c_double),
                ("precision", C.c_int),
                ("design_box", C.c_int * 6), ("gap_box", C.c_int * 6),
                ("n_freq", C.c_int), ("freqs_hz", C.POINTER(C.c_double)),
                ("freq_weights", C.POINTER(C.c_double)),
                ("src_kind", C.c_int), ("src_comp", C.c_int), ("src_pos", C.c_int * 3),
                ("src_f0", C.c_double), ("src_fwhm_hz", C.c_double), ("src_t0", C.c_double),
                ("src_amp", C.c_double), ("adj_tau", C.c_double), ("src_wave", C.POINTER(C.c_double)),
                ("density_layout", C.c_int)]


class Material(C.Structure):
    _fields_ = [("eps_inf", C.c_double * 3), ("sigma", C.c_double * 3), ("n_poles", C.c_int * 3),
                ("a_re", C.POINTER(C.c_double) * 3), ("a_im", C.POINTER(C.c_double) * 3),
                ("c_re", C.POINTER(C.c_double) * 3), ("c_im", C.POINTER(C.c_double) * 3)]


class Timings(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("shell_h_ms", "step_ms", "shell_e_ms", "ed_ms", "dft_ms", "grad_ms")] + \
               [(k, C.c_longlong) for k in ("shell_h_launches", "step_launches", "shell_e_launches", "ed_launches",
                                            "dft_launches", "grad_launches", "launches")] + \
               [(k, C.c_double) for k in ("bytes_shell_h_per_launch", "bytes_step_per_launch",
                                          "bytes_shell_e_per_launch", "bytes_ed_per_launch", "bytes_dft_per_launch",
                                          "bytes_grad_per_launch", "dft_steps_per_launch")] + \
               [("fused_step", C.c_longlong), ("interior_cells", C.c_double), ("interior_design_cells", C.c_double),
                ("paired_shell", C.c_longlong), ("pdl_graphs", C.c_longlong), ("paired_design", C.c_longlong)]


class FdtdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library():
    """Load the in-tree CUDA library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FdtdError(3, f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    P, vp, sz, d, i = C.POINTER, C.c_void_p, C.c_size_t, C.c_double, C.c_int
    sig = {
        "fdtd_create_grid": [P(GridDesc), vp, P(vp)],
        "fdtd_footprint_bytes": [P(GridDesc), P(C.c_int), P(sz)],
        "fdtd_set_materials": [vp, P(Material), P(Material), P(Material), d],
        "fdtd_set_density": [vp, vp, sz, i, i],
        "fdtd_forward": [vp, P(d), P(d)],
        "fdtd_adjoint": [vp],
        "fdtd_gradient": [vp, vp, sz, i, i],
        "fdtd_gradient_norm": [vp, P(d)],
        "fdtd_paper_forward": [vp, i, P(d)],
        "fdtd_paper_gradient": [vp, i, vp, sz, i, i],
        "fdtd_get_field": [vp, i, vp, sz, i],
        "fdtd_get_dft": [vp, i, vp, sz, i],
        "fdtd_get_gradient_constants": [vp, P(d), sz],
        "fdtd_batch_create": [vp, P(vp)],
        "fdtd_batch_submit": [vp, vp, i],
        "fdtd_batch_run": [vp, i, P(vp), P(C.c_int), i, P(C.c_int)],
        "fdtd_batch_set_wait_limit": [vp, C.c_longlong, i],
        "fdtd_batch_set_blocks": [vp, i],
        "fdtd_batch_info": [vp, P(C.c_int), P(C.c_longlong)],
        "fdtd_batch_destroy": [vp],
        "fdtd_get_objective": [vp, P(d), P(d)],
        "fdtd_inject_wait_timeout": [vp, C.c_longlong],
        "fdtd_get_index_map": [vp, i, P(C.c_int32), sz],
        "fdtd_set_profiling": [vp, i],
        "fdtd_get_timings": [vp, P(Timings)],
        "fdtd_reset_timings": [vp],
        "fdtd_get_info": [vp, P(d), P(sz), P(sz), P(sz)],
        "fdtd_cancel": [vp],
        "fdtd_last_error": [vp],
        "fdtd_destroy": [vp],
        "fdtd_gradient_static": [vp, vp, vp, i, P(C.c_int), P(C.c_int), i, P(d), vp, P(d), vp],
        "fdtd_filter_project": [vp, vp, vp, i, i, i, d, d, d, vp],
        "fdtd_filter_project_grad": [vp, vp, vp, i, i, i, d, d, d, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_char_p if name == "fdtd_last_error" else C.c_int
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_desc(desc, keep):
    """GridDesc from a description dict (keys as in the C struct); arrays kept alive in `keep`."""
    g = GridDesc()
    for key in ("nx", "ny", "nz", "n_steps", "precision", "src_kind", "src_comp"):
        setattr(g, key, int(desc[key]))
    g.density_layout = int(desc.get("density_layout", 0))
    for key in ("dx", "courant", "cpml_m", "cpml_sigma_scale", "cpml_kappa_max", "cpml_a_max",
                "src_f0", "src_fwhm_hz", "src_t0", "src_amp", "adj_tau"):
        setattr(g, key, float(desc[key]))
    for key, n in (("cpml", 6), ("design_box", 6), ("gap_box", 6), ("src_pos", 3)):
        for q in range(n):
            getattr(g, key)[q] = int(desc[key][q])
    f = np.ascontiguousarray(desc["freqs_hz"], dtype=np.float64)
    w = np.ascontiguousarray(desc["freq_weights"], dtype=np.float64)
    keep += [f, w]
    g.n_freq = f.size
    g.freqs_hz = _dptr(f)
    g.freq_weights = _dptr(w)
    if desc.get("src_wave") is not None:
        wv = np.ascontiguousarray(desc["src_wave"], dtype=np.float64)
        if wv.size != 2 * int(desc["n_steps"]) + 1:
            raise ValueError("src_wave needs 2 n_steps + 1 samples (t = s dt / 2)")
        keep.append(wv)
        g.src_wave = _dptr(wv)
    return g


def make_material(m, keep):
    s = Material()
    for k in range(3):
        s.eps_inf[k] = float(m["eps_inf"][k])
        s.sigma[k] = float(m["sigma"][k])
        poles = m["poles"][k]
        s.n_poles[k] = len(poles)
        arrs = [np.ascontiguousarray([complex(a).real for a, _ in poles] or [0.0]),
                np.ascontiguousarray([complex(a).imag for a, _ in poles] or [0.0]),
                np.ascontiguousarray([complex(c).real for _, c in poles] or [0.0]),
                np.ascontiguousarray([complex(c).imag for _, c in poles] or [0.0])]
        keep += arrs
        s.a_re[k], s.a_im[k], s.c_re[k], s.c_im[k] = (_dptr(a) for a in arrs)
    return s


def _check(h, rc, what):
    if rc != FDTD_OK:
        msg = load_library().fdtd_last_error(h)
        raise FdtdError(rc, f"{what}: {msg.decode() if msg else ''}")


# ---- same names as the C-ABI (thin marshalling) ----------------------------------------------

def fdtd_create_grid(desc, stream=None):
    lib = load_library()
    keep = []
    g = make_desc(desc, keep)
    h = C.c_void_p()
    rc = lib.fdtd_create_grid(C.byref(g), C.c_void_p(stream or 0), C.byref(h))
    if rc != FDTD_OK:
        raise FdtdError(rc, "fdtd_create_grid: " + lib.fdtd_last_error(None).decode())
    return h


def fdtd_footprint_bytes(desc, p_total):
    lib = load_library()
    keep = []
    g = make_desc(desc, keep)
    pt = (C.c_int * 3)(*[int(x) for x in p_total])
    out = C.c_size_t()
    rc = lib.fdtd_footprint_bytes(C.byref(g), pt, C.byref(out))
    if rc != FDTD_OK:
        raise FdtdError(rc, "fdtd_footprint_bytes: " + lib.fdtd_last_error(None).decode())
    return out.value


def fdtd_set_materials(h, bg, m1, m2, gamma=0.0):
    keep = []
    b, a1, a2 = make_material(bg, keep), make_material(m1, keep), make_material(m2, keep)
    _check(h, load_library().fdtd_set_materials(h, C.byref(b), C.byref(a1), C.byref(a2),
                                                 float(gamma)), "fdtd_set_materials")


def _buffer(x):
    """(pointer, n, dtype code, on_device, keepalive) for a numpy array or torch tensor."""
    if hasattr(x, "data_ptr"):                  # torch tensor
        import torch
        if x.dtype not in (torch.float32, torch.float64):
            raise TypeError("float32 or float64 tensor expected")
        if not x.is_contiguous():
            raise ValueError("contiguous tensor expected")
        return x.data_ptr(), x.numel(), 0 if x.dtype == torch.float32 else 1, int(x.is_cuda), x
    a = np.ascontiguousarray(x)
    if a.dtype not in (np.float32, np.float64):
        a = a.astype(np.float64)
    return a.ctypes.data, a.size, 0 if a.dtype == np.float32 else 1, 0, a


def fdtd_set_density(h, rho):
    p, n, dt, dev, keep = _buffer(rho)
    _check(h, load_library().fdtd_set_density(h, C.c_void_p(p), n, dt, dev), "fdtd_set_density")


def fdtd_forward(h, n_gap_doubles=0):
    F = C.c_double()
    g = np.zeros(max(n_gap_doubles, 1), dtype=np.float64)
    _check(h, load_library().fdtd_forward(h, C.byref(F), _dptr(g) if n_gap_doubles else None),
           "fdtd_forward")
    return F.value, g[:n_gap_doubles]


def fdtd_adjoint(h):
    _check(h, load_library().fdtd_adjoint(h), "fdtd_adjoint")


def fdtd_gradient(h, out):
    p, n, dt, dev, keep = _buffer(out)
    _check(h, load_library().fdtd_gradient(h, C.c_void_p(p), n, dt, dev), "fdtd_gradient")
    return out


def fdtd_paper_forward(h, checkpoint_steps=0):
    v = C.c_double()
    _check(h, load_library().fdtd_paper_forward(h, int(checkpoint_steps), C.byref(v)), "fdtd_paper_forward")
    return v.value


def fdtd_paper_gradient(h, out, pole_pairing=0):
    p, n, dt, dev, keep = _buffer(out)
    _check(h, load_library().fdtd_paper_gradient(h, int(pole_pairing), C.c_void_p(p), n, dt, dev), "fdtd_paper_gradient")
    return out


def fdtd_gradient_norm(h):
    v = C.c_double()
    _check(h, load_library().fdtd_gradient_norm(h, C.byref(v)), "fdtd_gradient_norm")
    return v.value


def _f64_out(out, n, name):
    """(pointer, on_device, array) of an output buffer of n doubles: a new host array when out is
    None, else a numpy float64 array or a float64 torch tensor (CUDA: on_device)."""
    if out is None:
        a = np.zeros(n, dtype=np.float64)
        return a.ctypes.data, 0, a
    if hasattr(out, "data_ptr"):
        import torch
        if out.dtype != torch.float64 or not out.is_contiguous() or out.numel() != n:
            raise ValueError(f"{name}: a contiguous float64 tensor of {n} elements expected")
        return out.data_ptr(), int(out.is_cuda), out
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous and out.size == n):
        raise ValueError(f"{name}: a contiguous float64 array of {n} elements expected")
    return out.ctypes.data, 0, out


def fdtd_get_field(h, which, n, out=None):
    """Field `which` (0..5 = Ex..Hz) as n doubles into `out` (host array or CUDA tensor; new host
    array if None)."""
    ptr, dev, a = _f64_out(out, n, "fdtd_get_field")
    _check(h, load_library().fdtd_get_field(h, which, C.c_void_p(ptr), n, dev), "fdtd_get_field")
    return a


def fdtd_get_dft(h, adjoint, n_doubles, out=None):
    ptr, dev, a = _f64_out(out, n_doubles, "fdtd_get_dft")
    _check(h, load_library().fdtd_get_dft(h, int(adjoint), C.c_void_p(ptr), n_doubles, dev), "fdtd_get_dft")
    return a


def fdtd_get_gradient_constants(h, n_freq):
    """(3, n_freq, 4) doubles: A.re, A.im, B.re, B.im of dY/drho = A + (1 - 2 rho) B."""
    a = np.zeros(12 * n_freq, dtype=np.float64)
    _check(h, load_library().fdtd_get_gradient_constants(h, _dptr(a), a.size), "fdtd_get_gradient_constants")
    return a.reshape(3, n_freq, 4)


def fdtd_inject_wait_timeout(h, timeout_ns):
    _check(h, load_library().fdtd_inject_wait_timeout(h, int(timeout_ns)), "fdtd_inject_wait_timeout")


def fdtd_get_index_map(h, which, n):
    a = np.zeros(n, dtype=np.int32)
    _check(h, load_library().fdtd_get_index_map(h, which, a.ctypes.data_as(C.POINTER(C.c_int32)), n),
           "fdtd_get_index_map")
    return a


def fdtd_set_profiling(h, on):
    _check(h, load_library().fdtd_set_profiling(h, int(bool(on))), "fdtd_set_profiling")


def fdtd_get_timings(h):
    t = Timings()
    _check(h, load_library().fdtd_get_timings(h, C.byref(t)), "fdtd_get_timings")
    return {k: getattr(t, k) for k, _ in Timings._fields_}


def fdtd_reset_timings(h):
    _check(h, load_library().fdtd_reset_timings(h), "fdtd_reset_timings")


def fdtd_get_info(h):
    dt, nd, ng, b = C.c_double(), C.c_size_t(), C.c_size_t(), C.c_size_t()
    _check(h, load_library().fdtd_get_info(h, C.byref(dt), C.byref(nd), C.byref(ng), C.byref(b)),
           "fdtd_get_info")
    return {"dt": dt.value, "n_design": nd.value, "n_gap": ng.value, "device_bytes": b.value}


def fdtd_cancel(h):
    _check(h, load_library().fdtd_cancel(h), "fdtd_cancel")


def fdtd_last_error(h):
    m = load_library().fdtd_last_error(h)
    return m.decode() if m else ""


def fdtd_gradient_static(dft_fwd, dft_adj, rho, design_box, gap_box, n_freq, dy_drho, grad, stream=None,
                         norm=True):
    """No-allocation gradient from caller-owned device buffers (torch CUDA tensors): dft_fwd,
    dft_adj float64 (interleaved complex, (n_freq, 3, dnz, dny, dnx) over design_box), rho
    float32/float64 (one per design voxel), grad float64 (one per design voxel, written).  dy_drho:
    host array (3, n_freq, 4).  Returns the squared norm of the gradient (the call then waits for
    the stream), or None with norm=False (the call only enqueues work on the stream).

    Every buffer size is checked here against design_box and n_freq, before the call: an undersized
    buffer would make the kernel read or write past its end."""
    import torch
    for name, t in (("dft_fwd", dft_fwd), ("dft_adj", dft_adj), ("grad", grad)):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if not (rho.is_cuda and rho.is_contiguous() and rho.dtype in (torch.float32, torch.float64)):
        raise TypeError("rho must be a contiguous float32/float64 CUDA tensor")
    db_l = [int(x) for x in design_box]
    if len(db_l) != 6 or any(db_l[2 * a + 1] <= db_l[2 * a] for a in range(3)):
        raise ValueError("design_box must be 6 ints with a non-empty extent on every axis")
    nd = (db_l[1] - db_l[0]) * (db_l[3] - db_l[2]) * (db_l[5] - db_l[4])
    nf = int(n_freq)
    if dft_fwd.numel() != 6 * nf * nd or dft_adj.numel() != 6 * nf * nd:
        raise ValueError(f"dft_fwd and dft_adj must hold 2*3*n_freq*nd = {6 * nf * nd} doubles")
    if rho.numel() < nd or grad.numel() < nd:
        raise ValueError(f"rho and grad must hold at least nd = {nd} values")
    cst = np.ascontiguousarray(dy_drho, dtype=np.float64)
    if cst.shape != (3, nf, 4):
        raise ValueError(f"dy_drho must have shape (3, n_freq, 4) = (3, {nf}, 4)")
    db = (C.c_int * 6)(*db_l)
    gb = (C.c_int * 6)(*[int(x) for x in gap_box]) if gap_box is not None else None
    cst = cst.ravel()
    norm2 = C.c_double()
    rc = load_library().fdtd_gradient_static(C.c_void_p(dft_fwd.data_ptr()), C.c_void_p(dft_adj.data_ptr()),
                                             C.c_void_p(rho.data_ptr()), 0 if rho.dtype == torch.float32 else 1,
                                             db, gb, nf, _dptr(cst), C.c_void_p(grad.data_ptr()),
                                             C.byref(norm2) if norm else None, C.c_void_p(stream or 0))
    if rc != FDTD_OK:
        raise FdtdError(rc, load_library().fdtd_last_error(None).decode())
    return norm2.value if norm else None


MAX_BATCH = 16


def _check_batch(rc, what):
    if rc != FDTD_OK:
        msg = load_library().fdtd_last_error(None)
        raise FdtdError(rc, f"{what}: {msg.decode() if msg else ''}")


def fdtd_batch_create(stream=None):
    b = C.c_void_p()
    _check_batch(load_library().fdtd_batch_create(C.c_void_p(stream or 0), C.byref(b)), "fdtd_batch_create")
    return b


def fdtd_batch_submit(b, h, adjoint=False):
    lib = load_library()
    rc = lib.fdtd_batch_submit(b, h, int(bool(adjoint)))
    if rc != FDTD_OK:
        msg = (lib.fdtd_last_error(h) if h else b"") or lib.fdtd_last_error(None)
        raise FdtdError(rc, "fdtd_batch_submit: " + (msg.decode() if msg else ""))


def fdtd_batch_run(b, max_steps):
    """One persistent launch; returns [(handle value, status), ...] of the runs that ended."""
    done = (C.c_void_p * MAX_BATCH)()
    st = (C.c_int * MAX_BATCH)()
    n = C.c_int()
    _check_batch(load_library().fdtd_batch_run(b, int(max_steps), done, st, MAX_BATCH, C.byref(n)), "fdtd_batch_run")
    return [(done[q], st[q]) for q in range(n.value)]


def fdtd_batch_set_wait_limit(b, wait_ns, gate=False):
    _check_batch(load_library().fdtd_batch_set_wait_limit(b, int(wait_ns), int(bool(gate))), "fdtd_batch_set_wait_limit")


def fdtd_batch_set_blocks(b, blocks):
    _check_batch(load_library().fdtd_batch_set_blocks(b, int(blocks)), "fdtd_batch_set_blocks")


def fdtd_batch_info(b):
    n, l = C.c_int(), C.c_longlong()
    _check_batch(load_library().fdtd_batch_info(b, C.byref(n), C.byref(l)), "fdtd_batch_info")
    return {"runs": n.value, "launches": l.value}


def fdtd_batch_destroy(b):
    if b:
        load_library().fdtd_batch_destroy(b)


def fdtd_get_objective(h, n_gap_doubles=0):
    F = C.c_double()
    g = np.zeros(max(n_gap_doubles, 1), dtype=np.float64)
    _check(h, load_library().fdtd_get_objective(h, C.byref(F), _dptr(g) if n_gap_doubles else None),
           "fdtd_get_objective")
    return F.value, g[:n_gap_doubles]


def _f32_dev(t, name):
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def fdtd_filter_project(rho, rho_t, rho_b, R, beta, eta, stream=None):
    """Filter + projection of a (nz, ny, nx) float32 CUDA tensor into rho_t, rho_b (same shape)."""
    nz, ny, nx = rho.shape
    rc = load_library().fdtd_filter_project(_f32_dev(rho, "rho"), _f32_dev(rho_t, "rho_t"), _f32_dev(rho_b, "rho_b"),
                                            nx, ny, nz, float(R), float(beta), float(eta), C.c_void_p(stream or 0))
    if rc != FDTD_OK:
        raise FdtdError(rc, load_library().fdtd_last_error(None).decode())


def fdtd_filter_project_grad(rho_t, dF_drho_b, dF_drho, R, beta, eta, stream=None):
    nz, ny, nx = rho_t.shape
    rc = load_library().fdtd_filter_project_grad(_f32_dev(rho_t, "rho_t"), _f32_dev(dF_drho_b, "dF_drho_b"),
                                                 _f32_dev(dF_drho, "dF_drho"), nx, ny, nz, float(R), float(beta),
                                                 float(eta), C.c_void_p(stream or 0))
    if rc != FDTD_OK:
        raise FdtdError(rc, load_library().fdtd_last_error(None).decode())


def fdtd_destroy(h):
    if h:
        load_library().fdtd_destroy(h)
