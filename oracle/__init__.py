"""ctypes binding of the plain FP64 CPU oracle (``oracle/fdtd_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline/reference leg of ``bench.py``; never by the product package.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboracle.so")


class _Desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("courant", C.c_double), ("n_steps", C.c_int),
                ("cpml", C.c_int * 6),
                ("cpml_m", C.c_double), ("cpml_sigma_scale", C.c_double),
                ("cpml_kappa_max", C.c_double), ("cpml_a_max", C.c_double),
                ("bc", C.c_int * 3),
                ("design_box", C.c_int * 6), ("gap_box", C.c_int * 6),
                ("n_freq", C.c_int), ("freqs_hz", C.POINTER(C.c_double)),
                ("freq_weights", C.POINTER(C.c_double)),
                ("src_kind", C.c_int), ("src_comp", C.c_int), ("src_pos", C.c_int * 3),
                ("src_f0", C.c_double), ("src_fwhm_hz", C.c_double), ("src_t0", C.c_double),
                ("src_amp", C.c_double), ("adj_tau", C.c_double), ("src_wave", C.POINTER(C.c_double)),
                ("density_layout", C.c_int)]


class _Mat(C.Structure):
    _fields_ = [("eps_inf", C.c_double * 3), ("sigma", C.c_double * 3), ("n_poles", C.c_int * 3),
                ("a_re", C.POINTER(C.c_double) * 3), ("a_im", C.POINTER(C.c_double) * 3),
                ("c_re", C.POINTER(C.c_double) * 3), ("c_im", C.POINTER(C.c_double) * 3)]


_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        from . import build as _b
        _b.build()
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    lib.oracle_create.argtypes = [P(_Desc), P(C.c_void_p)]
    lib.oracle_set_materials.argtypes = [C.c_void_p, P(_Mat), P(_Mat), P(_Mat), C.c_double]
    lib.oracle_set_density.argtypes = [C.c_void_p, P(C.c_double), C.c_size_t]
    lib.oracle_forward.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double)]
    lib.oracle_adjoint.argtypes = [C.c_void_p]
    lib.oracle_gradient.argtypes = [C.c_void_p, P(C.c_double), C.c_size_t]
    lib.oracle_tangent.argtypes = [C.c_void_p, P(C.c_double), C.c_size_t, P(C.c_double), P(C.c_double),
                                   P(C.c_double), P(C.c_double)]
    lib.oracle_paper_objective.argtypes = [C.c_void_p, P(C.c_double)]
    lib.oracle_paper_gradient.argtypes = [C.c_void_p, C.c_int, P(C.c_double), P(C.c_double), C.c_size_t]
    lib.oracle_reset.argtypes = [C.c_void_p]
    lib.oracle_step.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
    lib.oracle_get_field.argtypes = [C.c_void_p, C.c_int, P(C.c_double), C.c_size_t]
    lib.oracle_set_field.argtypes = [C.c_void_p, C.c_int, P(C.c_double), C.c_size_t]
    lib.oracle_get_dft.argtypes = [C.c_void_p, C.c_int, P(C.c_double), C.c_size_t]
    lib.oracle_get_source.argtypes = [C.c_void_p, C.c_int, P(C.c_double), C.c_size_t]
    lib.oracle_get_index_map.argtypes = [C.c_void_p, C.c_int, P(C.c_int32), C.c_size_t]
    lib.oracle_sample_response.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int,
                                           P(C.c_double), P(C.c_double)]
    lib.oracle_dt.argtypes = [C.c_void_p]
    lib.oracle_dt.restype = C.c_double
    lib.oracle_last_error.argtypes = [C.c_void_p]
    lib.oracle_last_error.restype = C.c_char_p
    lib.oracle_destroy.argtypes = [C.c_void_p]
    lib.oracle_destroy.restype = None
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _make_mat(m, keep):
    s = _Mat()
    for k in range(3):
        s.eps_inf[k] = float(m["eps_inf"][k])
        s.sigma[k] = float(m["sigma"][k])
        poles = m["poles"][k]
        s.n_poles[k] = len(poles)
        arrs = [np.ascontiguousarray([complex(a).real for a, _ in poles] or [0.0], dtype=np.float64),
                np.ascontiguousarray([complex(a).imag for a, _ in poles] or [0.0], dtype=np.float64),
                np.ascontiguousarray([complex(c).real for _, c in poles] or [0.0], dtype=np.float64),
                np.ascontiguousarray([complex(c).imag for _, c in poles] or [0.0], dtype=np.float64)]
        keep.extend(arrs)
        s.a_re[k], s.a_im[k], s.c_re[k], s.c_im[k] = (_dptr(x) for x in arrs)
    return s


class OracleError(RuntimeError):
    pass


class Oracle:
    """One oracle problem.  ``desc`` is a grid-description dict (see ``synth.base_desc``)."""

    def __init__(self, desc):
        self.lib = load()
        self.desc = dict(desc)
        d = _Desc()
        for key in ("nx", "ny", "nz", "n_steps", "src_kind", "src_comp"):
            setattr(d, key, int(desc[key]))
        self.layout = int(desc.get("density_layout", 0))
        d.density_layout = self.layout
        for key in ("dx", "courant", "cpml_m", "cpml_sigma_scale", "cpml_kappa_max", "cpml_a_max",
                    "src_f0", "src_fwhm_hz", "src_t0", "src_amp", "adj_tau"):
            setattr(d, key, float(desc[key]))
        for key, n in (("cpml", 6), ("design_box", 6), ("gap_box", 6), ("src_pos", 3)):
            for i in range(n):
                getattr(d, key)[i] = int(desc[key][i])
        bc = desc.get("bc", (0, 0, 0))
        for i in range(3):
            d.bc[i] = int(bc[i])
        self._freqs = np.ascontiguousarray(desc["freqs_hz"], dtype=np.float64)
        self._w = np.ascontiguousarray(desc["freq_weights"], dtype=np.float64)
        d.n_freq = len(self._freqs)
        d.freqs_hz = _dptr(self._freqs)
        d.freq_weights = _dptr(self._w)
        if desc.get("src_wave") is not None:
            self._wave = np.ascontiguousarray(desc["src_wave"], dtype=np.float64)
            if self._wave.size != 2 * int(desc["n_steps"]) + 1:
                raise ValueError("src_wave needs 2 n_steps + 1 samples (t = s dt / 2)")
            d.src_wave = _dptr(self._wave)
        self._d = d
        h = C.c_void_p()
        if self.lib.oracle_create(C.byref(d), C.byref(h)) != 0:
            raise OracleError("oracle_create failed (see stderr)")
        self.h = h
        self.n = (int(desc["nz"]), int(desc["ny"]), int(desc["nx"]))
        db = desc["design_box"]
        gb = desc["gap_box"]
        self.dshape = (db[5] - db[4], db[3] - db[2], db[1] - db[0]) if db[1] > db[0] else (0, 0, 0)
        self.wshape = self.dshape          # DFT arrays: the working box
        self.vshape = self.dshape          # design variables
        if self.layout == 1 and db[1] > db[0]:
            # one density per E sample: E_k spans the design voxels extended on the +l faces, l != k
            nz, ny, nx = self.dshape
            self.wshape = (nz + 1, ny + 1, nx + 1)
            self.sample_shapes = [(nz + 1, ny + 1, nx), (nz + 1, ny, nx + 1), (nz, ny + 1, nx + 1)]
            self.vshape = (sum(a * b * c for a, b, c in self.sample_shapes),)
        self.gshape = (gb[5] - gb[4], gb[3] - gb[2], gb[1] - gb[0]) if gb[1] > gb[0] else (0, 0, 0)
        self.nf = len(self._freqs)

    def _check(self, rc, what):
        if rc != 0:
            raise OracleError(f"{what}: {self.lib.oracle_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.oracle_destroy(self.h)
            self.h = None

    __del__ = close

    @property
    def dt(self):
        return self.lib.oracle_dt(self.h)

    def set_materials(self, bg, m1, m2, gamma=0.0):
        keep = []
        b, a1, a2 = _make_mat(bg, keep), _make_mat(m1, keep), _make_mat(m2, keep)
        self._check(self.lib.oracle_set_materials(self.h, C.byref(b), C.byref(a1), C.byref(a2),
                                                  float(gamma)), "set_materials")

    def set_density(self, rho):
        r = np.ascontiguousarray(rho, dtype=np.float64).ravel()
        self._check(self.lib.oracle_set_density(self.h, _dptr(r), r.size), "set_density")

    def forward(self):
        F = C.c_double()
        ng = int(np.prod(self.gshape))
        g = np.zeros(2 * self.nf * 3 * ng, dtype=np.float64)
        self._check(self.lib.oracle_forward(self.h, C.byref(F), _dptr(g)), "forward")
        gd = (g[0::2] + 1j * g[1::2]).reshape((self.nf, 3) + self.gshape)
        return F.value, gd

    def adjoint(self):
        self._check(self.lib.oracle_adjoint(self.h), "adjoint")

    def gradient(self):
        g = np.zeros(self.vshape, dtype=np.float64)
        self._check(self.lib.oracle_gradient(self.h, _dptr(g), g.size), "gradient")
        return g

    def tangent(self, drho, time_domain=False):
        """(F, dF): the forward objective and its exact derivative along the density direction drho
        (forward-mode differentiation of the discrete scheme; see fdtd_oracle.h); with time_domain, the
        paper-mode energy objective and its derivative instead."""
        d = np.ascontiguousarray(drho, dtype=np.float64).ravel()
        F, dF, Ft, dFt = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        self._check(self.lib.oracle_tangent(self.h, _dptr(d), d.size, C.byref(F), C.byref(dF), C.byref(Ft),
                                            C.byref(dFt)), "tangent")
        return (Ft.value, dFt.value) if time_domain else (F.value, dF.value)

    def paper_objective(self):
        """Time-domain objective of Eq. (Objective_analyitically_enhancement) (paper mode)."""
        F = C.c_double()
        self._check(self.lib.oracle_paper_objective(self.h, C.byref(F)), "paper_objective")
        return F.value

    def paper_gradient(self, align=0):
        """(F_td, gradient of Eq. (Gradient_FDTD) per design voxel); align: see fdtd_oracle.h."""
        F = C.c_double()
        g = np.zeros(self.dshape, dtype=np.float64)
        self._check(self.lib.oracle_paper_gradient(self.h, int(align), C.byref(F), _dptr(g), g.size), "paper_gradient")
        return F.value, g

    def reset(self):
        self._check(self.lib.oracle_reset(self.h), "reset")

    def step(self, n_first, n_count, source_mode=0):
        self._check(self.lib.oracle_step(self.h, n_first, n_count, source_mode), "step")

    def get_field(self, which):
        a = np.zeros(self.n, dtype=np.float64)
        self._check(self.lib.oracle_get_field(self.h, which, _dptr(a), a.size), "get_field")
        return a

    def set_field(self, which, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        self._check(self.lib.oracle_set_field(self.h, which, _dptr(a), a.size), "set_field")

    def get_dft(self, adjoint=False):
        n = 2 * self.nf * 3 * int(np.prod(self.wshape))
        a = np.zeros(n, dtype=np.float64)
        self._check(self.lib.oracle_get_dft(self.h, 1 if adjoint else 0, _dptr(a), n), "get_dft")
        return (a[0::2] + 1j * a[1::2]).reshape((self.nf, 3) + self.wshape)

    def get_source(self, which):
        M = int(self.desc["n_steps"])
        n = 3 * int(np.prod(self.gshape)) * M if which == 3 else M
        a = np.zeros(n, dtype=np.float64)
        self._check(self.lib.oracle_get_source(self.h, which, _dptr(a), n), "get_source")
        return a.reshape((3 * int(np.prod(self.gshape)), M)) if which == 3 else a

    def get_index_map(self, which):
        shape = ((3,) + self.n) if which <= 1 else self.n
        a = np.zeros(shape, dtype=np.int32)
        self._check(self.lib.oracle_get_index_map(self.h, which,
                                                  a.ctypes.data_as(C.POINTER(C.c_int32)), a.size),
                    "get_index_map")
        return a

    def sample_response(self, comp, rho, curl):
        c = np.ascontiguousarray(curl, dtype=np.float64)
        e = np.zeros_like(c)
        self._check(self.lib.oracle_sample_response(self.h, comp, float(rho), c.size, _dptr(c),
                                                    _dptr(e)), "sample_response")
        return e


def problem(w):
    """Oracle set up for a workload dict (desc, bg, m1, m2, gamma, rho) from ``synth``."""
    o = Oracle(w["desc"])
    o.set_materials(w["bg"], w["m1"], w["m2"], w.get("gamma", 0.0))
    if w.get("rho") is not None:
        o.set_density(w["rho"])
    return o
