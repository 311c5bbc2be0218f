"""Thin ctypes binding of libjgs2.so (argument marshalling only; every step of the sweep runs
in the library's CUDA kernels). Names follow the C ABI in include/jgs2.h.

Device state is passed as torch CUDA tensors (torch supplies device memory and streams);
host arrays as numpy. There is no CPU fallback: if the shared library is missing or a
call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libjgs2.so")

TRACE_MAX = 4096
NKERNELS = 11
KERNEL_NAMES = ["k_pool", "k_gather", "k_correct", "k_energy", "k_update", "setup", "contact", "k_elem",
                "k_pair_trials", "k_ls_decide", "k_batch_persistent"]
FP64, FP32 = 0, 1
CORR_ASM, CORR_ELEM, CORR_OFF = 0, 1, 2
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTPRECOMPUTED", 5: "ENOTCONVERGED",
          6: "EDIVERGED", 7: "ENONSPD", 8: "ETIMEOUT", 9: "EINTERSECT"}


class MeshDesc(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("n_tets", C.c_int32),
                ("rest_pos", C.POINTER(C.c_double)), ("tets", C.POINTER(C.c_int32)),
                ("youngs", C.POINTER(C.c_double)), ("poisson", C.POINTER(C.c_double)),
                ("density", C.POINTER(C.c_double)), ("pinned", C.POINTER(C.c_uint8)),
                ("gravity", C.c_double * 3), ("dt", C.c_double),
                ("contact", C.c_int32), ("n_planes", C.c_int32), ("planes", C.POINTER(C.c_double)),
                ("dhat", C.c_double), ("kappa", C.c_double),
                ("friction_mu", C.c_double), ("friction_eps_v", C.c_double)]


class ClothDesc(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("n_tris", C.c_int32),
                ("rest_pos", C.POINTER(C.c_double)), ("tris", C.POINTER(C.c_int32)),
                ("youngs", C.c_double), ("poisson", C.c_double), ("thickness", C.c_double),
                ("density", C.c_double), ("bend", C.c_double), ("pinned", C.POINTER(C.c_uint8)),
                ("gravity", C.c_double * 3), ("dt", C.c_double),
                ("n_planes", C.c_int32), ("planes", C.POINTER(C.c_double)), ("dhat", C.c_double),
                ("kappa", C.c_double)]


class ClothReport(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("converged", C.c_int32), ("ls_rejects", C.c_int32), ("pad_", C.c_int32),
                ("rel_residual", C.c_double), ("g0", C.c_double)]


class PrecomputeOpts(C.Structure):
    _fields_ = [("n_cub", C.c_int32), ("n_train", C.c_int32), ("n_cand", C.c_int32),
                ("n_pool", C.c_int32), ("nnls_tol", C.c_double), ("seed", C.c_uint64),
                ("n_threads", C.c_int32), ("gs", C.c_int32), ("gpu", C.c_int32)]


class CubatureBlob(C.Structure):
    _fields_ = [("n_cub", C.c_int32), ("elem", C.POINTER(C.c_int32)),
                ("weight", C.POINTER(C.c_double)), ("ubar", C.POINTER(C.c_double))]


class StepOpts(C.Structure):
    _fields_ = [("max_sweeps", C.c_int32), ("rel_tol", C.c_double), ("precision", C.c_int32),
                ("correction", C.c_int32), ("line_search", C.c_int32), ("check_every", C.c_int32),
                ("record_trace", C.c_int32), ("profile", C.c_int32), ("dx_tol", C.c_double),
                ("length_scale", C.c_double), ("persistent", C.c_int32), ("wait_polls", C.c_int32),
                ("test_unreachable_barrier", C.c_int32), ("contact_coupling", C.c_int32)]


class AdjointOpts(C.Structure):
    _fields_ = [("max_iters", C.c_int32), ("rel_tol", C.c_double), ("precision", C.c_int32),
                ("correction", C.c_int32), ("check_every", C.c_int32)]


class AdjointReport(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("rel_residual", C.c_double),
                ("ms", C.c_double)]


class StepReport(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("converged", C.c_int32), ("fallback", C.c_int32),
                ("ls_rejects", C.c_int32), ("dj_steps", C.c_int32), ("contact_rebuilds", C.c_int32),
                ("contact_candidates", C.c_int32), ("contact_near", C.c_int32),
                ("rel_residual", C.c_double), ("g0", C.c_double),
                ("ms", C.c_double), ("launches", C.c_int32), ("profiled_sweeps", C.c_int32),
                ("kernel_launches", C.c_int32 * NKERNELS), ("kernel_ms", C.c_double * NKERNELS),
                ("trace_len", C.c_int32), ("trace", C.c_double * TRACE_MAX),
                ("stopped_dx", C.c_int32), ("pad_", C.c_int32), ("last_dx", C.c_double),
                ("ls_passes", C.c_int32 * 3), ("pad2_", C.c_int32)]


_lib = None

EXPORTS = ["jgs2_precompute_opts_default", "jgs2_step_opts_default", "jgs2_mesh_create",
           "jgs2_precompute", "jgs2_precompute_import", "jgs2_precompute_export",
           "jgs2_mesh_n_cub", "jgs2_step", "jgs2_step_gs", "jgs2_step_host", "jgs2_sweeps",
           "jgs2_energy_gradient", "jgs2_energy_gradient_static", "jgs2_contact_pairs",
           "jgs2_step_adjoint", "jgs2_adjoint_opts_default", "jgs2_mesh_set_youngs",
           "jgs2_mesh_create_batch", "jgs2_batch_report", "jgs2_autotune", "jgs2_mesh_launch_config", "jgs2_alu_peak",
           "jgs2_cloth_create", "jgs2_cloth_step", "jgs2_cloth_sweeps", "jgs2_cloth_energy_gradient",
           "jgs2_cloth_n_hinges", "jgs2_cloth_destroy", "jgs2_mesh_destroy", "jgs2_last_error"]


def lib():
    """Loads libjgs2.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libjgs2.so not built ({LIB_PATH}); run python -m paper_2506_06494_b300.build")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    L.jgs2_precompute_opts_default.argtypes = [C.POINTER(PrecomputeOpts)]
    L.jgs2_step_opts_default.argtypes = [C.POINTER(StepOpts)]
    L.jgs2_mesh_create.argtypes = [C.POINTER(MeshDesc), C.POINTER(P)]
    L.jgs2_precompute.argtypes = [P, C.POINTER(PrecomputeOpts)]
    L.jgs2_precompute_import.argtypes = [P, C.POINTER(CubatureBlob)]
    L.jgs2_precompute_export.argtypes = [P, P, P, P, P]
    L.jgs2_mesh_n_cub.argtypes = [P]
    L.jgs2_mesh_n_cub.restype = C.c_int32
    L.jgs2_step.argtypes = [P, P, P, C.POINTER(StepOpts), P, C.POINTER(StepReport)]
    L.jgs2_step_gs.argtypes = [P, P, P, C.POINTER(StepOpts), P, C.POINTER(StepReport)]
    L.jgs2_step_host.argtypes = [P, P, P, C.POINTER(StepOpts), P, C.POINTER(StepReport)]
    L.jgs2_sweeps.argtypes = [P, P, P, P, C.c_int32, C.POINTER(StepOpts), P]
    L.jgs2_energy_gradient.argtypes = [P, P, P, P, P, P, P]
    L.jgs2_contact_pairs.argtypes = [P, P, P, C.c_double, P, C.c_int32, C.POINTER(C.c_int32), P]
    L.jgs2_contact_pairs.restype = C.c_int
    L.jgs2_adjoint_opts_default.argtypes = [C.POINTER(AdjointOpts)]
    L.jgs2_step_adjoint.argtypes = [P] * 9 + [C.POINTER(AdjointOpts), P, C.POINTER(AdjointReport)]
    L.jgs2_mesh_set_youngs.argtypes = [P, P]
    L.jgs2_mesh_create_batch.argtypes = [C.POINTER(MeshDesc), C.c_int32, C.POINTER(P)]
    L.jgs2_batch_report.argtypes = [P, P, P, P]
    L.jgs2_autotune.argtypes = [P, P, P, C.POINTER(StepOpts), P, C.POINTER(C.c_int32)]
    L.jgs2_alu_peak.argtypes = [C.c_int32, C.POINTER(C.c_double), P]
    L.jgs2_mesh_launch_config.argtypes = [P, C.c_int32, P]
    L.jgs2_mesh_destroy.argtypes = [P]
    L.jgs2_cloth_create.argtypes = [C.POINTER(ClothDesc), C.POINTER(P)]
    L.jgs2_cloth_step.argtypes = [P, P, P, C.POINTER(StepOpts), P, C.POINTER(ClothReport)]
    L.jgs2_cloth_sweeps.argtypes = [P, P, P, P, C.c_int32, C.POINTER(StepOpts), P]
    L.jgs2_cloth_energy_gradient.argtypes = [P, P, P, P, P, P, P]
    L.jgs2_cloth_n_hinges.argtypes = [P]
    L.jgs2_cloth_n_hinges.restype = C.c_int32
    L.jgs2_cloth_destroy.argtypes = [P]
    L.jgs2_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("jgs2_mesh_destroy", "jgs2_last_error", "jgs2_mesh_n_cub", "jgs2_cloth_destroy",
                        "jgs2_cloth_n_hinges", "jgs2_precompute_opts_default", "jgs2_step_opts_default",
                        "jgs2_adjoint_opts_default"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


class JGS2Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status, ok=(0,)):
    if status not in ok:
        raise JGS2Error(status, lib().jgs2_last_error().decode())
    return status


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def alu_peak(precision, stream=None) -> float:
    """jgs2_alu_peak: the current device's measured FMA throughput in GFLOP/s."""
    g = C.c_double()
    _check(lib().jgs2_alu_peak(int(precision), C.byref(g), C.c_void_p(_stream_ptr(stream))))
    return g.value


def step_opts(**kw) -> StepOpts:
    o = StepOpts()
    lib().jgs2_step_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def precompute_opts(**kw) -> PrecomputeOpts:
    o = PrecomputeOpts()
    lib().jgs2_precompute_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def adjoint_opts(**kw) -> AdjointOpts:
    o = AdjointOpts()
    lib().jgs2_adjoint_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _dev(t):
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), \
        "device state must be a contiguous float64 CUDA tensor [V,3]"
    return C.c_void_p(t.data_ptr())


def _desc(X, tets, youngs, poisson, density, pinned, gravity, dt, planes, dhat, kappa, contact, keep,
          friction_mu=0.0, friction_eps_v=1e-3):
    arrs = [np.ascontiguousarray(X, dtype=np.float64),
            np.ascontiguousarray(tets, dtype=np.int32),
            np.ascontiguousarray(youngs, dtype=np.float64),
            np.ascontiguousarray(poisson, dtype=np.float64),
            np.ascontiguousarray(density, dtype=np.float64),
            None if pinned is None else np.ascontiguousarray(pinned, dtype=np.uint8),
            np.ascontiguousarray(np.zeros((0, 4)) if planes is None else planes, dtype=np.float64)]
    keep.extend(arrs)
    X, T, E, nu, rho, pin, pl = arrs
    d = MeshDesc()
    d.n_vertices = X.shape[0]
    d.n_tets = T.shape[0]
    d.rest_pos = _ptr(X, C.c_double)
    d.tets = _ptr(T, C.c_int32)
    d.youngs = _ptr(E, C.c_double)
    d.poisson = _ptr(nu, C.c_double)
    d.density = _ptr(rho, C.c_double)
    d.pinned = _ptr(pin, C.c_uint8) if pin is not None else C.POINTER(C.c_uint8)()
    for q in range(3):
        d.gravity[q] = float(gravity[q])
    d.dt = float(dt)
    d.contact = int(contact)
    d.n_planes = int(pl.shape[0])
    d.planes = _ptr(pl, C.c_double)
    d.dhat = float(dhat)
    d.kappa = float(kappa)
    d.friction_mu = float(friction_mu)
    d.friction_eps_v = float(friction_eps_v)
    return d


class Mesh:
    """A tet mesh living on the current CUDA device (jgs2_mesh_create)."""

    @classmethod
    def batch(cls, scenes_list):
        """Several independent scenes in one mesh (jgs2_mesh_create_batch)."""
        self = cls.__new__(cls)
        self._keep = []
        descs = (MeshDesc * len(scenes_list))()
        for k, s in enumerate(scenes_list):
            descs[k] = _desc(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned, s.gravity, s.dt,
                             None, s.dhat, s.kappa, 0, self._keep)
        h = C.c_void_p()
        _check(lib().jgs2_mesh_create_batch(descs, len(scenes_list), C.byref(h)))
        self.handle = h
        self.V = int(sum(s.n_vertices for s in scenes_list))
        self.T = int(sum(s.n_tets for s in scenes_list))
        self.n_scenes = len(scenes_list)
        return self

    def batch_report(self):
        n = self.n_scenes
        sw, cv, rr = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n)
        _check(lib().jgs2_batch_report(self.handle, sw.ctypes.data, cv.ctypes.data, rr.ctypes.data))
        return sw, cv, rr

    def autotune(self, x, v, opts=None, stream=None):
        bs = C.c_int32()
        _check(lib().jgs2_autotune(self.handle, _dev(x), _dev(v), C.byref(opts or step_opts()),
                                   C.c_void_p(_stream_ptr(stream)), C.byref(bs)))
        return bs.value

    def launch_config(self, precision):
        """(gather threads per block, gather threads per vertex, correction threads per block,
        correction slot prefetch)."""
        cfg = np.zeros(4, dtype=np.int32)
        _check(lib().jgs2_mesh_launch_config(self.handle, int(precision), cfg.ctypes.data))
        return tuple(int(c) for c in cfg)

    def __init__(self, X, tets, youngs, poisson, density, pinned=None, gravity=(0, 0, -9.8), dt=1 / 120,
                 planes=None, dhat=1e-3, kappa=1e5, contact=0, friction_mu=0.0, friction_eps_v=1e-3):
        self._keep = []
        d = _desc(X, tets, youngs, poisson, density, pinned, gravity, dt, planes, dhat, kappa, contact, self._keep,
                  friction_mu, friction_eps_v)
        h = C.c_void_p()
        _check(lib().jgs2_mesh_create(C.byref(d), C.byref(h)))
        self.handle = h
        self.V = int(d.n_vertices)
        self.T = int(d.n_tets)

    @classmethod
    def from_scene(cls, s, contact=None, friction_mu=0.0, friction_eps_v=1e-3):
        c = s.contact if contact is None else contact
        return cls(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned, s.gravity, s.dt,
                   s.planes, s.dhat, s.kappa, c, friction_mu, friction_eps_v)

    def contact_pairs(self, x_t, x, radius, cap=1 << 20, stream=None):
        """Canonical candidate pair rows (kind, a, b, c, d) within radius (jgs2_contact_pairs)."""
        out = np.zeros((cap, 5), np.int32)
        n = C.c_int32()
        _check(lib().jgs2_contact_pairs(self.handle, _dev(x_t), _dev(x), float(radius), out.ctypes.data, cap,
                                        C.byref(n), C.c_void_p(_stream_ptr(stream))))
        return out[:n.value].copy()

    def close(self):
        if getattr(self, "handle", None):
            lib().jgs2_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def precompute(self, **kw):
        o = precompute_opts(**kw)
        _check(lib().jgs2_precompute(self.handle, C.byref(o)))

    def precompute_import(self, elem, weight, ubar):
        elem = np.ascontiguousarray(elem, dtype=np.int32)
        weight = np.ascontiguousarray(weight, dtype=np.float64)
        ubar = np.ascontiguousarray(ubar, dtype=np.float64)
        V, nc = elem.shape
        assert V == self.V and weight.shape == (V, nc) and ubar.size == V * nc * 36
        b = CubatureBlob()
        b.n_cub = nc
        b.elem = _ptr(elem, C.c_int32)
        b.weight = _ptr(weight, C.c_double)
        b.ubar = _ptr(ubar, C.c_double)
        _check(lib().jgs2_precompute_import(self.handle, C.byref(b)))

    def precompute_export(self):
        nc = lib().jgs2_mesh_n_cub(self.handle)
        elem = np.zeros((self.V, nc), np.int32)
        w = np.zeros((self.V, nc))
        u = np.zeros((self.V, nc, 4, 3, 3))
        r = np.zeros(self.V)
        _check(lib().jgs2_precompute_export(self.handle, elem.ctypes.data, w.ctypes.data, u.ctypes.data,
                                            r.ctypes.data))
        return elem, w, u, r

    def step(self, x, v, opts=None, stream=None, report=None):
        """jgs2_step on float64 CUDA tensors x, v [V,3] (updated in place)."""
        opts = opts or step_opts()
        rep = report if report is not None else StepReport()
        st = lib().jgs2_step(self.handle, _dev(x), _dev(v), C.byref(opts), C.c_void_p(_stream_ptr(stream)),
                             C.byref(rep))
        _check(st, ok=(0, 5))
        return rep

    def step_gs(self, x, v, opts=None, stream=None, report=None):
        """jgs2_step_gs (Gauss-Seidel sweeps) on float64 CUDA tensors x, v [V,3]."""
        opts = opts or step_opts()
        rep = report if report is not None else StepReport()
        st = lib().jgs2_step_gs(self.handle, _dev(x), _dev(v), C.byref(opts), C.c_void_p(_stream_ptr(stream)),
                                C.byref(rep))
        _check(st, ok=(0, 5))
        return rep

    def step_host(self, x, v, opts=None, stream=None, report=None):
        """jgs2_step_host on C-contiguous float64 numpy arrays (updated in place)."""
        assert x.dtype == np.float64 and v.dtype == np.float64 and x.flags.c_contiguous and v.flags.c_contiguous
        opts = opts or step_opts()
        rep = report if report is not None else StepReport()
        st = lib().jgs2_step_host(self.handle, x.ctypes.data, v.ctypes.data, C.byref(opts),
                                  C.c_void_p(_stream_ptr(stream)), C.byref(rep))
        _check(st, ok=(0, 5))
        return rep

    def sweeps(self, x_t, v_t, x_k, n, opts=None, stream=None):
        opts = opts or step_opts()
        _check(lib().jgs2_sweeps(self.handle, _dev(x_t), _dev(v_t), _dev(x_k), int(n), C.byref(opts),
                                 C.c_void_p(_stream_ptr(stream))))

    def set_youngs(self, youngs):
        E = np.ascontiguousarray(youngs, dtype=np.float64)
        assert E.shape == (self.T,)
        _check(lib().jgs2_mesh_set_youngs(self.handle, E.ctypes.data))

    def step_adjoint(self, x_t, v_t, x_t1, gx_t1, gv_t1, gE=None, opts=None, stream=None):
        """jgs2_step_adjoint on CUDA tensors; returns (gx_t, gv_t, gE, report). gE accumulates."""
        import torch
        gx = torch.empty_like(x_t)
        gv = torch.empty_like(x_t)
        if gE is None:
            gE = torch.zeros(self.T, dtype=torch.float64, device=x_t.device)
        rep = AdjointReport()
        st = lib().jgs2_step_adjoint(self.handle, _dev(x_t), _dev(v_t), _dev(x_t1), _dev(gx_t1), _dev(gv_t1),
                                     _dev(gx), _dev(gv), C.c_void_p(gE.data_ptr()), C.byref(opts or adjoint_opts()),
                                     C.c_void_p(_stream_ptr(stream)), C.byref(rep))
        _check(st, ok=(0, 5))
        return gx, gv, gE, rep

    def energy_gradient(self, x_t, v_t, x, stream=None):
        import torch
        g = torch.empty_like(x)
        E = C.c_double()
        _check(lib().jgs2_energy_gradient(self.handle, _dev(x_t), _dev(v_t), _dev(x), C.byref(E), _dev(g),
                                          C.c_void_p(_stream_ptr(stream))))
        return E.value, g


class Cloth:
    """A cloth (jgs2_cloth_*): StVK membrane triangles, quadratic bending, Jacobi sweeps."""

    def __init__(self, X, tris, youngs, poisson, thickness, density, bend, pinned=None, gravity=(0, 0, -9.8),
                 dt=1 / 120, planes=None, dhat=1e-3, kappa=1e5):
        self._keep = [np.ascontiguousarray(X, dtype=np.float64), np.ascontiguousarray(tris, dtype=np.int32),
                      None if pinned is None else np.ascontiguousarray(pinned, dtype=np.uint8),
                      np.ascontiguousarray(np.zeros((0, 4)) if planes is None else planes, dtype=np.float64)]
        Xa, Ta, Pa, PLa = self._keep
        d = ClothDesc()
        d.n_vertices, d.n_tris = Xa.shape[0], Ta.shape[0]
        d.rest_pos = _ptr(Xa, C.c_double)
        d.tris = _ptr(Ta, C.c_int32)
        d.youngs, d.poisson, d.thickness = float(youngs), float(poisson), float(thickness)
        d.density, d.bend = float(density), float(bend)
        d.pinned = _ptr(Pa, C.c_uint8) if Pa is not None else C.POINTER(C.c_uint8)()
        for q in range(3):
            d.gravity[q] = float(gravity[q])
        d.dt = float(dt)
        d.n_planes = int(PLa.reshape(-1, 4).shape[0])
        d.planes = _ptr(PLa, C.c_double)
        d.dhat, d.kappa = float(dhat), float(kappa)
        h = C.c_void_p()
        _check(lib().jgs2_cloth_create(C.byref(d), C.byref(h)))
        self.handle = h
        self.V = int(d.n_vertices)

    @classmethod
    def from_scene(cls, s):
        return cls(s.X, s.tris, s.youngs, s.poisson, s.thickness, s.density, s.bend, s.pinned, s.gravity, s.dt,
                   s.planes, s.dhat, s.kappa)

    @property
    def n_hinges(self):
        return int(lib().jgs2_cloth_n_hinges(self.handle))

    def step(self, x, v, opts=None, stream=None):
        """jgs2_cloth_step on float64 CUDA tensors x, v [V,3] (updated in place)."""
        rep = ClothReport()
        st = lib().jgs2_cloth_step(self.handle, _dev(x), _dev(v), C.byref(opts or step_opts()),
                                   C.c_void_p(_stream_ptr(stream)), C.byref(rep))
        _check(st, ok=(0, 5))
        return rep

    def sweeps(self, x_t, v_t, x, n, opts=None, stream=None):
        _check(lib().jgs2_cloth_sweeps(self.handle, _dev(x_t), _dev(v_t), _dev(x), int(n),
                                       C.byref(opts or step_opts()), C.c_void_p(_stream_ptr(stream))))

    def energy_gradient(self, x_t, v_t, x, stream=None):
        import torch
        g = torch.empty_like(x)
        E = C.c_double()
        _check(lib().jgs2_cloth_energy_gradient(self.handle, _dev(x_t), _dev(v_t), _dev(x), C.byref(E), _dev(g),
                                                C.c_void_p(_stream_ptr(stream))))
        return E.value, g

    def close(self):
        if getattr(self, "handle", None):
            lib().jgs2_cloth_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

