"""Thin ctypes binding of ``libfga_gb300.so`` (C ABI in ``include/fga.h``).

Argument marshalling only: every step of the FGA path runs in the library's CUDA kernels.  The
binding takes torch CUDA tensors for device buffers (PyTorch supplies device memory and streams)
and raises ``FGAError`` on any non-OK status.  If the library is not built it raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfga_gb300.so")

(FGA_OK, FGA_ERR_INVALID_ARG, FGA_ERR_OOM, FGA_ERR_CUDA, FGA_ERR_TIMEOUT, FGA_ERR_NUMERIC, FGA_ERR_UNSUPPORTED,
 FGA_ERR_CANCELLED) = range(8)
SERVE_FIFO, SERVE_SHORTEST = 0, 1
PREC_FP32, PREC_FP64 = 0, 1
MEDIUM = {"const": 0, "sine": 1, "grid": 2, "layered": 3}
LAYER_SHAPE = {"planes": 0, "spheres": 1, "undulating": 2}
EXPORTED = ["fga_model_create", "fga_model_destroy", "fga_decompose", "fga_transform", "fga_propagate", "fga_reconstruct",
            "fga_reconstruct_spherical",
            "fga_reconstruct_lattice", "fga_reconstruct_noalloc", "fga_solve", "fga_beams_count", "fga_beams_export",
            "fga_beams_export_all", "fga_beams_destroy", "fga_beams_params", "fga_beams_import", "fga_bin", "fga_profile_enable", "fga_profile_read",
            "fga_solve_vjp", "fga_server_create", "fga_server_submit", "fga_server_wait", "fga_server_stats",
            "fga_server_destroy", "fga_server_cancel", "fga_traveltime_adjoint", "fga_set_device_memory_limit",
            "fga_device_memory_in_use", "fga_point_force_field", "fga_last_error", "fga_version"]
PROFILE_CATEGORIES = ["decompose", "propagate", "binning", "records", "gauss_sum", "gauss_reduce", "gauss_sum_state",
                      "interfaces", "adjoint_forward", "adjoint_reverse", "adjoint_init", "misfit"]


class FGAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fga status {status}: {msg}")
        self.status = status


class ModelDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("cp0", C.c_double), ("cs0", C.c_double), ("amp", C.c_double),
                ("cs_ratio", C.c_double), ("n", C.c_int * 3), ("origin", C.c_double * 3),
                ("spacing", C.c_double * 3), ("nlayers", C.c_int), ("z_interfaces", C.c_void_p),
                ("layer_cp", C.c_void_p), ("layer_cs", C.c_void_p), ("layer_rho", C.c_void_p),
                ("layer_normal", C.c_double * 3), ("layer_shape", C.c_int), ("layer_center", C.c_double * 3),
                ("layer_amp", C.c_double * 8), ("layer_wavelength", C.c_double * 2)]


class InitDesc(C.Structure):
    _fields_ = [("k", C.c_double), ("ny", C.c_int * 3), ("y0", C.c_double * 3), ("dy", C.c_double * 3),
                ("f", C.c_void_p), ("g", C.c_void_p), ("nq", C.c_int), ("q0", C.c_double * 3),
                ("dq", C.c_double * 3), ("np", C.c_int), ("p0", C.c_double * 3), ("dp", C.c_double * 3),
                ("class_mask", C.c_uint), ("precision", C.c_int), ("max_interfaces", C.c_int),
                ("child_rel_min", C.c_double), ("growth", C.c_double), ("psi_rel_min", C.c_double)]


class PointForce(C.Structure):
    _fields_ = [("x0", C.c_double * 3), ("force", C.c_double * 3), ("rho", C.c_double), ("cp", C.c_double),
                ("cs", C.c_double), ("f", C.c_double), ("T0", C.c_double), ("sigma", C.c_double)]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64), ("count", C.c_int64 * 12), ("ms", C.c_double * 12),
                ("beam_steps", C.c_int64), ("pairs_in_window", C.c_int64), ("pairs_tested", C.c_int64)]


class ServerDesc(C.Structure):
    _fields_ = [("n_workers", C.c_int), ("hbm_budget_bytes", C.c_double), ("record_cap_bytes", C.c_double),
                ("policy", C.c_int), ("age_limit_s", C.c_double)]


class RequestInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("worker", C.c_int), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_end", C.c_double), ("bytes", C.c_double), ("beams", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int64), ("running", C.c_int64), ("completed", C.c_int64), ("peak_running", C.c_int64),
                ("inflight_bytes", C.c_double), ("peak_bytes", C.c_double), ("budget_bytes", C.c_double)]


class Lattice(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("axis", C.c_void_p * 3)]


class SolveDesc(C.Structure):
    _fields_ = [("dt", C.c_double), ("nsteps", C.c_int), ("n_times", C.c_int), ("times", C.c_void_p),
                ("n_rx", C.c_int64), ("rx", C.c_void_p), ("n_snap", C.c_int64), ("snap", C.c_void_p),
                ("rw", C.c_double), ("rx_lattice", C.c_void_p), ("snap_lattice", C.c_void_p), ("coords", C.c_int)]


def make_lattice(axes):
    """(ctypes Lattice, kept arrays) from three 1-D coordinate arrays."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in axes]
    L = Lattice()
    L.n[:] = [a.size for a in arrs]
    for d in range(3):
        L.axis[d] = arrs[d].ctypes.data
    return L, arrs


_lib = None


def lib(path: Optional[str] = None) -> C.CDLL:
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise FGAError(FGA_ERR_UNSUPPORTED, f"{p} not built; run paper_1810_06760_gb300.build.build()")
    L = C.CDLL(p)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    L.fga_model_create.argtypes = [C.POINTER(vp), C.POINTER(ModelDesc), vp, vp, vp]
    L.fga_model_destroy.argtypes = [vp]
    L.fga_decompose.argtypes = [vp, C.POINTER(InitDesc), C.POINTER(vp), vp]
    L.fga_transform.argtypes = [C.POINTER(InitDesc), vp, vp]
    L.fga_point_force_field.argtypes = [C.POINTER(PointForce), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.c_double, vp, vp, vp]
    L.fga_propagate.argtypes = [vp, vp, C.c_double, i32, vp]
    L.fga_reconstruct.argtypes = [vp, vp, i64, C.c_double, vp, vp]
    L.fga_reconstruct_noalloc.argtypes = [vp, vp, i64, C.c_double, vp, vp]
    L.fga_reconstruct_spherical.argtypes = [vp, vp, i64, C.c_double, vp, vp]
    L.fga_reconstruct_lattice.argtypes = [vp, C.POINTER(Lattice), C.c_double, vp, vp]
    L.fga_solve.argtypes = [vp, C.POINTER(InitDesc), C.POINTER(SolveDesc), vp, vp, vp]
    L.fga_solve_vjp.argtypes = [vp, C.POINTER(InitDesc), C.POINTER(SolveDesc), vp, vp, vp, i32, vp]
    L.fga_server_create.argtypes = [C.POINTER(vp), vp, C.POINTER(ServerDesc)]
    L.fga_server_submit.argtypes = [vp, C.POINTER(InitDesc), C.POINTER(SolveDesc), vp, vp, C.POINTER(i64)]
    L.fga_server_wait.argtypes = [vp, i64, C.c_double, C.POINTER(RequestInfo)]
    L.fga_server_stats.argtypes = [vp, C.POINTER(ServerStats)]
    L.fga_server_destroy.argtypes = [vp]
    L.fga_server_cancel.argtypes = [vp, i64]
    L.fga_set_device_memory_limit.argtypes = [C.c_double]
    L.fga_device_memory_in_use.argtypes = []
    L.fga_beams_count.argtypes = [vp, vp]
    L.fga_beams_export.argtypes = [vp, vp, vp]
    L.fga_beams_export_all.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
    L.fga_beams_destroy.argtypes = [vp]
    L.fga_beams_params.argtypes = [vp, vp, vp, vp]
    L.fga_beams_import.argtypes = [i64, vp, vp, C.c_double, C.c_double, i32, vp, vp]
    L.fga_bin.argtypes = [vp, i64, vp, C.c_float, vp, vp, vp, vp, vp]
    L.fga_traveltime_adjoint.argtypes = [vp, vp, i32, i64, i64, C.c_double, i32, vp, vp, vp, vp]
    L.fga_profile_enable.argtypes = [i32]
    L.fga_profile_read.argtypes = [C.POINTER(Profile), i32]
    L.fga_last_error.argtypes = [C.c_char_p, C.c_size_t]
    L.fga_last_error.restype = None
    L.fga_version.restype = C.c_int
    L.fga_device_memory_in_use.restype = C.c_double
    for name in EXPORTED:
        if name not in ("fga_last_error", "fga_version", "fga_device_memory_in_use"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    lib().fga_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(status: int) -> None:
    if status != FGA_OK:
        raise FGAError(status, last_error())


def _stream(stream) -> C.c_void_p:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dptr(t) -> Optional[int]:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return t.data_ptr()


def _arr3(v) -> C.Array:
    a = (C.c_double * 3)()
    a[:] = [float(x) for x in np.asarray(v, dtype=np.float64).reshape(3)]
    return a


class Model:
    """Handle of a velocity model (fga_model_create / fga_model_destroy)."""

    def __init__(self, kind: str, *, cp0=2.0, cs0=1.0, amp=0.0, cs_ratio=1.0 / math.sqrt(3.0),
                 grid_p=None, grid_s=None, origin=(0, 0, 0), spacing=(1, 1, 1),
                 z_interfaces=(), layer_cp=(), layer_cs=(), layer_rho=(), layer_normal=(0.0, 0.0, 0.0),
                 layer_shape="planes", layer_center=(0.0, 0.0, 0.0), layer_amp=(), layer_wavelength=(1.0, 1.0),
                 stream=None):
        d = ModelDesc()
        d.kind = MEDIUM[kind]
        d.cp0, d.cs0, d.amp, d.cs_ratio = cp0, cs0, amp, cs_ratio
        self._keep = []
        gp = gs = None
        if kind == "grid":
            gp, gs = grid_p.contiguous(), grid_s.contiguous()
            d.n[:] = list(gp.shape[:3])
            d.origin[:] = [float(v) for v in origin]
            d.spacing[:] = [float(v) for v in spacing]
        if kind == "layered":
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (z_interfaces, layer_cp, layer_cs, layer_rho)]
            self._keep += arrs
            d.nlayers = arrs[1].size
            d.z_interfaces, d.layer_cp, d.layer_cs, d.layer_rho = [a.ctypes.data for a in arrs]
            d.layer_normal[:] = [float(v) for v in layer_normal]
            d.layer_shape = LAYER_SHAPE[layer_shape]
            d.layer_center[:] = [float(v) for v in layer_center]
            amp = [float(v) for v in layer_amp]
            d.layer_amp[:] = amp + [0.0] * (8 - len(amp))
            d.layer_wavelength[:] = [float(v) for v in layer_wavelength]
        h = C.c_void_p()
        _check(lib().fga_model_create(C.byref(h), C.byref(d), _dptr(gp), _dptr(gs), _stream(stream)))
        self.grid_shape = tuple(gp.shape[:3]) if gp is not None else None
        self.h = h
        self.kind = kind

    def close(self):
        if getattr(self, "h", None):
            lib().fga_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def model_from_medium(med, device="cuda") -> Model:
    """Model from a ``workloads.Medium``."""
    import torch
    if med.kind == "layered":
        return Model("layered", z_interfaces=med.z_interfaces, layer_cp=med.layer_cp, layer_cs=med.layer_cs,
                     layer_rho=med.layer_rho, layer_normal=med.layer_normal, layer_shape=med.layer_shape,
                     layer_center=med.layer_center, layer_amp=med.layer_amp,
                     layer_wavelength=med.layer_wavelength)
    if med.kind == "grid":
        gp = torch.as_tensor(med.grid_p, device=device)
        gs = torch.as_tensor(med.grid_s, device=device)
        m = Model("grid", grid_p=gp, grid_s=gs, origin=med.origin, spacing=med.spacing)
        torch.cuda.current_stream().synchronize()
        return m
    return Model(med.kind, cp0=med.cp0, cs0=med.cs0, amp=med.amp, cs_ratio=med.cs_ratio)


def init_desc(k, f, g, y0, dy, mesh, classes: Sequence[int], precision: int, psi_rel_min: float = 0.0) -> InitDesc:
    """Decomposition descriptor.  f, g: complex128 CUDA tensors [ny0, ny1, ny2, 3] (g may be None).
    psi_rel_min > 0 creates only the beams with |psi| > psi_rel_min max|psi|."""
    d = InitDesc()
    d.k = float(k)
    d.ny[:] = list(f.shape[:3])
    d.y0, d.dy = _arr3(y0), _arr3(dy)
    d.f, d.g = _dptr(f), _dptr(g)
    d.nq, d.q0, d.dq = int(mesh.nq), _arr3(mesh.q0), _arr3(mesh.dq)
    d.np, d.p0, d.dp = int(mesh.np_), _arr3(mesh.p0), _arr3(mesh.dp)
    d.class_mask = sum(1 << int(c) for c in classes)
    d.precision = int(precision)
    d.psi_rel_min = float(psi_rel_min)
    return d


def set_layered_options(desc: InitDesc, max_interfaces: int = 0, child_rel_min: float = 0.0, growth: float = 0.0):
    desc.max_interfaces, desc.child_rel_min, desc.growth = int(max_interfaces), float(child_rel_min), float(growth)
    return desc


class Beams:
    """Handle of a beam set (fga_decompose ... fga_beams_destroy)."""

    def __init__(self, h: C.c_void_p, precision: int, k: float):
        self.h, self.precision, self.k = h, precision, k

    def count(self):
        out = np.zeros(4, dtype=np.int64)
        _check(lib().fga_beams_count(self.h, out.ctypes.data))
        return out

    def export(self):
        """(state [nb, 48] float64, meta [nb] int32) in mesh order per class (synchronous)."""
        n = int(self.count().sum())
        st = np.zeros((n, 48))
        meta = np.zeros(n, dtype=np.int32)
        _check(lib().fga_beams_export(self.h, st.ctypes.data, meta.ctypes.data))
        return st, meta

    def export_all(self):
        """Live beams in storage order: (state [n,48], meta [n], mesh_id [n], path [n], dropped)."""
        n = C.c_int64()
        dropped = C.c_int64()
        _check(lib().fga_beams_export_all(self.h, 0, C.byref(n), C.byref(dropped), None, None, None, None))
        cnt = n.value
        st = np.zeros((cnt, 48))
        meta = np.zeros(cnt, dtype=np.int32)
        mid = np.zeros(cnt, dtype=np.int64)
        path = np.zeros(cnt, dtype=np.int64)
        _check(lib().fga_beams_export_all(self.h, cnt, C.byref(n), C.byref(dropped), st.ctypes.data, meta.ctypes.data,
                                          mid.ctypes.data, path.ctypes.data))
        return st, meta, mid, path, dropped.value

    def close(self):
        if getattr(self, "h", None):
            lib().fga_beams_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def beams_params(beams: Beams):
    """(k, w, precision) of a beam set: its FGA parameter, quadrature weight and precision."""
    k, w, prec = C.c_double(), C.c_double(), C.c_int()
    _check(lib().fga_beams_params(beams.h, C.byref(k), C.byref(w), C.byref(prec)))
    return k.value, w.value, prec.value


def beams_import(state, meta, k: float, w: float, precision: int, stream=None) -> Beams:
    """fga_beams_import: a beam set from exported states (HOST float64 [n, 48]) and meta (int32 [n], class and
    S-frame bits), with the k, w and precision of the set they came from."""
    state = np.ascontiguousarray(state, dtype=np.float64)
    meta = np.ascontiguousarray(meta, dtype=np.int32)
    assert state.ndim == 2 and state.shape[1] == 48 and meta.shape == (state.shape[0],)
    h = C.c_void_p()
    _check(lib().fga_beams_import(state.shape[0], state.ctypes.data, meta.ctypes.data, float(k), float(w),
                                  int(precision), C.byref(h), _stream(stream)))
    return Beams(h, int(precision), float(k))


def decompose(model: Model, desc: InitDesc, stream=None) -> Beams:
    h = C.c_void_p()
    _check(lib().fga_decompose(model.h, C.byref(desc), C.byref(h), _stream(stream)))
    return Beams(h, desc.precision, desc.k)


def transform(desc: InitDesc, out=None, stream=None):
    """fga_transform: the wave-packet transform F(q,p) of desc's f on its mesh (Eq. psi), complex
    [A, A, A, 3] (A = nq np; entry (a0, a1, a2), a_d = iq_d np + jp_d) in desc's precision."""
    import torch
    A = desc.nq * desc.np
    if out is None:
        out = torch.empty((A, A, A, 3), dtype=_cdtype(desc.precision),
                          device=torch.device("cuda", torch.cuda.current_device()))
    _check(lib().fga_transform(C.byref(desc), _dptr(out), _stream(stream)))
    return out


def point_force(x0, force, rho, cp, cs, f, T0, sigma) -> PointForce:
    """Point force `force` s(t) at x0 in a homogeneous medium, s(t) = cos(2 pi f (t+T0)) exp(-(t+T0)^2/sigma^2)."""
    p = PointForce()
    p.x0, p.force = _arr3(x0), _arr3(force)
    p.rho, p.cp, p.cs, p.f, p.T0, p.sigma = float(rho), float(cp), float(cs), float(f), float(T0), float(sigma)
    return p


def point_force_field(src: PointForce, ny, y0, dy, t: float, velocity: bool = True, stream=None):
    """fga_point_force_field: (u, du/dt) of the point force at time t on the grid y0 + i dy, complex128
    CUDA tensors [ny0, ny1, ny2, 3] (v is None when velocity is False)."""
    import torch
    n = [int(v) for v in np.broadcast_to(np.asarray(ny), (3,))]
    dev = torch.device("cuda", torch.cuda.current_device())
    u = torch.empty(tuple(n) + (3,), dtype=torch.complex128, device=dev)
    v = torch.empty_like(u) if velocity else None
    nyc = (C.c_int * 3)(*n)
    _check(lib().fga_point_force_field(C.byref(src), nyc, _arr3(y0), _arr3(dy), float(t), _dptr(u), _dptr(v),
                                       _stream(stream)))
    return u, v


def propagate(model: Model, beams: Beams, dt: float, nsteps: int, stream=None) -> None:
    _check(lib().fga_propagate(model.h, beams.h, float(dt), int(nsteps), _stream(stream)))


def _cdtype(precision: int):
    import torch
    return torch.complex128 if precision == PREC_FP64 else torch.complex64


def reconstruct(beams: Beams, x, rw: float = 0.0, out=None, stream=None):
    """u(x) at the current beam state; x: float64 CUDA tensor [n, 3].  Returns complex [n, 3]."""
    import torch
    n = x.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=_cdtype(beams.precision), device=x.device)
    _check(lib().fga_reconstruct(beams.h, _dptr(x) if n else None, n, float(rw), _dptr(out) if n else None,
                                 _stream(stream)))
    return out


def reconstruct_spherical(beams: Beams, rtp, rw: float = 0.0, out=None, stream=None):
    """u at points given as (r, theta, phi) (float64 CUDA tensor [n, 3]; theta longitude, phi latitude):
    the sum of Eq. FGA at x = (r cos theta cos phi, r sin theta cos phi, r sin phi).  Returns complex [n, 3]."""
    import torch
    n = rtp.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=_cdtype(beams.precision), device=rtp.device)
    _check(lib().fga_reconstruct_spherical(beams.h, _dptr(rtp) if n else None, n, float(rw), _dptr(out) if n else None,
                                           _stream(stream)))
    return out


def reconstruct_lattice(beams: Beams, axes, rw: float = 0.0, out=None, stream=None):
    """u at the lattice points (axes[0][i], axes[1][j], axes[2][l]); returns complex [n0, n1, n2, 3]."""
    import torch
    L, keep = make_lattice(axes)
    shape = tuple(int(a.size) for a in keep)
    if out is None:
        out = torch.empty(shape + (3,), dtype=_cdtype(beams.precision), device=torch.device("cuda", torch.cuda.current_device()))
    _check(lib().fga_reconstruct_lattice(beams.h, C.byref(L), float(rw), _dptr(out), _stream(stream)))
    return out


def reconstruct_noalloc(beams: Beams, x, out, rw: float = 0.0, stream=None):
    """fga_reconstruct_noalloc: the same sum as ``reconstruct`` without any device allocation inside
    the library (fixed internal scratch; at most 4096 points per call).  The caller supplies ``out``
    (complex [n, 3] in the beams' precision) as well as ``x``."""
    n = x.shape[0]
    _check(lib().fga_reconstruct_noalloc(beams.h, _dptr(x) if n else None, n, float(rw), _dptr(out) if n else None,
                                         _stream(stream)))
    return out


def solve(model: Model, desc: InitDesc, dt: float, nsteps: int, times, rx=None, snap=None, rw: float = 0.0,
          seis_out=None, snap_out=None, stream=None, rx_axes=None, snap_axes=None, spherical: bool = False):
    """Whole forward solve.  Receivers: points rx [n_rx, 3] (CUDA float64) or a lattice rx_axes (three
    1-D arrays); snapshot likewise (snap or snap_axes).  Returns (seismograms [n_times, n_rx, 3] or
    [n_times, n0, n1, n2, 3], snapshot [n_snap, 3] or [n0, n1, n2, 3]); None where not requested.
    spherical: the point arrays hold (r, theta, phi) (fga_solve_desc.coords = FGA_COORDS_SPHERICAL)."""
    import torch
    times = np.ascontiguousarray(times, dtype=np.float64)
    sd = SolveDesc()
    sd.coords = 1 if spherical else 0
    sd.dt, sd.nsteps = float(dt), int(nsteps)
    sd.n_times, sd.times = times.size, times.ctypes.data if times.size else None
    dev = torch.device("cuda", torch.cuda.current_device())
    cdt = _cdtype(desc.precision)
    keep = []
    if rx_axes is not None:
        Lr, ka = make_lattice(rx_axes)
        keep += [Lr, ka]
        sd.rx_lattice = C.cast(C.pointer(Lr), C.c_void_p)
        rshape = tuple(a.size for a in ka)
        if times.size and seis_out is None:
            seis_out = torch.empty((times.size,) + rshape + (3,), dtype=cdt, device=dev)
        nrx = 0
    else:
        nrx = 0 if rx is None else rx.shape[0]
        if nrx and times.size and seis_out is None:
            seis_out = torch.empty((times.size, nrx, 3), dtype=cdt, device=dev)
    if snap_axes is not None:
        Ls, ks = make_lattice(snap_axes)
        keep += [Ls, ks]
        sd.snap_lattice = C.cast(C.pointer(Ls), C.c_void_p)
        if snap_out is None:
            snap_out = torch.empty(tuple(a.size for a in ks) + (3,), dtype=cdt, device=dev)
        nsn = 0
    else:
        nsn = 0 if snap is None else snap.shape[0]
        if nsn and snap_out is None:
            snap_out = torch.empty((nsn, 3), dtype=cdt, device=dev)
    sd.n_rx, sd.rx = nrx, _dptr(rx) if nrx else None
    sd.n_snap, sd.snap = nsn, _dptr(snap) if nsn else None
    sd.rw = float(rw)
    _check(lib().fga_solve(model.h, C.byref(desc), C.byref(sd), _dptr(seis_out), _dptr(snap_out),
                           _stream(stream)))
    return seis_out, snap_out


def solve_vjp(model: Model, desc: InitDesc, dt: float, nsteps: int, times, rx, ubar, grad_p=None, grad_s=None,
              rw: float = 0.0, checkpoint_every: int = 20, stream=None):
    """Reverse mode of the seismograms of `solve` (receivers as points rx [n_rx, 3], CUDA float64) with
    respect to the model's node fields.  ubar: CUDA complex [n_times, n_rx, 3] in the init precision
    (dL/dRe u + i dL/dIm u).  Adds into grad_p / grad_s (CUDA float64 [n0, n1, n2, 10], created zeroed
    when None; None is returned for both with a constant medium) and returns them."""
    import torch
    times = np.ascontiguousarray(times, dtype=np.float64)
    sd = SolveDesc()
    sd.dt, sd.nsteps = float(dt), int(nsteps)
    sd.n_times, sd.times = times.size, times.ctypes.data
    sd.n_rx, sd.rx = rx.shape[0], _dptr(rx)
    sd.rw = float(rw)
    ub = ubar.contiguous()
    assert ub.dtype == _cdtype(desc.precision) and tuple(ub.shape) == (times.size, rx.shape[0], 3)
    if model.kind == "grid":
        shape = tuple(model.grid_shape) + (10,)
        dev = ub.device
        if grad_p is None:
            grad_p = torch.zeros(shape, dtype=torch.float64, device=dev)
        if grad_s is None:
            grad_s = torch.zeros(shape, dtype=torch.float64, device=dev)
        assert grad_p.dtype == torch.float64 and grad_p.is_contiguous() and tuple(grad_p.shape) == shape
        assert grad_s.dtype == torch.float64 and grad_s.is_contiguous() and tuple(grad_s.shape) == shape
    _check(lib().fga_solve_vjp(model.h, C.byref(desc), C.byref(sd), _dptr(ub), _dptr(grad_p), _dptr(grad_s),
                               int(checkpoint_every), _stream(stream)))
    return grad_p, grad_s


def traveltime_adjoint(syn, obs, dt: float, max_lag: int, stream=None):
    """Cross-correlation delays of obs relative to syn (CUDA complex [n_t, n_rx, 3], both complex64 or
    both complex128), the misfit 1/2 sum tau^2 and its seismogram cotangent (the adjoint source for
    solve_vjp).  Returns (tau CUDA float64 [n_rx], ubar like syn, misfit CUDA float64 [1])."""
    import torch
    s, o = syn.contiguous(), obs.contiguous()
    assert s.dtype == o.dtype and s.shape == o.shape and s.dim() == 3 and s.shape[2] == 3
    assert s.dtype in (torch.complex64, torch.complex128)
    prec = PREC_FP32 if s.dtype == torch.complex64 else PREC_FP64
    n_t, n_rx = int(s.shape[0]), int(s.shape[1])
    tau = torch.empty(n_rx, dtype=torch.float64, device=s.device)
    ubar = torch.empty_like(s)
    misfit = torch.empty(1, dtype=torch.float64, device=s.device)
    _check(lib().fga_traveltime_adjoint(_dptr(s), _dptr(o), prec, n_t, n_rx, float(dt), int(max_lag), _dptr(tau),
                                        _dptr(ubar), _dptr(misfit), _stream(stream)))
    return tau, ubar, misfit


class Server:
    """Serving loop (fga_server_*): forward solves of independent requests on one resident model.
    submit() returns a request id; wait(id) blocks until it is done and returns its timing record
    (seconds since the server started).  Tensors a request uses are kept alive until it is waited."""

    def __init__(self, model: Model, n_workers: int = 4, hbm_budget_bytes: float = 0.0,
                 record_cap_bytes: float = 0.0, policy: int = SERVE_FIFO, age_limit_s: float = 0.0):
        d = ServerDesc(int(n_workers), float(hbm_budget_bytes), float(record_cap_bytes), int(policy),
                       float(age_limit_s))
        h = C.c_void_p()
        _check(lib().fga_server_create(C.byref(h), model.h, C.byref(d)))
        self.h, self.model, self._keep = h, model, {}

    def submit(self, desc: InitDesc, dt: float, nsteps: int, times, rx=None, rw: float = 0.0, keep=(),
               rx_axes=None):
        """Queue a forward solve; receivers as points rx [n_rx, 3] (CUDA float64) or a lattice rx_axes
        (three 1-D arrays).  Returns the request id."""
        import torch
        times = np.ascontiguousarray(times, dtype=np.float64)
        sd = SolveDesc()
        sd.dt, sd.nsteps = float(dt), int(nsteps)
        sd.n_times, sd.times = times.size, times.ctypes.data if times.size else None
        sd.rw = float(rw)
        extra = ()
        dev = torch.device("cuda", torch.cuda.current_device())
        if rx_axes is not None:
            Lr, ka = make_lattice(rx_axes)
            sd.rx_lattice = C.cast(C.pointer(Lr), C.c_void_p)
            shape = (times.size,) + tuple(a.size for a in ka) + (3,)
            extra = (Lr, ka)
        else:
            sd.n_rx, sd.rx = rx.shape[0], _dptr(rx)
            shape = (times.size, rx.shape[0], 3)
            dev = rx.device
        out = torch.empty(shape, dtype=_cdtype(desc.precision), device=dev)
        rid = C.c_int64()
        _check(lib().fga_server_submit(self.h, C.byref(desc), C.byref(sd), _dptr(out), None, C.byref(rid)))
        self._keep[rid.value] = (desc, times, rx, out, keep, extra)
        return rid.value

    def wait(self, rid: int, timeout: float = 0.0):
        """(seismograms, info dict); raises FGAError with the request's own status on failure."""
        info = RequestInfo()
        st = lib().fga_server_wait(self.h, int(rid), float(timeout), C.byref(info))
        if st == FGA_ERR_TIMEOUT:       # still queued or running: its buffers stay referenced
            raise FGAError(st, last_error())
        kept = self._keep.pop(rid, None)
        if st != 0:
            raise FGAError(st, last_error())
        return kept[3], {"worker": info.worker, "t_submit": info.t_submit, "t_start": info.t_start,
                         "t_end": info.t_end, "bytes": info.bytes, "beams": info.beams}

    def cancel(self, rid: int) -> None:
        """fga_server_cancel: drop a queued request, stop a running one at its next window of steps."""
        _check(lib().fga_server_cancel(self.h, int(rid)))

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().fga_server_stats(self.h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().fga_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_device_memory_limit(nbytes: float) -> None:
    """fga_set_device_memory_limit: bound on the library's own device allocations (<= 0: none)."""
    _check(lib().fga_set_device_memory_limit(float(nbytes)))


def device_memory_in_use() -> float:
    return float(lib().fga_device_memory_in_use())


def profile_enable(mode: int) -> None:
    """0 off, 1 counters incl. in-window pairs, 2 counters + per-kernel CUDA-event device times, 3 both."""
    _check(lib().fga_profile_enable(int(mode)))


def profile_read(reset: bool = True) -> dict:
    p = Profile()
    _check(lib().fga_profile_read(C.byref(p), int(bool(reset))))
    return {"launches": p.launches,
            "count": {n: p.count[i] for i, n in enumerate(PROFILE_CATEGORIES)},
            "ms": {n: p.ms[i] for i, n in enumerate(PROFILE_CATEGORIES)},
            "beam_steps": p.beam_steps, "pairs_in_window": p.pairs_in_window, "pairs_tested": p.pairs_tested}


def bin_centres(Q, origin, inv_h: float, nc, stream=None):
    """Cell keys, stable permutation and cell offsets of FP32 centres Q [n, 3] (CUDA float32)."""
    import torch
    n = Q.shape[0]
    nc = np.ascontiguousarray(nc, dtype=np.int32)
    o = np.ascontiguousarray(origin, dtype=np.float32)
    keys = torch.empty(max(n, 1), dtype=torch.int32, device=Q.device)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=Q.device)
    start = torch.empty(int(np.prod(nc)) + 1, dtype=torch.int32, device=Q.device)
    _check(lib().fga_bin(_dptr(Q) if n else None, n, o.ctypes.data, C.c_float(np.float32(inv_h)), nc.ctypes.data,
                         _dptr(keys), _dptr(perm), _dptr(start), _stream(stream)))
    return keys[:n], perm[:n], start
