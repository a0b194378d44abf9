"""Python side of the FP64 CPU oracle for the frozen Gaussian approximation (FGA).

THIS MODULE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It shares no code
with the CUDA library (``paper_1810_06760_gb300``) and never imports it.

It compiles ``fga_oracle.c`` with gcc on first use (into ``oracle/_build/``) and drives it
through ctypes.  Everything is FP64.  The three steps follow the paper's algorithm
(Fig. ``fig:FGA_alg``): decompose the initial data into Gaussian packets (Eqs. psi, alpha^k),
propagate every packet with RK4 (Eqs. char_plus, char_minus, amp_P, amp_SV, amp_SH, DzDt),
and sum the packets (Eq. FGA).

Parity status: every routine here is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, brute force or an independent formulation; see the test docstrings.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fga_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libfga_oracle.so")
_lock = threading.Lock()
_lib = None

CLS_PP, CLS_PM, CLS_SP, CLS_SM = 0, 1, 2, 3
META_REF_E1 = 4
META_VECTOR = 8


def meta_layer(mt):
    return (np.asarray(mt) >> 4) & 15


def meta_gen(mt):
    return (np.asarray(mt) >> 8) & 15


def meta_root(mt):
    """Class of the initial beam a layered-medium beam descends from."""
    return (np.asarray(mt) >> 13) & 3

STATE_DOUBLES = 48


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, FP64, OpenMP over independent beams)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (beams and points are independent)."""
    lib()
    gomp = C.CDLL("libgomp.so.1")
    gomp.omp_set_num_threads(int(n))


def get_threads() -> int:
    lib()
    gomp = C.CDLL("libgomp.so.1")
    gomp.omp_get_max_threads.restype = C.c_int
    return int(gomp.omp_get_max_threads())


class _Model(C.Structure):
    _fields_ = [
        ("kind", C.c_int),
        ("cp0", C.c_double), ("cs0", C.c_double),
        ("amp", C.c_double), ("cs_ratio", C.c_double),
        ("n", C.c_int * 3), ("o", C.c_double * 3), ("h", C.c_double * 3),
        ("gp", C.c_void_p), ("gs", C.c_void_p),
        ("nlay", C.c_int),
        ("zif", C.c_void_p), ("lcp", C.c_void_p), ("lcs", C.c_void_p), ("lrho", C.c_void_p),
        ("shells", C.c_int), ("ctr", C.c_double * 3),
        ("undul", C.c_int), ("uk", C.c_double * 2), ("uamp", C.c_void_p),
    ]


_P = C.c_void_p


def _declare(L):
    L.orc_model_eval_many.argtypes = [_P, C.c_int, C.c_int, _P, _P]
    L.orc_fbi_direct.argtypes = [_P, _P, _P, _P, C.c_double, C.c_int, _P, _P, C.c_int, _P, _P, _P]
    L.orc_fbi_separable.argtypes = L.orc_fbi_direct.argtypes
    L.orc_beam_init.argtypes = [_P, C.c_double, C.c_int, _P, _P, C.c_int, _P, _P, _P, _P,
                                C.c_int, C.c_int, _P, _P]
    L.orc_rhs_many.argtypes = [_P, C.c_int, _P, _P, _P]
    L.orc_propagate.argtypes = [_P, C.c_int, _P, _P, C.c_double, C.c_int, C.c_int, _P, _P,
                                C.c_double, _P]
    L.orc_records.argtypes = [C.c_int, _P, _P, C.c_double, _P]
    L.orc_gauss_sum.argtypes = [C.c_int, _P, C.c_double, C.c_double, C.c_int, _P, _P]
    L.orc_bin_keys_f32.argtypes = [C.c_int, _P, _P, C.c_float, _P, _P]
    L.orc_bin_sort.argtypes = [C.c_int, _P, C.c_int, _P, _P]
    L.orc_s_ref_e1.argtypes = [_P]
    L.orc_s_ref_e1.restype = C.c_int
    L.orc_interface_event.argtypes = [_P, C.c_int, _P, C.c_int, C.c_double, _P, _P]
    L.orc_interface_event.restype = C.c_int
    L.orc_layered_step.argtypes = [_P, C.c_int, _P, _P, _P, C.c_double, C.c_int, C.c_double, C.c_int, _P, _P, _P, _P]
    L.orc_layered_step.restype = C.c_int
    L.orc_rk4_many.argtypes = [_P, C.c_int, _P, _P, C.c_double, _P]
    L.orc_rhs_vjp.argtypes = [_P, C.c_int, _P, _P, _P, _P, _P]
    L.orc_solve_vjp.argtypes = [_P, C.c_int, _P, _P, C.c_double, C.c_int, C.c_int, _P, _P, C.c_double,
                                C.c_double, C.c_double, C.c_int, _P, _P, _P, _P, _P]
    L.orc_solve_vjp.restype = C.c_int
    L.orc_beam_init_vjp.argtypes = [_P, C.c_double, C.c_int, _P, _P, C.c_int, _P, _P, _P, _P, C.c_int, _P, _P, _P]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _d3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))


class Model:
    """Velocity model for the oracle.  kinds: 'const', 'sine', 'grid', 'layered'.  Layered media have
    flat interfaces at the depths z_interfaces (x3, increasing) or, with layer_shape='spheres', spherical
    ones |x - layer_center| = z_interfaces[i] (radii, decreasing; layer 0 outside the largest)."""

    def __init__(self, kind: str, *, cp0=2.0, cs0=1.0, amp=0.0, cs_ratio=1.0 / math.sqrt(3.0),
                 grid_p=None, grid_s=None, origin=(0, 0, 0), spacing=(1, 1, 1),
                 z_interfaces=(), layer_cp=(), layer_cs=(), layer_rho=(), layer_shape="planes",
                 layer_center=(0.0, 0.0, 0.0), layer_amp=(), layer_wavelength=(1.0, 1.0)):
        s = _Model()
        self._keep = []
        s.kind = {"const": 0, "sine": 1, "grid": 2, "layered": 3}[kind]
        s.cp0, s.cs0, s.amp, s.cs_ratio = cp0, cs0, amp, cs_ratio
        if kind == "grid":
            gp = np.ascontiguousarray(grid_p, dtype=np.float32)
            gs = np.ascontiguousarray(grid_s, dtype=np.float32)
            assert gp.ndim == 4 and gp.shape[3] == 10 and gs.shape == gp.shape
            self._keep += [gp, gs]
            s.n[:] = gp.shape[:3]
            s.o[:] = [float(v) for v in origin]
            s.h[:] = [float(v) for v in spacing]
            s.gp, s.gs = gp.ctypes.data, gs.ctypes.data
        if kind == "layered":
            zi = np.ascontiguousarray(z_interfaces, dtype=np.float64)
            lc = np.ascontiguousarray(layer_cp, dtype=np.float64)
            ls = np.ascontiguousarray(layer_cs, dtype=np.float64)
            lr = np.ascontiguousarray(layer_rho, dtype=np.float64)
            assert lc.size == zi.size + 1 == ls.size == lr.size
            self._keep += [zi, lc, ls, lr]
            s.nlay = lc.size
            s.zif, s.lcp, s.lcs, s.lrho = zi.ctypes.data, lc.ctypes.data, ls.ctypes.data, lr.ctypes.data
            assert layer_shape in ("planes", "spheres", "undulating")
            s.shells = int(layer_shape == "spheres")
            s.ctr[:] = [float(v) for v in layer_center]
            self.radii = zi.copy() if s.shells else None
            self.center = np.array(s.ctr[:], dtype=np.float64)
            s.undul = int(layer_shape == "undulating")
            ua = np.zeros(max(zi.size, 1))
            ua[:len(layer_amp)] = [float(v) for v in layer_amp]
            self._keep.append(ua)
            s.uamp = ua.ctypes.data
            s.uk[:] = [2.0 * math.pi / float(v) for v in layer_wavelength]
            self.z_interfaces, self.amp = zi.copy(), ua[:zi.size].copy()
            self.k_und = np.array(s.uk[:], dtype=np.float64)
        self.s = s
        self.kind = kind

    @property
    def ptr(self):
        return C.cast(C.pointer(self.s), C.c_void_p)

    def eval(self, wave: int, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        out = np.zeros((x.shape[0], 10))
        lib().orc_model_eval_many(self.ptr, int(wave), x.shape[0], _ptr(x), _ptr(out))
        return out


class Mesh:
    """Tensor (q, p) mesh: q_{d,i} = q0[d] + i dq[d] (nq per axis), p_{d,j} = p0[d] + j dp[d]."""

    def __init__(self, nq, q0, dq, np_, p0, dp):
        self.nq, self.np = int(nq), int(np_)
        self.q0, self.dq, self.p0, self.dp = _d3(q0), _d3(dq), _d3(p0), _d3(dp)

    @property
    def M(self):
        return self.nq ** 3 * self.np ** 3

    def weight(self, k: float) -> float:
        """delta q delta p / (2 pi / k)^{9/2}, the quadrature weight of Eq. FGA."""
        return float(np.prod(self.dq) * np.prod(self.dp) / (2.0 * math.pi / k) ** 4.5)

    def points(self):
        """(q, p) of every mesh point, mesh order (q-major, p-minor)."""
        iq = np.arange(self.nq)
        ip = np.arange(self.np)
        Q = np.stack(np.meshgrid(iq, iq, iq, indexing="ij"), -1).reshape(-1, 3) * self.dq + self.q0
        P = np.stack(np.meshgrid(ip, ip, ip, indexing="ij"), -1).reshape(-1, 3) * self.dp + self.p0
        q = np.repeat(Q, P.shape[0], axis=0)
        p = np.tile(P, (Q.shape[0], 1))
        return q, p


def fbi(f: np.ndarray, y0, dy, k: float, mesh: Mesh, method: str = "separable") -> np.ndarray:
    """Wave-packet transform F(q,p) = sum_y f(y) exp(-ik p.(y-q) - k|y-q|^2/2) dy^3 (Eq. psi).

    f: complex [ny0, ny1, ny2, 3] sampled at y0 + i*dy.  Returns complex [M, 3] in mesh order."""
    f = np.ascontiguousarray(f, dtype=np.complex128)
    ny = np.ascontiguousarray(f.shape[:3], dtype=np.int32)
    F = np.zeros((mesh.M, 3), dtype=np.complex128)
    fn = lib().orc_fbi_separable if method == "separable" else lib().orc_fbi_direct
    fn(_ptr(ny), _ptr(_d3(y0)), _ptr(_d3(dy)), _ptr(f), float(k), mesh.nq, _ptr(mesh.q0), _ptr(mesh.dq),
       mesh.np, _ptr(mesh.p0), _ptr(mesh.dp), _ptr(F))
    return F


def beam_init(model: Model, k: float, mesh: Mesh, F: np.ndarray, G, cls: int, vector_form: bool = False):
    """Beams of one class (0 P+, 1 P-, 2 S+, 3 S-) at t = 0.  Returns (state [M,48], meta [M])."""
    F = np.ascontiguousarray(F, dtype=np.complex128)
    Gp = None
    if G is not None:
        G = np.ascontiguousarray(G, dtype=np.complex128)
        Gp = _ptr(G)
    st = np.zeros((mesh.M, STATE_DOUBLES))
    meta = np.zeros(mesh.M, dtype=np.int32)
    lib().orc_beam_init(model.ptr, float(k), mesh.nq, _ptr(mesh.q0), _ptr(mesh.dq), mesh.np, _ptr(mesh.p0),
                        _ptr(mesh.dp), _ptr(F), Gp, int(cls), int(bool(vector_form)), _ptr(st), _ptr(meta))
    return st, meta


def psi_select(groups, eps: float):
    """Beam selection of step 1 of Fig. fig:FGA_alg (the algorithm decomposes into the sets of packets
    worth propagating): of the beams of every class, given as [(state, meta)] from beam_init, keep those
    whose |psi| exceeds eps times the largest |psi| over all of them.  |psi| is the norm of the beam's
    psi vector: the initial amplitudes are 2^{3/2} psi (one complex value for P, SV and SH for S), so
    the ratio is taken on the amplitudes.  Survivors keep their order.  eps = 0 keeps every beam.
    Returns [(state, meta, mesh_index)] per class."""
    if eps <= 0:
        return [(st, mt, np.arange(len(st))) for st, mt in groups]
    mags = [np.sqrt(np.sum(np.abs(state_a(st)) ** 2, axis=1)) for st, _ in groups]
    top = max(float(m.max()) if m.size else 0.0 for m in mags)
    out = []
    for (st, mt), m in zip(groups, mags):
        idx = np.nonzero(m > eps * top)[0]
        out.append((st[idx], mt[idx], idx))
    return out


def rhs(model: Model, st: np.ndarray, meta: np.ndarray) -> np.ndarray:
    st = np.ascontiguousarray(st, dtype=np.float64)
    meta = np.ascontiguousarray(meta, dtype=np.int32)
    out = np.zeros_like(st)
    lib().orc_rhs_many(model.ptr, st.shape[0], _ptr(st), _ptr(meta), _ptr(out))
    return out


def sample_schedule(times, dt: float, nsteps: int, t0: float = 0.0):
    """Step index and fraction of each sample time: n = min(floor((t - t0)/dt), nsteps - 1),
    theta = (t - t0)/dt - n."""
    times = np.asarray(times, dtype=np.float64)
    u = (times - t0) / dt
    n = np.minimum(np.floor(u), nsteps - 1).astype(np.int32)
    th = u - n
    return n, th


def propagate(model: Model, st: np.ndarray, meta: np.ndarray, dt: float, nsteps: int,
              s_step=None, s_theta=None, w: float = 1.0):
    """RK4 (in place on st) with reconstruction records at the scheduled samples: [ns, nb, 12]."""
    assert st.flags.c_contiguous and st.dtype == np.float64
    meta = np.ascontiguousarray(meta, dtype=np.int32)
    if s_step is None:
        s_step = np.zeros(0, dtype=np.int32)
        s_theta = np.zeros(0)
    s_step = np.ascontiguousarray(s_step, dtype=np.int32)
    s_theta = np.ascontiguousarray(s_theta, dtype=np.float64)
    assert np.all(np.diff(s_step) >= 0)
    nb = st.shape[0]
    rec = np.zeros((s_step.size, nb, 12))
    lib().orc_propagate(model.ptr, nb, _ptr(st), _ptr(meta), float(dt), int(nsteps), s_step.size,
                        _ptr(s_step), _ptr(s_theta), float(w), _ptr(rec))
    return rec


def records(st: np.ndarray, meta: np.ndarray, w: float) -> np.ndarray:
    st = np.ascontiguousarray(st, dtype=np.float64)
    meta = np.ascontiguousarray(meta, dtype=np.int32)
    rec = np.zeros((st.shape[0], 12))
    lib().orc_records(st.shape[0], _ptr(st), _ptr(meta), float(w), _ptr(rec))
    return rec


def gauss_sum(rec: np.ndarray, k: float, rw: float, x: np.ndarray) -> np.ndarray:
    """u(x) = sum_b A_b exp(ik P_b.(x-Q_b) - k|x-Q_b|^2/2) (Eq. FGA); rw <= 0: every beam."""
    rec = np.ascontiguousarray(rec, dtype=np.float64).reshape(-1, 12)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    u = np.zeros((x.shape[0], 3), dtype=np.complex128)
    lib().orc_gauss_sum(rec.shape[0], _ptr(rec), float(k), float(rw), x.shape[0], _ptr(x), _ptr(u))
    return u


def interface_event(model: Model, mt: int, state: np.ndarray, lb: int, rel_min: float = 1e-6):
    """Children (states [n,48], metas [n]) of one beam at the interface to layer lb (Sec. 3.1)."""
    st = np.ascontiguousarray(state, dtype=np.float64).reshape(STATE_DOUBLES)
    out = np.zeros((4, STATE_DOUBLES))
    mo = np.zeros(4, dtype=np.int32)
    n = lib().orc_interface_event(model.ptr, int(mt), _ptr(st), int(lb), float(rel_min), _ptr(out), _ptr(mo))
    return out[:n].copy(), mo[:n].copy()


def layered_step(model: Model, st: np.ndarray, meta: np.ndarray, path: np.ndarray, dt: float, gmax: int = 4,
                 rel_min: float = 1e-6, return_parent: bool = False):
    """One RK4 step of a layered medium with interface events; returns the new (st, meta, path)
    (and the index of each output beam's input beam if return_parent)."""
    st = np.ascontiguousarray(st, dtype=np.float64)
    meta = np.ascontiguousarray(meta, dtype=np.int32)
    path = np.ascontiguousarray(path, dtype=np.int64)
    cap = 4 * st.shape[0] + 4
    out = np.zeros((cap, STATE_DOUBLES))
    mo = np.zeros(cap, dtype=np.int32)
    po = np.zeros(cap, dtype=np.int64)
    par = np.zeros(cap, dtype=np.int32)
    n = lib().orc_layered_step(model.ptr, st.shape[0], _ptr(st), _ptr(meta), _ptr(path), float(dt), int(gmax),
                               float(rel_min), cap, _ptr(out), _ptr(mo), _ptr(po), _ptr(par))
    assert n >= 0
    if return_parent:
        return out[:n].copy(), mo[:n].copy(), po[:n].copy(), par[:n].copy()
    return out[:n].copy(), mo[:n].copy(), po[:n].copy()


def layer_frame(normal) -> np.ndarray:
    """Tilted layers (interfaces normal . x = z_i): an orthonormal frame whose third axis is the unit
    normal, as the rows of a rotation R (x' = R x).  The in-plane axes come from Gram-Schmidt on the
    coordinate axis least parallel to the normal; a layered medium is invariant under rotations about
    its normal, so any in-plane choice gives the same physics."""
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    e = np.zeros(3)
    e[int(np.argmin(np.abs(n)))] = 1.0
    e1 = e - (e @ n) * n
    e1 /= np.linalg.norm(e1)
    return np.stack([e1, np.cross(n, e1), n])


def to_vector_form(st: np.ndarray, meta: np.ndarray):
    """S beams given by (a_sv, a_sh) in their frame (N_sh = e x P/|e x P|, N_sv = N_sh x P/|P|, e = e1
    for beams flagged META_REF_E1, else e3) rewritten with the displacement vector a_sv N_sv + a_sh N_sh
    in the amplitude slot (META_VECTOR).  P beams and vector-form beams are unchanged."""
    out = np.array(st, dtype=np.float64, copy=True)
    mo = np.array(meta, dtype=np.int32, copy=True)
    for b in np.nonzero(((mo & 3) >= 2) & ((mo & META_VECTOR) == 0))[0]:
        P = out[b, 3:6]
        e = np.array([1.0, 0.0, 0.0]) if mo[b] & META_REF_E1 else np.array([0.0, 0.0, 1.0])
        nsh = np.cross(e, P)
        nsh /= np.linalg.norm(nsh)
        nsv = np.cross(nsh, P / np.linalg.norm(P))
        a = out[b, 42:48].copy().view(complex)
        out[b, 42:48] = (a[0] * nsv + a[1] * nsh).view(np.float64)
        mo[b] |= META_VECTOR
    return out, mo


def rotate_beams(st: np.ndarray, meta: np.ndarray, Rm: np.ndarray, z_interfaces=None):
    """Beams into the frame x' = Rm x: Q, P, each row m of dzQ and dzP (the vector dQ/dz_m, dP/dz_m) and,
    for S beams, the amplitude vector rotate (vector form, meta bit META_VECTOR: the amplitude slot holds
    the displacement vector; a P beam's scalar amplitude along P/|P| is unchanged).
    With z_interfaces the layer bits (4-7) are set from the rotated depth Q'_3 (a beam on an interface
    belongs to the deeper side, as in the flat medium).  S beams in frame form are first rewritten in
    vector form (to_vector_form).  Returns new (st, meta)."""
    st, meta = to_vector_form(st, meta)
    swave = (meta & 3) >= 2
    out = np.array(st, dtype=np.float64, copy=True)
    out[:, 0:3] = st[:, 0:3] @ Rm.T
    out[:, 3:6] = st[:, 3:6] @ Rm.T
    for sl in (slice(6, 24), slice(24, 42)):
        M = st[:, sl].copy().view(complex).reshape(-1, 3, 3)        # [beam][m][j]
        out[:, sl] = (M @ Rm.T).reshape(-1, 9).view(np.float64)
    a = st[:, 42:48].copy().view(complex)
    out[swave, 42:48] = (a[swave] @ Rm.T).view(np.float64)
    mo = np.array(meta, dtype=np.int32, copy=True)
    if z_interfaces is not None:
        lay = np.searchsorted(np.asarray(z_interfaces, dtype=np.float64), out[:, 2], side="right")
        mo = (mo & ~np.int32(0xF0)) | (lay.astype(np.int32) << 4)
    return out, mo


def rk4_many(model: Model, st: np.ndarray, meta: np.ndarray, dt: float) -> np.ndarray:
    """One classical RK4 step of size dt for each beam (in a layered medium, each in its own layer)."""
    st = np.ascontiguousarray(st, dtype=np.float64).reshape(-1, STATE_DOUBLES)
    meta = np.ascontiguousarray(meta, dtype=np.int32).reshape(-1)
    out = np.zeros_like(st)
    if st.shape[0]:
        lib().orc_rk4_many(model.ptr, st.shape[0], _ptr(st), _ptr(meta), float(dt), _ptr(out))
    return out


def shell_layer(model: Model, x: np.ndarray) -> np.ndarray:
    """Layer of points in spherical layers: the number of spheres |x - centre| = radius that enclose the
    point (layer 0 outside the largest; a point on a sphere counts as inside it)."""
    r = np.linalg.norm(np.asarray(x, dtype=np.float64).reshape(-1, 3) - model.center, axis=1)
    return np.sum(r[:, None] <= model.radii[None, :], axis=1)


def shell_crossing(model: Model, q0: np.ndarray, q1: np.ndarray, layer: np.ndarray):
    """Spherical layers: where the straight path of one step q0 -> q1 (in a homogeneous layer a beam moves
    on a line) first meets a sphere that bounds its layer.  The points q0 + th (q1 - q0) at distance rho
    from the centre solve a th^2 + b th + c = 0.  Entering the inner sphere is the smaller root, taken when
    it lies below 1 with the path heading inward; leaving the enclosing sphere (a ball is convex, so only
    an end point outside it can mean that) is the larger root.  Returns arrays th (NaN: no crossing), the
    layer entered and the radius crossed, per beam."""
    q0 = np.asarray(q0, dtype=np.float64).reshape(-1, 3)
    q1 = np.asarray(q1, dtype=np.float64).reshape(-1, 3)
    L = np.asarray(layer).reshape(-1)
    n = q0.shape[0]
    s0, d = q0 - model.center, q1 - q0
    a = np.sum(d * d, axis=1)
    b = 2.0 * np.sum(s0 * d, axis=1)
    th = np.full(n, np.nan)
    lb = L.copy()
    rho = np.zeros(n)
    R = model.radii
    nl = R.size + 1
    for i in range(n):
        cand = []
        if L[i] < nl - 1:                                       # the inner sphere
            r = R[L[i]]
            c = s0[i] @ s0[i] - r * r
            disc = b[i] * b[i] - 4.0 * a[i] * c
            if b[i] < 0.0 and disc >= 0.0:
                t = (-b[i] - math.sqrt(disc)) / (2.0 * a[i])
                if t < 1.0:
                    cand.append((t, L[i] + 1, r))
        if L[i] > 0:                                            # the enclosing sphere
            r = R[L[i] - 1]
            e = q1[i] - model.center
            if e @ e > r * r:
                c = s0[i] @ s0[i] - r * r
                disc = max(b[i] * b[i] - 4.0 * a[i] * c, 0.0)
                cand.append(((-b[i] + math.sqrt(disc)) / (2.0 * a[i]), L[i] - 1, r))
        if cand:
            th[i], lb[i], rho[i] = min(cand, key=lambda v: v[0])
    return th, lb, rho


def shell_event(model: Model, mt: int, state: np.ndarray, lb: int, rel_min: float = 1e-6):
    """Children of a beam sitting on a sphere of a spherically layered medium.  Sec. 3.1 handles an
    interface of general shape in the local tangent-normal coordinates of the point hit, with the tangent
    plane as the flat interface: the beam is rotated into a frame whose third axis is the sphere's outward
    normal there (layer_frame), split by the flat event (interface_event), and its children are rotated
    back.  S beams go through in vector form.  Returns (states, metas) in global coordinates."""
    st = np.asarray(state, dtype=np.float64).reshape(1, STATE_DOUBLES)
    nrm = st[0, 0:3] - model.center
    Rm = layer_frame(nrm)
    st_l, mt_l = rotate_beams(st, np.array([mt], dtype=np.int32), Rm)
    kids, km = interface_event(model, int(mt_l[0]), st_l[0], lb, rel_min)
    if kids.shape[0] == 0:
        return kids, km
    return rotate_beams(kids, km, Rm.T)


def shell_step(model: Model, st: np.ndarray, meta: np.ndarray, path: np.ndarray, dt: float, gmax: int = 4,
               rel_min: float = 1e-6, return_parent: bool = False):
    """One RK4 step of a medium of spherical layers with interface events, the spherical counterpart of
    layered_step: a beam whose step meets a sphere (shell_crossing) is advanced to the crossing, put on the
    sphere, replaced by the children of shell_event, and each child is advanced through the rest of the
    step.  Beams that have crossed gmax interfaces are dropped at their next one.  Returns (st, meta, path)
    and, with return_parent, the input index of each output beam."""
    st = np.ascontiguousarray(st, dtype=np.float64)
    meta = np.ascontiguousarray(meta, dtype=np.int32)
    path = np.ascontiguousarray(path, dtype=np.int64)
    y1 = rk4_many(model, st, meta, dt)
    th, lb, rho = shell_crossing(model, st[:, 0:3], y1[:, 0:3], meta_layer(meta))
    out, mo, po, par = [], [], [], []
    for b in range(st.shape[0]):
        if np.isnan(th[b]):
            out.append(y1[b])
            mo.append(meta[b])
            po.append(path[b])
            par.append(b)
            continue
        if meta_gen(meta[b]) >= gmax:
            continue
        yc = rk4_many(model, st[b:b + 1], meta[b:b + 1], th[b] * dt)[0]
        s = yc[0:3] - model.center
        yc[0:3] = model.center + rho[b] * s / np.linalg.norm(s)
        kids, km = shell_event(model, int(meta[b]), yc, int(lb[b]), rel_min)
        ye = rk4_many(model, kids, km, (1.0 - th[b]) * dt)
        L = int(meta_layer(meta[b]))
        for k in range(ye.shape[0]):
            slot = (1 if km[k] & 2 else 0) + (0 if int(meta_layer(km[k])) == L else 2)   # rP, rS, tP, tS
            out.append(ye[k])
            mo.append(km[k])
            po.append(path[b] * 4 + slot + 1)
            par.append(b)
    res = (np.array(out).reshape(-1, STATE_DOUBLES), np.array(mo, dtype=np.int32), np.array(po, dtype=np.int64))
    return res + (np.array(par, dtype=np.int32),) if return_parent else res


def surface_height(model: Model, i: int, x: np.ndarray) -> np.ndarray:
    """Undulating layers: the height x3 of interface i above the points' (x1, x2),
    z_i + a_i cos(k1 x1) cos(k2 x2) with k_d = 2 pi / wavelength_d."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    k1, k2 = model.k_und
    return model.z_interfaces[i] + model.amp[i] * np.cos(k1 * x[:, 0]) * np.cos(k2 * x[:, 1])


def surface_normal(model: Model, i: int, x) -> np.ndarray:
    """Unit normal of undulating interface i at the point x (towards larger x3): (-dh/dx1, -dh/dx2, 1)
    normalised, from the derivatives of the height."""
    x = np.asarray(x, dtype=np.float64).reshape(3)
    k1, k2 = model.k_und
    a = model.amp[i]
    h1 = -a * k1 * math.sin(k1 * x[0]) * math.cos(k2 * x[1])
    h2 = -a * k2 * math.cos(k1 * x[0]) * math.sin(k2 * x[1])
    n = np.array([-h1, -h2, 1.0])
    return n / np.linalg.norm(n)


def surface_layer(model: Model, x: np.ndarray) -> np.ndarray:
    """Layer of points in undulating layers: the number of interfaces at or above them."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    nl = model.z_interfaces.size
    return sum((x[:, 2] >= surface_height(model, i, x)).astype(int) for i in range(nl)) if nl else \
        np.zeros(x.shape[0], dtype=int)


def surface_crossing(model: Model, q0: np.ndarray, q1: np.ndarray, layer: np.ndarray):
    """Undulating layers: where the straight path of one step q0 -> q1 meets an interface bounding its layer.
    An end point on or below the lower interface (or above the upper one) means a crossing; g(th) = x3(th) -
    h(x1(th), x2(th)) along the path then changes sign on [0, 1], and the root is found by Brent's method.
    Should the start already lie beyond the interface (no sign change), the root of g's linear
    interpolation between the ends is taken, as the flat layers do (the start itself when g is the same at
    both ends).  Returns arrays th (NaN: no crossing)
    and the layer entered, per beam."""
    from scipy.optimize import brentq
    q0 = np.asarray(q0, dtype=np.float64).reshape(-1, 3)
    q1 = np.asarray(q1, dtype=np.float64).reshape(-1, 3)
    L = np.asarray(layer).reshape(-1)
    n = q0.shape[0]
    nl = model.z_interfaces.size + 1
    th = np.full(n, np.nan)
    lb = L.copy()
    # beams whose end point lies beyond an interface of their layer (the others have no crossing)
    beyond = np.zeros(n, dtype=bool)
    for i in range(nl - 1):
        g1 = q1[:, 2] - surface_height(model, i, q1)
        beyond |= ((L == i) & (g1 >= 0.0)) | ((L == i + 1) & (g1 < 0.0))
    for b in np.nonzero(beyond)[0]:
        d = q1[b] - q0[b]
        cand = []
        for i, down in ((L[b], True), (L[b] - 1, False)):
            if i < 0 or i > nl - 2:
                continue
            g = lambda t, i=i: (q0[b, 2] + t * d[2]) - surface_height(model, i, (q0[b] + t * d)[None])[0]
            g0, g1 = g(0.0), g(1.0)
            if (down and g1 >= 0.0) or (not down and g1 < 0.0):
                if (g0 < 0.0) == down:          # a sign change on [0, 1]
                    t = brentq(g, 0.0, 1.0, xtol=1e-15, rtol=1e-15, maxiter=200)
                else:
                    t = g0 / (g0 - g1) if g0 != g1 else 0.0
                cand.append((t, L[b] + 1 if down else L[b] - 1))
        if cand:
            th[b], lb[b] = min(cand, key=lambda v: v[0])
    return th, lb


def surface_event(model: Model, mt: int, state: np.ndarray, i: int, lb: int, rel_min: float = 1e-6):
    """Children of a beam sitting on undulating interface i: as shell_event, in the frame of the surface's
    normal at the beam's centre (Sec. 3.1's local tangent-normal coordinates)."""
    st = np.asarray(state, dtype=np.float64).reshape(1, STATE_DOUBLES)
    Rm = layer_frame(surface_normal(model, i, st[0, 0:3]))
    st_l, mt_l = rotate_beams(st, np.array([mt], dtype=np.int32), Rm)
    kids, km = interface_event(model, int(mt_l[0]), st_l[0], lb, rel_min)
    if kids.shape[0] == 0:
        return kids, km
    return rotate_beams(kids, km, Rm.T)


def surface_step(model: Model, st: np.ndarray, meta: np.ndarray, path: np.ndarray, dt: float, gmax: int = 4,
                 rel_min: float = 1e-6, return_parent: bool = False):
    """One RK4 step of a medium of undulating layers with interface events, as shell_step: the crossing of
    surface_crossing, the crossing point put on the surface (x3 = h(x1, x2)), the children of
    surface_event, each advanced through the rest of the step."""
    st = np.ascontiguousarray(st, dtype=np.float64)
    meta = np.ascontiguousarray(meta, dtype=np.int32)
    path = np.ascontiguousarray(path, dtype=np.int64)
    y1 = rk4_many(model, st, meta, dt)
    th, lb = surface_crossing(model, st[:, 0:3], y1[:, 0:3], meta_layer(meta))
    out, mo, po, par = [], [], [], []
    for b in range(st.shape[0]):
        if np.isnan(th[b]):
            out.append(y1[b])
            mo.append(meta[b])
            po.append(path[b])
            par.append(b)
            continue
        if meta_gen(meta[b]) >= gmax:
            continue
        L = int(meta_layer(meta[b]))
        i = min(L, int(lb[b]))
        yc = rk4_many(model, st[b:b + 1], meta[b:b + 1], th[b] * dt)[0]
        yc[2] = surface_height(model, i, yc[None, 0:3])[0]
        kids, km = surface_event(model, int(meta[b]), yc, i, int(lb[b]), rel_min)
        ye = rk4_many(model, kids, km, (1.0 - th[b]) * dt)
        for k in range(ye.shape[0]):
            slot = (1 if km[k] & 2 else 0) + (0 if int(meta_layer(km[k])) == L else 2)   # rP, rS, tP, tS
            out.append(ye[k])
            mo.append(km[k])
            po.append(path[b] * 4 + slot + 1)
            par.append(b)
    res = (np.array(out).reshape(-1, STATE_DOUBLES), np.array(mo, dtype=np.int32), np.array(po, dtype=np.int64))
    return res + (np.array(par, dtype=np.int32),) if return_parent else res


def spherical_to_cartesian(rtp: np.ndarray) -> np.ndarray:
    """Points (r, theta, phi) -> x = (r cos theta cos phi, r sin theta cos phi, r sin phi): the change of
    the reconstruction point x of Eq. FGA that Sec. 3 uses for its spherical (layered-Earth) geometry,
    r the distance to the centre, theta the longitude, phi the latitude (radians)."""
    rtp = np.asarray(rtp, dtype=np.float64).reshape(-1, 3)
    r, th, ph = rtp[:, 0], rtp[:, 1], rtp[:, 2]
    return np.stack([r * np.cos(th) * np.cos(ph), r * np.sin(th) * np.cos(ph), r * np.sin(ph)], -1)


def bin_keys_f32(Q: np.ndarray, origin, inv_h: float, nc) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.float32).reshape(-1, 3)
    o = np.ascontiguousarray(origin, dtype=np.float32).reshape(3)
    nc = np.ascontiguousarray(nc, dtype=np.int32).reshape(3)
    key = np.zeros(Q.shape[0], dtype=np.int32)
    lib().orc_bin_keys_f32(Q.shape[0], _ptr(Q), _ptr(o), C.c_float(np.float32(inv_h)), _ptr(nc), _ptr(key))
    return key


def bin_sort(key: np.ndarray, ncells: int):
    key = np.ascontiguousarray(key, dtype=np.int32)
    perm = np.zeros(key.size, dtype=np.int32)
    start = np.zeros(ncells + 1, dtype=np.int32)
    lib().orc_bin_sort(key.size, _ptr(key), int(ncells), _ptr(perm), _ptr(start))
    return perm, start


# --------------------------------------------------------------------------------------------
# views of the 48-double state
# --------------------------------------------------------------------------------------------

def state_Q(st):
    return st[:, 0:3]


def state_P(st):
    return st[:, 3:6]


def state_DQ(st):
    """dz Q as complex [nb, 3, 3], row m = d/dz_m."""
    return st[:, 6:24].view(np.complex128).reshape(-1, 3, 3)


def state_DP(st):
    return st[:, 24:42].view(np.complex128).reshape(-1, 3, 3)


def state_a(st):
    return st[:, 42:48].view(np.complex128).reshape(-1, 3)


# --------------------------------------------------------------------------------------------
# the whole forward solve, step by step (Fig. fig:FGA_alg)
# --------------------------------------------------------------------------------------------

def solve(model: Model, k: float, mesh: Mesh, F: np.ndarray, G, classes, dt: float, nsteps: int,
          times, x: np.ndarray, rw: float, vector_form: bool = False, snap=None):
    """Decomposed data (F, G) -> beams of the given classes -> RK4 -> Gaussian sums at points x
    and sample times (and at the points `snap` at t = nsteps*dt).
    Returns complex [ns, nx, 3] (and complex [nsnap, 3] if snap is given)."""
    s_step, s_theta = sample_schedule(times, dt, nsteps)
    w = mesh.weight(k)
    out = np.zeros((len(times), x.shape[0], 3), dtype=np.complex128)
    snap_u = None if snap is None else np.zeros((snap.shape[0], 3), dtype=np.complex128)
    for cls in classes:
        st, meta = beam_init(model, k, mesh, F, G, cls, vector_form)
        rec = propagate(model, st, meta, dt, nsteps, s_step, s_theta, w)
        for j in range(len(times)):
            out[j] += gauss_sum(rec[j], k, rw, x)
        if snap is not None:
            snap_u += gauss_sum(records(st, meta, w), k, rw, snap)
    return out if snap is None else (out, snap_u)


def rhs_vjp(model: Model, state: np.ndarray, mt: int, fbar: np.ndarray, grads: bool = True):
    """Reverse mode of rhs at one state: returns (ybar [48], gp_bar, gs_bar) for the cotangent fbar
    of dy/dt (the node-field cotangents are None unless the model is a grid and grads is set)."""
    y = np.ascontiguousarray(state, dtype=np.float64).reshape(STATE_DOUBLES)
    fb = np.ascontiguousarray(fbar, dtype=np.float64).reshape(STATE_DOUBLES)
    yb = np.zeros(STATE_DOUBLES)
    gp = gs = None
    if grads and model.kind == "grid":
        shp = tuple(model.s.n) + (10,)
        gp, gs = np.zeros(shp), np.zeros(shp)
    lib().orc_rhs_vjp(model.ptr, int(mt), _ptr(y), _ptr(fb), _ptr(yb), None if gp is None else _ptr(gp),
                      None if gs is None else _ptr(gs))
    return yb, gp, gs


def solve_vjp(model: Model, k: float, mesh: Mesh, F: np.ndarray, G, classes, dt: float, nsteps: int, times,
              x: np.ndarray, rw: float, ubar: np.ndarray):
    """Reverse mode of `solve` (seismograms only) with respect to the node fields of a grid model.
    ubar: complex [ns, nx, 3] cotangent of the seismograms (dL/dRe u + i dL/dIm u).  Returns
    (gp_bar, gs_bar), float64 arrays shaped like the model's grids."""
    assert model.kind == "grid"
    s_step, s_theta = sample_schedule(times, dt, nsteps)
    w = mesh.weight(k)
    shp = tuple(model.s.n) + (10,)
    gp, gs = np.zeros(shp), np.zeros(shp)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    ub = np.ascontiguousarray(ubar, dtype=np.complex128)
    assert ub.shape == (len(times), x.shape[0], 3)
    Fc = np.ascontiguousarray(F, dtype=np.complex128)
    Gc = None if G is None else np.ascontiguousarray(G, dtype=np.complex128)
    for cls in classes:
        st, meta = beam_init(model, k, mesh, F, G, cls, False)
        stb = np.zeros_like(st)
        rc = lib().orc_solve_vjp(model.ptr, st.shape[0], _ptr(st), _ptr(meta), float(dt), int(nsteps), len(times),
                                 _ptr(s_step), _ptr(s_theta), w, float(k), float(rw), x.shape[0], _ptr(x), _ptr(ub),
                                 _ptr(stb), _ptr(gp), _ptr(gs))
        assert rc == 0, rc
        lib().orc_beam_init_vjp(model.ptr, float(k), mesh.nq, _ptr(mesh.q0), _ptr(mesh.dq), mesh.np, _ptr(mesh.p0),
                                _ptr(mesh.dp), _ptr(Fc), None if Gc is None else _ptr(Gc), int(cls), _ptr(stb),
                                _ptr(gp), _ptr(gs))
    return gp, gs
