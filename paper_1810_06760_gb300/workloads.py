"""Seeded synthetic inputs for the FGA solves (shared by the tests, the oracle and the benchmark).

This module only builds inputs: media, initial data sampled on the decomposition grid, (q,p)
meshes, receivers, sample times.  It holds none of the method's arithmetic (no transform,
no ray or amplitude equations, no summation) and imports neither the GPU library nor the oracle.

The workloads are shaped like the paper's experiments:
  * ``homogeneous``: constant c_p = 2, c_s = 1; a rightward P packet
    u0 = e1 exp(-k|x-x0|^2/2) exp(i k x1), v0 = -i k c_p u0 (P+ beams only); k = 32,
    q 12^3 x p 6^3 (373,248 beams) over x0 +- 4.8/sqrt(k) and (1,0,0) +- 4.8/sqrt(k), RK4 dt = 0.005 to T = 0.5, 1,000 seeded-uniform receivers.
  * ``smooth``: c_p = 2 + 0.2 sin(2 pi x1) sin(2 pi x2) sin(2 pi x3), c_s = c_p/sqrt(3), rho = 1,
    sampled with its analytic derivatives on a 128^3 FP32 node grid over [0,1]^3; a packet
    polarised neither along nor across its direction, so P, SV and SH are all excited; k = 64,
    q 24^3 over x0 +- 6/sqrt(k) x p 8^3 over d +- 4.8/sqrt(k) (7,077,888 mesh points, x4 classes), dt = 0.0025 to T = 1, a 64^3 snapshot and
    400 surface receivers x 1,000 samples.
Reduced sizes of the same recipes serve as parity cases.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

SQRT3 = math.sqrt(3.0)


def mesh_radius(k: float, rho: float = 4.8) -> float:
    """Half-width R = rho/sqrt(k) of a q or p mesh.  The wave-packet weights of a packet decay like
    exp(-k(|q-x0|^2 + |p-p0|^2)/4), i.e. exp(-rho^2/4) at the mesh edge (rho = 4.8: 3e-3 of the peak;
    rho = 7.43: 1e-6).  A wider mesh with the same point count aliases the phase of the
    reconstruction integrand, so rho is chosen together with the point count."""
    return rho / math.sqrt(k)


def window_radius(k: float) -> float:
    """Truncation radius 6/sqrt(k) of the Gaussian sum (exp(-k r^2/2) = e^-18 at the edge)."""
    return 6.0 / math.sqrt(k)


@dataclasses.dataclass
class MeshSpec:
    nq: int
    q0: np.ndarray   # first q node, per axis
    dq: np.ndarray   # q spacing, per axis
    np_: int
    p0: np.ndarray
    dp: np.ndarray

    @property
    def M(self) -> int:
        return self.nq ** 3 * self.np_ ** 3


def centred_mesh(nq: int, qc, np_: int, pc, R: float, Rp: Optional[float] = None) -> MeshSpec:
    """Cell-centred tensor meshes over qc +- R (nq per axis) and pc +- Rp (np per axis; Rp = R if
    not given)."""
    Rp = R if Rp is None else Rp
    qc = np.asarray(qc, dtype=np.float64)
    pc = np.asarray(pc, dtype=np.float64)
    dq = np.full(3, 2.0 * R / nq)
    dp = np.full(3, 2.0 * Rp / np_)
    return MeshSpec(nq, qc - R + 0.5 * dq, dq, np_, pc - Rp + 0.5 * dp, dp)


@dataclasses.dataclass
class Medium:
    kind: str                       # 'const' | 'sine' | 'grid'
    cp0: float = 2.0
    cs0: float = 1.0
    amp: float = 0.0
    cs_ratio: float = 1.0 / SQRT3
    grid_p: Optional[np.ndarray] = None   # float32 [n0, n1, n2, 10]
    grid_s: Optional[np.ndarray] = None
    origin: Sequence[float] = (0.0, 0.0, 0.0)
    spacing: Sequence[float] = (1.0, 1.0, 1.0)
    z_interfaces: Sequence[float] = ()
    layer_cp: Sequence[float] = ()
    layer_cs: Sequence[float] = ()
    layer_rho: Sequence[float] = ()
    layer_normal: Sequence[float] = (0.0, 0.0, 0.0)   # layered: interfaces are normal . x = z_i ((0,0,0): x3)
    layer_shape: str = "planes"                       # layered: 'planes', 'spheres' (|x - layer_center| = z_i) or
    layer_center: Sequence[float] = (0.0, 0.0, 0.0)   # 'undulating' (x3 = z_i + a_i cos(2 pi x1/l1) cos(2 pi x2/l2))
    layer_amp: Sequence[float] = ()
    layer_wavelength: Sequence[float] = (1.0, 1.0)


def sine_fields_on_nodes(n: int, c0: float, amp: float, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """c = c0 + amp sin(2 pi x1) sin(2 pi x2) sin(2 pi x3) with its exact gradient and Hessian,
    sampled on an n^3 node grid over [lo, hi]^3.  Field order: c, c_1, c_2, c_3, c_11, c_12, c_13,
    c_22, c_23, c_33.  Returns float32 [n, n, n, 10]."""
    x = np.linspace(lo, hi, n)
    w = 2.0 * math.pi
    s, co = np.sin(w * x), np.cos(w * x)
    S1, S2, S3 = np.meshgrid(s, s, s, indexing="ij")
    C1, C2, C3 = np.meshgrid(co, co, co, indexing="ij")
    out = np.empty((n, n, n, 10))
    out[..., 0] = c0 + amp * S1 * S2 * S3
    out[..., 1] = amp * w * C1 * S2 * S3
    out[..., 2] = amp * w * S1 * C2 * S3
    out[..., 3] = amp * w * S1 * S2 * C3
    out[..., 4] = -amp * w * w * S1 * S2 * S3
    out[..., 5] = amp * w * w * C1 * C2 * S3
    out[..., 6] = amp * w * w * C1 * S2 * C3
    out[..., 7] = -amp * w * w * S1 * S2 * S3
    out[..., 8] = amp * w * w * S1 * C2 * C3
    out[..., 9] = -amp * w * w * S1 * S2 * S3
    return out.astype(np.float32)


@dataclasses.dataclass
class Workload:
    name: str
    k: float
    medium: Medium
    ny: int
    y0: np.ndarray            # first y node per axis
    dy: np.ndarray            # y spacing per axis
    f: np.ndarray             # complex128 [ny, ny, ny, 3] initial displacement on the y grid
    g: Optional[np.ndarray]   # complex128 [ny, ny, ny, 3] initial velocity, or None (zero)
    mesh: MeshSpec
    classes: tuple            # subset of (0 P+, 1 P-, 2 S+, 3 S-)
    dt: float
    nsteps: int
    times: np.ndarray         # sample times, increasing, in (0, nsteps*dt]
    receivers: np.ndarray     # float64 [nr, 3]
    rw: float                 # Gaussian-sum truncation radius
    snapshot: Optional[np.ndarray] = None   # float64 [ns, 3] grid points sampled at T
    rx_axes: Optional[tuple] = None         # receivers as a lattice (three 1-D arrays), same order
    snap_axes: Optional[tuple] = None       # snapshot as a lattice, same order as `snapshot`

    @property
    def T(self) -> float:
        return self.dt * self.nsteps

    @property
    def n_beams(self) -> int:
        return self.mesh.M * len(self.classes)


def _ygrid(x0, half: float, ny):
    """Cell-centred y grid over x0 +- half with ny points per axis (an int or three ints)."""
    n = np.broadcast_to(np.asarray(ny, dtype=np.float64), (3,))
    dy = 2.0 * half / n
    y0 = np.asarray(x0, dtype=np.float64) - half + 0.5 * dy
    return y0, dy


def _packet(y0, dy, ny, k: float, x0, pol, d) -> np.ndarray:
    """pol * exp(-k|y-x0|^2/2) * exp(i k d.y) on the y grid (a complex [ny0,ny1,ny2,3] array; ny an int
    or three ints)."""
    n = np.broadcast_to(np.asarray(ny, dtype=np.int64), (3,))
    ax = [y0[a] + dy[a] * np.arange(n[a]) for a in range(3)]
    Y = np.stack(np.meshgrid(*ax, indexing="ij"), -1)
    r2 = np.sum((Y - np.asarray(x0)) ** 2, axis=-1)
    ph = k * (Y @ np.asarray(d, dtype=np.float64))
    env = np.exp(-0.5 * k * r2 + 1j * ph)
    return env[..., None] * np.asarray(pol, dtype=np.float64)


def homogeneous(nq: int = 12, np_: int = 6, ny: int = 96, nsteps: int = 100, dt: float = 0.005,
                n_receivers: int = 1000, k: float = 32.0, seed: int = 0, n_times: int = 1) -> Workload:
    x0 = np.array([0.5, 0.5, 0.5])
    y0, dy = _ygrid(x0, window_radius(k), ny)
    f = _packet(y0, dy, ny, k, x0, [1.0, 0.0, 0.0], [1.0, 0.0, 0.0])
    cp = 2.0
    g = -1j * k * cp * f
    mesh = centred_mesh(nq, x0, np_, [1.0, 0.0, 0.0], mesh_radius(k, 4.8))
    rng = np.random.default_rng(seed)
    rx = rng.uniform(0.0, 1.0, size=(n_receivers, 3))
    T = dt * nsteps
    times = T * np.arange(1, n_times + 1) / n_times
    return Workload("homogeneous", k, Medium("const", cp0=cp, cs0=1.0), ny, y0, dy, f, g, mesh, (0,),
                    dt, nsteps, times, rx, window_radius(k))


def smooth(nq: int = 24, np_: int = 8, ny: int = 128, nsteps: int = 400, dt: float = 0.0025,
           n_samples: int = 1000, rx_side: int = 20, snap_side: int = 64, grid_n: int = 128,
           k: float = 64.0, grid: bool = True, classes=(0, 1, 2, 3)) -> Workload:
    x0 = np.array([0.35, 0.45, 0.55])
    dhat = np.array([3.0, 2.0, 1.0]) / math.sqrt(14.0)
    b = np.array([0.2, -0.5, 1.0])
    b = b / np.linalg.norm(b)
    y0, dy = _ygrid(x0, window_radius(k), ny)
    f = _packet(y0, dy, ny, k, x0, b, dhat)
    mesh = centred_mesh(nq, x0, np_, dhat, mesh_radius(k, 6.0), mesh_radius(k, 4.8))
    if grid:
        gp = sine_fields_on_nodes(grid_n, 2.0, 0.2)
        gs = (gp.astype(np.float64) / SQRT3).astype(np.float32)
        h = 1.0 / (grid_n - 1)
        med = Medium("grid", grid_p=gp, grid_s=gs, origin=(0.0, 0.0, 0.0), spacing=(h, h, h))
    else:
        med = Medium("sine", cp0=2.0, amp=0.2, cs_ratio=1.0 / SQRT3)
    T = dt * nsteps
    times = T * np.arange(1, n_samples + 1) / n_samples
    r = (np.arange(rx_side) + 0.5) / rx_side
    R1, R2 = np.meshgrid(r, r, indexing="ij")
    rx = np.stack([R1.ravel(), R2.ravel(), np.zeros(R1.size)], -1)
    rx_axes = (r, r, np.zeros(1))
    snap = snap_axes = None
    if snap_side:
        s = (np.arange(snap_side) + 0.5) / snap_side
        S1, S2, S3 = np.meshgrid(s, s, s, indexing="ij")
        snap = np.stack([S1.ravel(), S2.ravel(), S3.ravel()], -1)
        snap_axes = (s, s, s)
    return Workload("smooth", k, med, ny, y0, dy, f, None, mesh, tuple(classes), dt, nsteps, times, rx,
                    window_radius(k), snap, rx_axes, snap_axes)


def transform_case(ny=(128, 128, 128), nq: int = 24, np_: int = 8, k: float = 64.0):
    """Input of the wave-packet transform alone, shaped like the smooth workload's decomposition: its
    packet (centre, direction, polarisation) sampled on a y grid over x0 +- 6/sqrt(k) with ny points per
    axis (an int or three ints), and its q, p mesh (nq, np_ per axis).  Returns (f, y0, dy, mesh, k)."""
    x0 = np.array([0.35, 0.45, 0.55])
    dhat = np.array([3.0, 2.0, 1.0]) / math.sqrt(14.0)
    b = np.array([0.2, -0.5, 1.0])
    b = b / np.linalg.norm(b)
    y0, dy = _ygrid(x0, window_radius(k), ny)
    f = _packet(y0, dy, ny, k, x0, b, dhat)
    mesh = centred_mesh(nq, x0, np_, dhat, mesh_radius(k, 6.0), mesh_radius(k, 4.8))
    return f, y0, dy, mesh, k


def random_points(n: int, lo, hi, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n, 3))


def explosive_source(y0, dy, ny: int, x0, ell: float, sigma: float) -> np.ndarray:
    """u0 = grad[exp(-r^2/(2 sigma^2)) cos(2 pi r/ell)], r = |y - x0| (the radially symmetric source form
    of the paper's layered-Earth example), on the y grid: complex [ny, ny, ny, 3]."""
    ax = [y0[a] + dy[a] * np.arange(ny) for a in range(3)]
    Y = np.stack(np.meshgrid(*ax, indexing="ij"), -1) - np.asarray(x0)
    r = np.sqrt(np.sum(Y * Y, -1))
    rs = np.where(r == 0, 1.0, r)
    dphi = np.exp(-r * r / (2 * sigma * sigma)) * (-r / sigma ** 2 * np.cos(2 * np.pi * r / ell)
                                                   - 2 * np.pi / ell * np.sin(2 * np.pi * r / ell))
    return (dphi / rs)[..., None] * Y + 0j


def layered(nq: int = 4, np_: int = 6, ny: int = 32, nsteps: int = 60, dt: float = 0.05, n_times: int = 12,
            rx_side: int = 8, extent: float = 40.0, classes=(0, 1, 2, 3)) -> Workload:
    """Flat 3-layer crust in km and s: 0-15 km (c_p 5.8, c_s 3.46, rho 2.72), 15-35 km (6.5, 3.85, 2.92),
    half-space (8.04, 4.47, 3.32); depth is x3.  Explosive source at 10 km depth with dominant
    frequency 2 Hz: ell = c_p/2 Hz = 2.9 km, sigma = 0.45 ell, k = 2 pi/ell; v0 = 0.  The wavefront is
    spherical, so the p-mesh is the cube [-1.5, 1.5]^3 and the q-mesh spans the source.  Receivers on
    an rx_side^2 lattice at the surface spanning +-extent/2 km; samples on step ends."""
    ell = 5.8 / 2.0
    sigma = 0.45 * ell
    k = 2 * math.pi / ell
    x0 = np.array([0.0, 0.0, 10.0])
    half = 3.2 * sigma
    y0, dy = _ygrid(x0, half, ny)
    f = explosive_source(y0, dy, ny, x0, ell, sigma)
    mesh = centred_mesh(nq, x0, np_, [0.0, 0.0, 0.0], 2.2 * sigma, 1.5)
    med = Medium("layered", z_interfaces=(15.0, 35.0), layer_cp=(5.8, 6.5, 8.04), layer_cs=(3.46, 3.85, 4.47),
                 layer_rho=(2.72, 2.92, 3.32))
    T = dt * nsteps
    every = max(1, nsteps // n_times)
    times = dt * np.arange(every, nsteps + 1, every)
    r = np.linspace(-extent / 2, extent / 2, rx_side)
    R1, R2 = np.meshgrid(r, r, indexing="ij")
    rx = np.stack([R1.ravel(), R2.ravel(), np.zeros(R1.size)], -1)
    return Workload("layered", k, med, ny, y0, dy, f, None, mesh, tuple(classes), dt, nsteps, times, rx,
                    window_radius(k), None, (r, r, np.zeros(1)), None)


def shells(nq: int = 4, np_: int = 6, ny: int = 32, nsteps: int = 60, dt: float = 0.05, n_times: int = 12,
           rx_side: int = 8, extent: float = 30.0, rc: float = 60.0, classes=(0, 1, 2, 3)) -> Workload:
    """The 3-layer crust of ``layered`` bent into concentric spheres about (0, 0, rc): the interfaces are the
    spheres of radii rc - 15 and rc - 35 km (15 and 35 km below the point (0, 0, 0) of the outer sphere
    r = rc), layer 0 outside the larger one.  With rc = 60 km the interfaces curve strongly over the beams'
    paths.  The same explosive source at (0, 0, 10) (2 Hz, v0 = 0) and meshes as ``layered``; receivers on
    an rx_side^2 patch of the sphere r = rc around (0, 0, 0) spanning +-extent/2 km in x1 and x2."""
    w = layered(nq=nq, np_=np_, ny=ny, nsteps=nsteps, dt=dt, n_times=n_times, rx_side=rx_side, classes=classes)
    med = Medium("layered", z_interfaces=(rc - 15.0, rc - 35.0), layer_cp=w.medium.layer_cp,
                 layer_cs=w.medium.layer_cs, layer_rho=w.medium.layer_rho, layer_shape="spheres",
                 layer_center=(0.0, 0.0, rc))
    r = np.linspace(-extent / 2, extent / 2, rx_side)
    R1, R2 = np.meshgrid(r, r, indexing="ij")
    x3 = rc - np.sqrt(rc * rc - R1 ** 2 - R2 ** 2)
    rx = np.stack([R1.ravel(), R2.ravel(), x3.ravel()], -1)
    return Workload("shells", w.k, med, w.ny, w.y0, w.dy, w.f, None, w.mesh, w.classes, w.dt, w.nsteps, w.times, rx,
                    w.rw, None, None, None)


def undulating(nq: int = 4, np_: int = 6, ny: int = 32, nsteps: int = 60, dt: float = 0.05, n_times: int = 12,
               rx_side: int = 8, extent: float = 40.0, amp=(3.0, -2.0), wavelength=(20.0, 30.0),
               classes=(0, 1, 2, 3)) -> Workload:
    """The 3-layer crust of ``layered`` with undulating interfaces x3 = z_i + a_i cos(2 pi x1/l1) cos(2 pi x2/l2),
    z = (15, 35) km, a = amp (opposite signs by default, so the layer between them thickens and thins:
    the interfaces are not parallel), wavelengths (20, 30) km.  Same source, meshes and surface receivers."""
    w = layered(nq=nq, np_=np_, ny=ny, nsteps=nsteps, dt=dt, n_times=n_times, rx_side=rx_side, extent=extent,
                classes=classes)
    med = Medium("layered", z_interfaces=w.medium.z_interfaces, layer_cp=w.medium.layer_cp,
                 layer_cs=w.medium.layer_cs, layer_rho=w.medium.layer_rho, layer_shape="undulating",
                 layer_amp=tuple(amp), layer_wavelength=tuple(wavelength))
    return Workload("undulating", w.k, med, w.ny, w.y0, w.dy, w.f, None, w.mesh, w.classes, w.dt, w.nsteps, w.times,
                    w.receivers, w.rw, None, w.rx_axes, None)


def _bump_fields(fields: np.ndarray, n: int, centre, sigma: float, eps: float, lo: float = 0.0,
                 hi: float = 1.0) -> np.ndarray:
    """Fields (c, grad c, Hess c) of c * (1 + eps exp(-|x - centre|^2 / (2 sigma^2))) by the product rule,
    from the fields of c on the same n^3 node grid over [lo, hi]^3."""
    x = np.linspace(lo, hi, n)
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1) - np.asarray(centre, dtype=np.float64)
    e = np.exp(-np.sum(X * X, -1) / (2.0 * sigma * sigma))
    s = 1.0 + eps * e
    gs = (eps * e / sigma ** 2)[..., None] * -X                        # grad s
    Hs = (eps * e)[..., None, None] * (X[..., :, None] * X[..., None, :] / sigma ** 4 - np.eye(3) / sigma ** 2)
    F = fields.astype(np.float64)
    c = F[..., 0]
    gc = F[..., 1:4]
    iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    Hc = np.zeros(c.shape + (3, 3))
    for f, (a, b) in enumerate(iu):
        Hc[..., a, b] = Hc[..., b, a] = F[..., 4 + f]
    out = np.empty_like(F)
    out[..., 0] = c * s
    out[..., 1:4] = s[..., None] * gc + c[..., None] * gs
    Ht = (s[..., None, None] * Hc + gc[..., :, None] * gs[..., None, :] + gs[..., :, None] * gc[..., None, :]
          + c[..., None, None] * Hs)
    for f, (a, b) in enumerate(iu):
        out[..., 4 + f] = Ht[..., a, b]
    return out.astype(np.float32)


def crosswell(n_src_side: int = 4, nq: int = 12, np_: int = 8, ny: int = 128, nsteps: int = 200,
              dt: float = 0.0025, k: float = 64.0, grid_n: int = 64, rx_side: int = 16, n_times: int = 100,
              classes=(0, 1, 2, 3), src_x1: float = 0.1, rx_x1: float = 0.9, times=None, v0=None,
              src_offset=(0.0, 0.0)):
    """Crosswell geometry for the adjoint: the smooth medium (c_p = 2 + 0.2 sin sin sin, c_s = c_p/sqrt 3)
    on a grid_n^3 node grid is the background; the true medium multiplies c_p and c_s by
    1 + 0.05 exp(-|x - (.5,.5,.5)|^2 / (2 0.1^2)).  Sources on an n_src_side^2 lattice in the plane
    x1 = src_x1 (shifted by src_offset in x2, x3), each a packet travelling along e1 with the polarisation
    of the smooth workload (P and S excited); v0 = None gives zero initial velocity, else g = v0 * f.
    Receivers on an rx_side^2 lattice in the plane x1 = rx_x1; samples t_j = (j+1) T / n_times unless
    `times` is given.  Returns (list of per-source Workloads on the background, true Medium)."""
    gp = sine_fields_on_nodes(grid_n, 2.0, 0.2)
    gs = (gp.astype(np.float64) / SQRT3).astype(np.float32)
    h = 1.0 / (grid_n - 1)
    back = Medium("grid", grid_p=gp, grid_s=gs, origin=(0.0, 0.0, 0.0), spacing=(h, h, h))
    tp = _bump_fields(gp, grid_n, (0.5, 0.5, 0.5), 0.1, 0.05)
    ts = (tp.astype(np.float64) / SQRT3).astype(np.float32)
    true = Medium("grid", grid_p=tp, grid_s=ts, origin=(0.0, 0.0, 0.0), spacing=(h, h, h))
    dhat = np.array([1.0, 0.0, 0.0])
    b = np.array([0.2, -0.5, 1.0])
    b = b / np.linalg.norm(b)
    T = dt * nsteps
    if times is None:
        times = T * np.arange(1, n_times + 1) / n_times
    times = np.asarray(times, dtype=np.float64)
    r = (np.arange(rx_side) + 0.5) / rx_side
    R1, R2 = np.meshgrid(r, r, indexing="ij")
    rx = np.stack([np.full(R1.size, rx_x1), R1.ravel(), R2.ravel()], -1)
    out = []
    sp = (np.arange(n_src_side) + 0.5) / n_src_side
    for a in sp:
        for c in sp:
            x0 = np.array([src_x1, a + src_offset[0], c + src_offset[1]])
            y0, dy = _ygrid(x0, window_radius(k), ny)
            f = _packet(y0, dy, ny, k, x0, b, dhat)
            g = None if v0 is None else v0 * f
            mesh = centred_mesh(nq, x0, np_, dhat, mesh_radius(k, 6.0), mesh_radius(k, 4.8))
            out.append(Workload("crosswell", k, back, ny, y0, dy, f, g, mesh, tuple(classes), dt, nsteps, times,
                                rx, window_radius(k)))
    return out, true


@dataclasses.dataclass
class ServingRequest:
    arrival: float            # seconds after the first arrival (rate 1; scale by 1/rate)
    workload: Workload
    n_target: int             # the drawn mesh size N (the realised count is workload.mesh.M)


def serving_requests(n: int = 64, seed: int = 1, n_range=(1e5, 2e7), ks=(32.0, 64.0, 128.0), np_: int = 8,
                     nsteps: int = 200, dt: float = 0.0025, rx_side: int = 16, n_times: int = 200,
                     grid_n: int = 128, classes=(0, 1, 2, 3)):
    """Request mix for the serving loop, on the smooth medium (resident, shared): arrivals of a Poisson
    process of rate 1 (exponential gaps, seed `seed`); per request a source centre x0 uniform in
    [0.2, 0.8]^3, k drawn from ks, N log-uniform in n_range mapped to p 8^3 and q n_q^3 with
    n_q = round((N/512)^(1/3)), a random unit direction d and a random unit polarisation b; zero initial
    velocity; the y grid spans x0 +- 6/sqrt(k) with ny = 8 ceil(sqrt(k)) points per axis (at least ~4
    points per wavelength).  Receivers rx_side^2 at x3 = 0, samples t_j = (j+1) T / n_times."""
    rng = np.random.default_rng(seed)
    gp = sine_fields_on_nodes(grid_n, 2.0, 0.2)
    gs = (gp.astype(np.float64) / SQRT3).astype(np.float32)
    h = 1.0 / (grid_n - 1)
    med = Medium("grid", grid_p=gp, grid_s=gs, origin=(0.0, 0.0, 0.0), spacing=(h, h, h))
    r = (np.arange(rx_side) + 0.5) / rx_side
    R1, R2 = np.meshgrid(r, r, indexing="ij")
    rx = np.stack([R1.ravel(), R2.ravel(), np.zeros(R1.size)], -1)
    T = dt * nsteps
    times = T * np.arange(1, n_times + 1) / n_times
    t = 0.0
    out = []
    for i in range(n):
        if i > 0:
            t += rng.exponential(1.0)
        x0 = rng.uniform(0.2, 0.8, 3)
        k = float(ks[rng.integers(len(ks))])
        N = math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))
        nq = max(1, int(round((N / np_ ** 3) ** (1.0 / 3.0))))
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        b = rng.normal(size=3)
        b /= np.linalg.norm(b)
        ny = 8 * int(math.ceil(math.sqrt(k)))
        y0, dy = _ygrid(x0, window_radius(k), ny)
        f = _packet(y0, dy, ny, k, x0, b, d)
        mesh = centred_mesh(nq, x0, np_, d, mesh_radius(k, 6.0), mesh_radius(k, 4.8))
        w = Workload("serving", k, med, ny, y0, dy, f, None, mesh, tuple(classes), dt, nsteps, times, rx,
                     window_radius(k), rx_axes=(r, r, np.zeros(1)))
        out.append(ServingRequest(t, w, int(round(N))))
    return out


@dataclasses.dataclass
class PointSourceCase:
    """A point-force run: the source, the FGA start and end times, the data grid, mesh and receivers."""
    x0: np.ndarray
    force: np.ndarray
    rho: float
    cp: float
    cs: float
    f: float
    T0: float
    sigma: float
    t0: float
    t1: float
    k: float
    ny: np.ndarray           # data grid points per axis
    y0: np.ndarray
    dy: np.ndarray
    mesh: MeshSpec
    receivers: np.ndarray    # [n, 3] km
    rw: float
    dt: float
    nsteps: int
    psi_rel_min: float
    rx_axes: tuple = ()      # the receivers as a lattice (x, y, z axes; receivers in x-major order)
    classes: tuple = (0, 1, 2, 3)


def e1_patch(k: float = 0.08, aq: float = 1.0, ap: float = 1.5, t0: float = 3.0, t1: float = 6.93,
             rw_mult: float = 5.0, spacing: float = 0.5, psi_rel_min: float = 1e-5, dt: float = 0.05,
             band_rel: float = 1e-3) -> PointSourceCase:
    """The paper's accuracy experiment: a point force (1, 1, 1) s(t) at x0 = (64, 64, 64) km in a
    homogeneous medium (c_p = 8, c_s = 4.619 km/s, rho = 1), s(t) = cos(2 pi f (t+T0)) exp(-(t+T0)^2/sigma^2)
    with f = 1.4702 Hz, T0 = 0.1768 s, sigma = 0.8660 s, compared at t1 = 6.93 s.

    The FGA starts at t0 = 3 s from the radiated field and its time derivative (by then the source-time
    function is below 2e-6 of its peak), and the field is compared on a patch of the slice y = 64 km:
    x - 64 in [24, 44] km, z - 64 in [-4, 4] km (`spacing` apart), where both the P and the S pulse are
    present at t1.  The q mesh covers the patch's domain of dependence at t0 (radii r - c_p (t1 - t0) to
    r - c_s (t1 - t0) along +x, widened by the summation window rw = rw_mult/sqrt(k) and 2/sqrt(k));
    the p mesh covers +-(xi_max + 3 sqrt(2k))/k along x and +-(0.4 xi_max + 3 sqrt(2k))/k across, xi_max
    the S wavenumber where the source spectrum exp(-sigma^2 (omega - 2 pi f)^2 / 4) falls to band_rel;
    spacings at most aq/sqrt(k) (q) and ap/sqrt(k) (p).  The data grid extends 6/sqrt(k) beyond the q
    mesh at about 0.35 km spacing.  RK4 steps of about dt."""
    cp, cs, f, T0, sigma = 8.0, 4.619, 1.4702, 0.1768, 0.8660
    x0 = np.array([64.0, 64.0, 64.0])
    w = 1.0 / math.sqrt(k)
    rw = rw_mult * w
    m = rw + 2.0 * w
    T = t1 - t0
    qlo = np.array([64.0 + 24.0 - cp * T - m, 64.0 - 4.0 - m, 64.0 - 4.0 - m])
    qhi = np.array([64.0 + 44.0 - cs * T + m, 64.0 + 4.0 + m, 64.0 + 4.0 + m])
    ext = qhi - qlo
    nq = int(math.ceil(ext.max() / (aq * w)))
    dq = ext / nq
    xi_max = (2.0 * math.pi * f + 2.0 * math.sqrt(math.log(1.0 / band_rel)) / sigma) / cs
    px = (xi_max + 3.0 * math.sqrt(2.0 * k)) / k
    pl = (0.4 * xi_max + 3.0 * math.sqrt(2.0 * k)) / k
    pext = np.array([2.0 * px, 2.0 * pl, 2.0 * pl])
    np_ = int(math.ceil(pext.max() / (ap * w)))
    dp = pext / np_
    mesh = MeshSpec(nq, qlo + 0.5 * dq, dq, np_, -0.5 * pext + 0.5 * dp, dp)
    ylo = qlo - 6.0 * w
    yhi = qhi + 6.0 * w
    ny = np.ceil((yhi - ylo) / 0.35).astype(np.int64)
    dy = (yhi - ylo) / ny
    r1 = np.arange(24.0, 44.0 + 1e-9, spacing)
    s3 = np.arange(-4.0, 4.0 + 1e-9, spacing)
    R1, S3 = np.meshgrid(r1, s3, indexing="ij")
    rx = np.stack([64.0 + R1.ravel(), np.full(R1.size, 64.0), 64.0 + S3.ravel()], -1)
    nsteps = max(1, int(round(T / dt)))
    return PointSourceCase(x0, np.array([1.0, 1.0, 1.0]), 1.0, cp, cs, f, T0, sigma, t0, t1, k, ny,
                           ylo + 0.5 * dy, dy, mesh, rx, rw, T / nsteps, nsteps, psi_rel_min,
                           (64.0 + r1, np.array([64.0]), 64.0 + s3))
