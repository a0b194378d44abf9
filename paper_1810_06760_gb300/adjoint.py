"""Seismograms as a differentiable function of the gridded velocity model (torch.autograd).

The forward solve and its reverse mode both run in the library (fga_solve, fga_solve_vjp); this
module only wires them into torch.autograd:

* ``Seismograms.apply(fields_p, fields_s, spec)`` maps the node fields of the P and S grids
  ([n0, n1, n2, 10] float32 CUDA tensors: c, grad c, Hess c per node) to the seismograms
  [n_times, n_rx, 3] of one source; its backward calls the library's adjoint.
* ``traveltime_misfit(u, d, dt, max_lag)`` is the cross-correlation traveltime misfit of the
  seismograms, whose backward is the library's adjoint source (fga_traveltime_adjoint).
* ``fields_from_nodes(c, h)`` builds the 10 fields of a node grid of speeds with second-order
  finite differences (plain differentiable torch ops), so a gradient with respect to the speeds
  themselves follows by the chain rule, e.g. for c_s = c_p / sqrt(3) tied to c_p.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

from . import fga


@dataclasses.dataclass
class SourceSpec:
    """One forward problem besides the model: the decomposition descriptor and the solve geometry."""
    desc: object            # fga.InitDesc (its f/g tensors must stay alive: keep them in `keep`)
    dt: float
    nsteps: int
    times: np.ndarray
    rx: object              # CUDA float64 [n_rx, 3]
    rw: float = 0.0
    origin: tuple = (0.0, 0.0, 0.0)
    spacing: tuple = (1.0, 1.0, 1.0)
    checkpoint_every: int = 20
    keep: tuple = ()


def _model(fields_p, fields_s, spec: SourceSpec) -> fga.Model:
    return fga.Model("grid", grid_p=fields_p.detach().float().contiguous(),
                     grid_s=fields_s.detach().float().contiguous(), origin=spec.origin, spacing=spec.spacing)


def _seismograms():
    import torch

    class Seismograms(torch.autograd.Function):
        @staticmethod
        def forward(ctx, fields_p, fields_s, spec: SourceSpec):
            model = _model(fields_p, fields_s, spec)
            u, _ = fga.solve(model, spec.desc, spec.dt, spec.nsteps, spec.times, spec.rx, rw=spec.rw)
            ctx.model, ctx.spec = model, spec
            ctx.dtypes = (fields_p.dtype, fields_s.dtype)
            return u

        @staticmethod
        def backward(ctx, gu):
            spec = ctx.spec
            gp, gs = fga.solve_vjp(ctx.model, spec.desc, spec.dt, spec.nsteps, spec.times, spec.rx,
                                   gu.contiguous(), rw=spec.rw, checkpoint_every=spec.checkpoint_every)
            ctx.model.close()
            return gp.to(ctx.dtypes[0]), gs.to(ctx.dtypes[1]), None

    return Seismograms


_FN = None


def seismograms(fields_p, fields_s, spec: SourceSpec):
    """Differentiable seismograms of one source (see the module docstring)."""
    global _FN
    if _FN is None:
        _FN = _seismograms()
    return _FN.apply(fields_p, fields_s, spec)


def fields_from_nodes(c, h):
    """[n0, n1, n2] node speeds -> [n0, n1, n2, 10] fields (c, c_1, c_2, c_3, c_11, c_12, c_13, c_22,
    c_23, c_33) by second-order differences (central inside, one-sided at the faces); the mixed
    derivatives apply the first-difference operators of two axes, which commute."""
    import torch
    hs = [float(v) for v in (h if hasattr(h, "__len__") else (h, h, h))]
    g = [torch.gradient(c, spacing=hs[a], dim=a, edge_order=2)[0] for a in range(3)]

    def d(t, a):
        return torch.gradient(t, spacing=hs[a], dim=a, edge_order=2)[0]

    return torch.stack([c, g[0], g[1], g[2], d(g[0], 0), d(g[0], 1), d(g[0], 2), d(g[1], 1), d(g[1], 2),
                        d(g[2], 2)], -1)


def misfit(u, d):
    """L2 waveform misfit 1/2 sum |u - d|^2."""
    return 0.5 * (u - d).abs().pow(2).sum()


def _traveltime():
    import torch

    class TraveltimeMisfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u, d, dt, max_lag):
            _, ubar, mis = fga.traveltime_adjoint(u.detach(), d.detach().to(u.dtype), dt, max_lag)
            ctx.save_for_backward(ubar)
            return mis[0]

        @staticmethod
        def backward(ctx, g):
            (ubar,) = ctx.saved_tensors
            # ubar is dL/dRe u + i dL/dIm u, the gradient torch keeps for a real loss of complex u
            return ubar * g.to(ubar.real.dtype), None, None, None

    return TraveltimeMisfit


_TT = None


def traveltime_misfit(u, d, dt: float, max_lag: int):
    """Cross-correlation traveltime misfit 1/2 sum_r tau_r^2 of seismograms u against data d (CUDA complex
    [n_times, n_rx, 3], samples dt apart, delays within max_lag samples), as a float64 scalar.  Its
    backward is the synthetic-only adjoint source of fga_traveltime_adjoint, so
    traveltime_misfit(seismograms(...), d, ...).backward() gives the traveltime-tomography gradient."""
    global _TT
    if _TT is None:
        _TT = _traveltime()
    return _TT.apply(u, d, float(dt), int(max_lag))


def cs_from_cp(cp, ratio: float = 1.0 / math.sqrt(3.0)):
    return cp * ratio
