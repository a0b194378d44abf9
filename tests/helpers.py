"""Shared test glue: turn a seeded workload into oracle arguments and into GPU-library arguments."""
import numpy as np


def oracle_model(O, med):
    if med.kind == "layered":
        return O.Model("layered", z_interfaces=med.z_interfaces, layer_cp=med.layer_cp, layer_cs=med.layer_cs,
                       layer_rho=med.layer_rho, layer_shape=med.layer_shape, layer_center=med.layer_center,
                       layer_amp=med.layer_amp, layer_wavelength=med.layer_wavelength)
    return O.Model(med.kind, cp0=med.cp0, cs0=med.cs0, amp=med.amp, cs_ratio=med.cs_ratio,
                   grid_p=med.grid_p, grid_s=med.grid_s, origin=med.origin, spacing=med.spacing)


def oracle_mesh(O, m):
    return O.Mesh(m.nq, m.q0, m.dq, m.np_, m.p0, m.dp)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def max_rel_dominant(a, b, frac=1e-3):
    """Largest element-wise relative error |a - b| / |b| over the entries of b whose magnitude is at
    least `frac` of its largest one (complex entries compared by modulus).  Beside a relative L2 over a
    whole array, this catches an error confined to a few beams, receivers or mesh points."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    mag = np.abs(b)
    if mag.size == 0 or mag.max() == 0:
        return float(np.abs(a).max()) if a.size else 0.0
    sel = mag >= frac * mag.max()
    return float(np.max(np.abs(a[sel] - b[sel]) / mag[sel]))


def oracle_beams(O, w, classes=None, vector_form=False):
    """Oracle decomposition + initialisation of a workload: list of (cls, state, meta)."""
    model = oracle_model(O, w.medium)
    mesh = oracle_mesh(O, w.mesh)
    F = O.fbi(w.f, w.y0, w.dy, w.k, mesh)
    G = O.fbi(w.g, w.y0, w.dy, w.k, mesh) if w.g is not None else None
    out = []
    for cls in (classes if classes is not None else w.classes):
        st, meta = O.beam_init(model, w.k, mesh, F, G, cls, vector_form)
        out.append((cls, st, meta))
    return model, mesh, out


def gpu_setup(w, precision, device="cuda"):
    """GPU model and decomposition descriptor of a workload (tensors kept alive by the caller)."""
    import torch
    from paper_1810_06760_gb300 import fga
    model = fga.model_from_medium(w.medium, device)
    f = torch.as_tensor(w.f, device=device)
    g = torch.as_tensor(w.g, device=device) if w.g is not None else None
    desc = fga.init_desc(w.k, f, g, w.y0, w.dy, w.mesh, w.classes, precision)
    return model, desc, (f, g)
