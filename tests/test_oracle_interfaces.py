"""Pins of the oracle's flat-interface events (Sec. 3.1): plane-wave continuity against closed forms
and energy conservation, and the dzQ/dzP jump (Eq. Inter_DzQDzP) against the limit of a thin smooth
transition layer integrated by the ordinary smooth-medium equations."""
import math

import numpy as np
import pytest


def _layered(O, cp, cs, rho, z):
    return O.Model("layered", z_interfaces=z, layer_cp=cp, layer_cs=cs, layer_rho=rho)


def _beam(O, model, cls, q, p, amps=(1.0 + 0.5j, -0.3 + 0.2j), k=16.0):
    mesh = O.Mesh(1, q, [0.1] * 3, 1, p, [0.1] * 3)
    F = np.zeros((1, 3), complex)
    st, meta = O.beam_init(model, k, mesh, np.array([[1.0, 0.0, 0.0]], complex), None, cls)
    a = O.state_a(st)
    a[0, 0] = amps[0]
    if cls >= 2:
        a[0, 1] = amps[1]
    return st[0], int(meta[0])


def _pol_energy(O, model, st, mt, lay):
    """rho c |A|^2 |P_z|/|P| of a beam (the z energy flux per omega^2/2)."""
    P = st[3:6]
    pn = np.linalg.norm(P)
    a = st[42:48].view(complex)
    wave = (mt & 3) >= 2
    rho = model._keep[3][lay]
    c = (model._keep[2] if wave else model._keep[1])[lay]
    A2 = abs(a[0]) ** 2 + (abs(a[1]) ** 2 if wave else 0.0)
    return rho * c * A2 * abs(P[2]) / pn


def test_identical_media_transmit_unchanged(oracle):
    O = oracle
    model = _layered(O, [2.0, 2.0], [1.1, 1.1], [1.5, 1.5], [0.5])
    for cls in range(4):
        st, mt = _beam(O, model, cls, [0.3, 0.4, 0.2], [0.5, -0.3, 0.8])
        assert O.meta_layer(mt) == 0
        # a little way along so dzQ is not the identity
        O.propagate(model, st[None].copy(), np.array([mt], np.int32), 0.01, 5)
        kids, km = O.interface_event(model, mt, st, 1)
        assert len(kids) == 1 and O.meta_layer(km[0]) == 1 and (km[0] & 3) == (mt & 3)
        np.testing.assert_allclose(kids[0][3:6], st[3:6], atol=1e-14)
        np.testing.assert_allclose(kids[0][6:42], st[6:42], atol=1e-13)
        np.testing.assert_allclose(kids[0][42:46], st[42:46], atol=1e-12)


def test_normal_incidence_impedance(oracle):
    """P at normal incidence: a_r = a (Z2 - Z1)/(Z1 + Z2), a_t = a 2 Z1/(Z1 + Z2), Z = rho c, with the
    polarisation along P (so the reflected displacement points back)."""
    O = oracle
    cp, rho = [2.0, 3.1], [1.2, 2.5]
    model = _layered(O, cp, [1.0, 1.6], rho, [0.5])
    st, mt = _beam(O, model, 0, [0.3, 0.3, 0.49], [0.0, 0.0, 1.0], amps=(0.7 - 0.2j, 0))
    kids, km = O.interface_event(model, mt, st, 1)
    Z1, Z2 = rho[0] * cp[0], rho[1] * cp[1]
    a = st[42:44].view(complex)[0]
    got = {("r" if O.meta_layer(m) == 0 else "t") + ("S" if m & 2 else "P"): k for k, m in zip(kids, km)}
    assert set(got) == {"rP", "tP"}
    np.testing.assert_allclose(got["rP"][42:44].view(complex)[0], a * (Z2 - Z1) / (Z1 + Z2), rtol=1e-12)
    np.testing.assert_allclose(got["tP"][42:44].view(complex)[0], a * 2 * Z1 / (Z1 + Z2), rtol=1e-12)
    assert got["rP"][5] < 0 and got["tP"][5] > 0


@pytest.mark.parametrize("cls,p", [(0, [0.45, 0.2, 0.75]), (2, [0.3, -0.25, 0.8]), (3, [0.1, 0.35, -0.7]),
                                   (1, [-0.4, 0.1, -0.9])])
def test_energy_flux_balance(oracle, cls, p):
    """Oblique incidence: the z energy flux of the incident wave equals the sum over the propagating
    reflected and transmitted waves (rho c |A|^2 cos theta, common omega); a post-critical wave
    (complex P_3, kept in the continuity system) carries none."""
    O = oracle
    model = _layered(O, [2.0, 2.6], [1.1, 1.5], [1.3, 1.9], [0.5])
    down = (1.0 if (cls & 1) == 0 else -1.0) * p[2] > 0      # the beam moves along +-P
    lay_in = 0 if down else 1
    st, mt = _beam(O, model, cls, [0.3, 0.4, 0.45 if down else 0.55], p)
    assert O.meta_layer(mt) == lay_in
    kids, km = O.interface_event(model, mt, st, 1 - lay_in, rel_min=0.0)
    assert len(kids) >= 2   # a post-critical (evanescent) wave is dropped and carries no vertical flux
    e_in = _pol_energy(O, model, st, mt, lay_in)
    e_out = sum(_pol_energy(O, model, k, m, int(O.meta_layer(m))) for k, m in zip(kids, km))
    np.testing.assert_allclose(e_out, e_in, rtol=1e-10)
    # Snell: tangential P kept, c |P| kept
    cin = (model._keep[2] if cls >= 2 else model._keep[1])[lay_in] * np.linalg.norm(st[3:6])
    for k, m in zip(kids, km):
        np.testing.assert_allclose(k[3:5], st[3:5], atol=1e-15)
        c = (model._keep[2] if m & 2 else model._keep[1])[int(O.meta_layer(m))]
        np.testing.assert_allclose(c * np.linalg.norm(k[3:6]), cin, rtol=1e-13)


def test_children_stay_symplectic(oracle):
    O = oracle
    model = _layered(O, [2.0, 2.6], [1.1, 1.5], [1.3, 1.9], [0.5])
    st, mt = _beam(O, model, 2, [0.3, 0.4, 0.4], [0.3, -0.25, 0.8])
    assert O.meta_layer(mt) == 0
    s1 = st[None].copy()
    O.propagate(model, s1, np.array([mt], np.int32), 0.01, 6)
    kids, km = O.interface_event(model, mt, s1[0], 1, rel_min=0.0)
    Om = np.block([[np.zeros((3, 3)), np.eye(3)], [-np.eye(3), np.zeros((3, 3))]])
    for k in kids:
        DQ = k[6:24].view(complex).reshape(3, 3)
        DP = k[24:42].view(complex).reshape(3, 3)
        J = np.block([[DQ.real.T, -DQ.imag.T], [DP.real.T, -DP.imag.T]])
        np.testing.assert_allclose(J.T @ Om @ J, Om, atol=1e-12)
        Z = DQ + 1j * DP
        S = np.linalg.solve(Z, DQ)
        np.testing.assert_allclose(S, S.T, atol=1e-12)


@pytest.mark.parametrize("cls", [0, 2])
def test_jump_is_the_thin_layer_limit(oracle, cls):
    """Eq. Inter_DzQDzP for the transmitted beam equals the limit of the ordinary dzQ/dzP equations
    (Eq. DzDt) through a thin smooth transition c(x3) = c1 + (c2-c1)(1 + tanh((x3-z0)/eps))/2:
    P, dzQ and dzP after the crossing agree to the accuracy of the sampled transition."""
    O = oracle
    c1, c2, z0 = 2.0, 2.6, 0.5
    ratio = 1.0 / math.sqrt(3.0)
    q, p = [0.3, 0.4, 0.42], [0.35, -0.2, 0.8]
    T, dt = 0.12, 2e-5
    layered = _layered(O, [c1, c2], [c1 * ratio, c2 * ratio], [1.0, 1.0], [z0])
    st, mt = _beam(O, layered, cls, q, p)
    cur_s, cur_m, cur_p = st[None].copy(), np.array([mt], np.int32), np.array([0], np.int64)
    for _ in range(int(round(T / dt))):
        cur_s, cur_m, cur_p = O.layered_step(layered, cur_s, cur_m, cur_p, dt, rel_min=0.0)
    trans = [i for i in range(len(cur_m)) if O.meta_layer(cur_m[i]) == 1 and (cur_m[i] & 2) == (mt & 2)]
    assert len(trans) == 1
    ref = cur_s[trans[0]]
    errs = []
    for eps in (4e-3, 2e-3):
        nz = 6001
        z = np.linspace(0.0, 1.0, nz)
        u = (z - z0) / eps
        th = np.tanh(u)
        c = c1 + (c2 - c1) * 0.5 * (1 + th)
        dc = (c2 - c1) * 0.5 * (1 - th ** 2) / eps
        d2c = (c2 - c1) * 0.5 * (-2 * th * (1 - th ** 2)) / eps ** 2
        g = np.zeros((2, 2, nz, 10), np.float32)
        g[..., 0], g[..., 3], g[..., 9] = c, dc, d2c
        gs = g.copy()
        gs[..., [0, 3, 9]] *= ratio
        smooth = O.Model("grid", grid_p=g, grid_s=gs, origin=(-5, -5, 0), spacing=(10, 10, 1.0 / (nz - 1)))
        s2, m2 = O.beam_init(smooth, 16.0, O.Mesh(1, q, [0.1] * 3, 1, p, [0.1] * 3),
                             np.array([[1.0, 0, 0]], complex), None, cls)
        O.propagate(smooth, s2, m2, dt, int(round(T / dt)))
        e = [np.linalg.norm(s2[0, sl] - ref[sl]) / np.linalg.norm(ref[sl]) for sl in (slice(3, 6), slice(6, 24),
                                                                                      slice(24, 42))]
        errs.append(max(e))
    # agreement to ~1e-4 (the floor of the FP32 node fields and the grid), at both widths ...
    assert max(errs) < 1e-3, errs
    # ... while the jump matters: without any interface the same beam misses by several percent
    homog = O.Model("const", cp0=c1, cs0=c1 * ratio)
    s3, m3 = O.beam_init(homog, 16.0, O.Mesh(1, q, [0.1] * 3, 1, p, [0.1] * 3), np.array([[1.0, 0, 0]], complex),
                         None, cls)
    O.propagate(homog, s3, m3, dt, int(round(T / dt)))
    miss = max(np.linalg.norm(s3[0, sl] - ref[sl]) / np.linalg.norm(ref[sl]) for sl in (slice(3, 6), slice(6, 24),
                                                                                          slice(24, 42)))
    assert miss > 0.03, miss


def test_lineage_keys_unique_after_splitting(oracle):
    """(root class, mesh point, path) names every beam of a split population exactly once."""
    from paper_1810_06760_gb300 import workloads as W
    from tests.helpers import oracle_beams
    w = W.layered(nq=3, np_=4, ny=24, nsteps=12, dt=0.1)
    model, mesh, obeams = oracle_beams(oracle, w)
    st = np.concatenate([b[1] for b in obeams])
    meta = np.concatenate([b[2] for b in obeams])
    mid = np.concatenate([np.arange(b[1].shape[0]) for b in obeams]).astype(np.int64)
    root0 = oracle.meta_root(meta)
    np.testing.assert_array_equal(root0, meta & 3)
    path = np.zeros(st.shape[0], dtype=np.int64)
    for _ in range(w.nsteps):
        st, meta, path, parent = oracle.layered_step(model, st, meta, path, w.dt, return_parent=True)
        mid = mid[parent]
    keys = list(zip(oracle.meta_root(meta).tolist(), mid.tolist(), path.tolist()))
    assert len(keys) > st.shape[0] // 2 and len(set(keys)) == len(keys)
    assert np.any(path > 0)


def _displacement(O, st, mt):
    """Displacement vector a N of a beam: P along P/|P|, S from its own SV/SH frame (Sec. 2.2 frame:
    N_sh = e x P/|e x P|, N_sv = N_sh x P/|P|, e = e1 for beams flagged so, else e3)."""
    P = st[3:6]
    ph = P / np.linalg.norm(P)
    a = st[42:48].view(complex)
    if (mt & 3) < 2:
        return a[0] * ph
    e = np.array([1.0, 0, 0]) if mt & O.META_REF_E1 else np.array([0, 0, 1.0])
    nsh = np.cross(e, P)
    nsh /= np.linalg.norm(nsh)
    return a[0] * np.cross(nsh, ph) + a[1] * nsh


def _traction(lam, mu, P, U):
    """sigma . e3 of the plane wave U exp(i k P.x), per unit i k: lam (P.U) e3 + mu (P U_3 + P_3 U)."""
    t = mu * (P * U[2] + P[2] * U)
    t[2] += lam * np.dot(P, U)
    return t


@pytest.mark.parametrize("cls,p,down", [
    (0, [0.3, 0.2, 0.9], True), (0, [-0.25, 0.3, -0.8], False),     # P from the slow and the fast side
    (1, [0.2, -0.3, -0.9], True),                                     # "-" branch: travels along -P
    (2, [0.3, 0.2, 0.9], True), (3, [0.1, -0.3, 0.9], False),        # S with SV and SH parts
    (2, [0.02, 0.01, 0.95], True),                                    # near-vertical S (frame about e1)
])
def test_children_satisfy_welded_continuity(oracle, cls, p, down):
    """Below every critical angle all four children propagate, and the printed Zoeppritz system
    (with the readings of its garbled entry, of SV incidence and of SH incidence) must give children
    whose displacement and traction sigma.e3 are continuous across the interface: the conditions of a
    welded interface that Eq. Yilmaz expresses in angle variables, checked here on the 3-D
    displacement vectors the children carry."""
    O = oracle
    cp, cs, rho = [2.0, 2.6], [1.1, 1.5], [1.3, 1.9]
    model = _layered(O, cp, cs, rho, [0.5])
    lay = 0 if down else 1
    st, mt = _beam(O, model, cls, [0.3, 0.4, 0.45 if down else 0.55], p)
    assert O.meta_layer(mt) == lay
    kids, km = O.interface_event(model, mt, st, 1 - lay, rel_min=0.0)
    expect = 2 if (cls >= 2 and abs(st[42:46].view(complex)[0]) == 0) else 4
    assert len(kids) == expect
    lam = [r * (a * a - 2 * b * b) for r, a, b in zip(rho, cp, cs)]
    mu = [r * b * b for r, b in zip(rho, cs)]
    U_in = _displacement(O, st, mt)
    du = U_in.copy()
    dtr = _traction(lam[lay], mu[lay], st[3:6], U_in)
    T_in = dtr.copy()
    for k, m in zip(kids, km):
        L = int(O.meta_layer(m))
        sgn = 1.0 if L == lay else -1.0
        U = _displacement(O, k, int(m))
        du += sgn * U
        dtr += sgn * _traction(lam[L], mu[L], k[3:6], U)
    assert np.linalg.norm(du) <= 1e-12 * np.linalg.norm(U_in), du
    assert np.linalg.norm(dtr) <= 1e-12 * np.linalg.norm(T_in), dtr


def test_sh_incidence_textbook_coefficients(oracle):
    """A pure SH beam (displacement horizontal, normal to the plane of incidence) yields only S
    children, with R = (Z1 cos phi1 - Z2 cos phi2)/(Z1 cos phi1 + Z2 cos phi2) and
    T = 2 Z1 cos phi1/(Z1 cos phi1 + Z2 cos phi2), Z = rho c_s (displacement amplitudes)."""
    O = oracle
    cp, cs, rho = [2.0, 2.6], [1.1, 1.5], [1.3, 1.9]
    model = _layered(O, cp, cs, rho, [0.5])
    p = np.array([0.35, 0.0, 0.8])
    st, mt = _beam(O, model, 2, [0.3, 0.4, 0.45], p, amps=(0.0, 0.8 - 0.3j))
    U_in = _displacement(O, st, mt)
    assert abs(U_in[0]) < 1e-15 and abs(U_in[2]) < 1e-15       # along e2: SH for this plane
    kids, km = O.interface_event(model, mt, st, 1, rel_min=1e-9)
    assert len(kids) == 2 and all((m & 2) for m in km)
    om = cs[0] * np.linalg.norm(p)
    c1 = math.sqrt(1 - (p[0] * cs[0] / om) ** 2)
    c2 = math.sqrt(1 - (p[0] * cs[1] / om) ** 2)
    Z1, Z2 = rho[0] * cs[0] * c1, rho[1] * cs[1] * c2
    got = {int(O.meta_layer(m)): _displacement(O, k, int(m)) for k, m in zip(kids, km)}
    np.testing.assert_allclose(got[0], U_in * (Z1 - Z2) / (Z1 + Z2), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(got[1], U_in * 2 * Z1 / (Z1 + Z2), rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------------------------------------
# tilted layers: the flat event in the frame whose third axis is the interface normal
# ---------------------------------------------------------------------------------------------

_NORMAL = np.array([0.3, -0.4, 0.85])


def _vector_beam(O, model, cls, q, p, k=16.0):
    """One beam in vector form (amplitude slot = displacement vector): P along P/|P|, S a vector
    normal to P with both in-plane components."""
    mesh = O.Mesh(1, q, [0.1] * 3, 1, p, [0.1] * 3)
    st, meta = O.beam_init(model, k, mesh, np.array([[1.0, 0.0, 0.0]], complex), None, cls, vector_form=True)
    P = np.asarray(p, dtype=np.float64)
    ph = P / np.linalg.norm(P)
    if cls < 2:
        a = np.array([1.0 + 0.5j, 0.0, 0.0])   # P: the scalar amplitude along P/|P|
    else:
        t1 = np.cross(ph, [0.2, 0.9, -0.3])
        t1 /= np.linalg.norm(t1)
        a = (1.0 + 0.5j) * t1 + (-0.3 + 0.2j) * np.cross(ph, t1)
    st[0, 42:48] = a.view(np.float64)
    return st, meta


def _traction_n(lam, mu, P, U, n):
    """sigma . n of the plane wave U exp(i k P.x), per unit i k."""
    return lam * np.dot(P, U) * n + mu * (P * np.dot(U, n) + np.dot(P, n) * U)


@pytest.mark.parametrize("cls,p,down", [(0, [0.3, 0.2, 0.9], True), (2, [0.3, 0.2, 0.9], True),
                                        (3, [0.1, -0.3, 0.9], False), (1, [0.2, -0.3, -0.9], True)])
def test_tilted_interface_children_satisfy_welded_continuity(oracle, cls, p, down):
    """A beam given in global coordinates meets the plane n.x = 0.5 (n tilted): rotated into the layer
    frame (rotate_beams with layer_frame(n)), split by the flat event, and its children rotated back,
    the displacement and the traction sigma.n are continuous across the tilted plane in global
    coordinates.  A transposed rotation or a vector left unrotated breaks this."""
    O = oracle
    cp, cs, rho = [2.0, 2.6], [1.1, 1.5], [1.3, 1.9]
    model = _layered(O, cp, cs, rho, [0.5])
    Rm = O.layer_frame(_NORMAL)
    n = Rm[2]
    lay = 0 if down else 1
    st_l, mt_l = _vector_beam(O, model, cls, [0.3, 0.4, 0.45 if down else 0.55], p)
    st_g, mt_g = O.rotate_beams(st_l, mt_l, Rm.T)                 # the beam as given in global coordinates
    st_r, mt_r = O.rotate_beams(st_g, mt_g, Rm, z_interfaces=[0.5])
    assert int(O.meta_layer(mt_r[0])) == lay
    np.testing.assert_allclose(st_r, st_l, rtol=0, atol=1e-14)
    kids, km = O.interface_event(model, int(mt_r[0]), st_r[0], 1 - lay, rel_min=0.0)
    assert len(kids) >= 2
    kids_g, km_g = O.rotate_beams(np.asarray(kids), np.asarray(km), Rm.T)
    lam = [r * (a * a - 2 * b * b) for r, a, b in zip(rho, cp, cs)]
    mu = [r * b * b for r, b in zip(rho, cs)]
    def disp(row, m):
        a = row[42:48].copy().view(complex)
        if (m & 3) < 2:
            return a[0] * row[3:6] / np.linalg.norm(row[3:6])
        return a

    U_in = disp(st_g[0], int(mt_g[0]))
    du = U_in.copy()
    dtr = _traction_n(lam[lay], mu[lay], st_g[0, 3:6], U_in, n)
    T_in = dtr.copy()
    for kg, m in zip(kids_g, km_g):
        L = int(O.meta_layer(m))
        sgn = 1.0 if L == lay else -1.0
        U = disp(kg, int(m))
        du += sgn * U
        dtr += sgn * _traction_n(lam[L], mu[L], kg[3:6], U, n)
    assert np.linalg.norm(du) <= 1e-12 * np.linalg.norm(U_in), du
    assert np.linalg.norm(dtr) <= 1e-12 * np.linalg.norm(T_in), dtr


def test_rotated_propagation_equals_global_propagation(oracle):
    """Inside one homogeneous layer, propagating beams in the layer frame and rotating them back equals
    propagating them in global coordinates (Q, P, dzQ, dzP and the amplitude vectors), which fixes the
    rotation of the Jacobian rows as well as of the vectors."""
    O = oracle
    Rm = O.layer_frame(_NORMAL)
    glob = O.Model("const", cp0=2.0, cs0=1.1)
    lay1 = O.Model("layered", z_interfaces=[], layer_cp=[2.0], layer_cs=[1.1], layer_rho=[1.3])
    for cls, p in ((0, [0.3, 0.2, 0.9]), (3, [0.1, -0.3, 0.9]), (2, [-0.5, 0.4, 0.2])):
        st_g, mt_g = _vector_beam(O, glob, cls, [0.3, 0.4, 0.45], p)
        ref = st_g.copy()
        O.propagate(glob, ref, mt_g, 0.01, 40)
        st_r, mt_r = O.rotate_beams(st_g, mt_g, Rm, z_interfaces=[])
        path = np.zeros(1, dtype=np.int64)
        for _ in range(40):
            st_r, mt_r, path = O.layered_step(lay1, st_r, mt_r, path, 0.01)
        back, _ = O.rotate_beams(st_r, mt_r, Rm.T)
        np.testing.assert_allclose(back, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


# ---------------------------------------------------------------------------------------------
# spherical layers: the flat event in the tangent-normal frame of the point where a beam meets a sphere
# ---------------------------------------------------------------------------------------------

def _spheres(O, centre, radii, cp=(2.0, 2.6, 3.1), cs=(1.1, 1.5, 1.8), rho=(1.3, 1.9, 2.4)):
    n = len(radii) + 1
    return O.Model("layered", z_interfaces=radii, layer_cp=cp[:n], layer_cs=cs[:n], layer_rho=rho[:n],
                   layer_shape="spheres", layer_center=centre)


def test_initial_layers_by_enclosing_spheres(oracle):
    """Beams start in the layer given by the spheres that enclose their centre; a centre on a sphere
    belongs to its inner side (as a centre on a plane belongs to the deeper layer)."""
    O = oracle
    c = np.array([0.2, -0.1, 3.0])
    model = _spheres(O, c, [2.0, 1.0])
    u = np.array([0.6, 0.0, -0.8])
    for r, want in ((2.5, 0), (2.0, 1), (1.5, 1), (1.0, 2), (0.3, 2)):
        st, mt = _beam(O, model, 0, c + r * u, [0.3, 0.2, 0.9])
        assert int(O.meta_layer(mt)) == want, (r, mt)
        assert int(O.shell_layer(model, (c + r * u)[None])[0]) == want


def test_crossing_of_a_path_that_dips_into_the_inner_sphere(oracle):
    """Both ends of a step may lie outside the inner sphere while the straight path between them cuts
    through it: the crossing is the entry point (on the sphere, inside the step).  A path passing just
    outside has none, and an end point beyond the enclosing sphere gives the exit point."""
    O = oracle
    c = np.zeros(3)
    model = _spheres(O, c, [3.0, 1.0])
    q0, q1 = np.array([[-0.5, 0.9, 0.0]]), np.array([[0.5, 0.9, 0.0]])       # chord at distance 0.9 < 1
    th, lb, rho = O.shell_crossing(model, q0, q1, np.array([1]))
    assert 0.0 < th[0] < 0.5 and lb[0] == 2 and rho[0] == 1.0
    x = q0[0] + th[0] * (q1[0] - q0[0])
    assert abs(np.linalg.norm(x) - 1.0) < 1e-14
    th, _, _ = O.shell_crossing(model, q0 + [0, 0.2, 0], q1 + [0, 0.2, 0], np.array([1]))
    assert np.isnan(th[0])
    q0, q1 = np.array([[0.0, 2.5, 0.5]]), np.array([[0.0, 3.5, 0.5]])
    th, lb, rho = O.shell_crossing(model, q0, q1, np.array([1]))
    assert lb[0] == 0 and rho[0] == 3.0
    x = q0[0] + th[0] * (q1[0] - q0[0])
    assert 0.0 < th[0] < 1.0 and abs(np.linalg.norm(x) - 3.0) < 1e-14


def test_radial_incidence_on_a_sphere(oracle):
    """A P beam travelling along the radius of a sphere with an arbitrary centre meets it at normal
    incidence: no converted S waves, the reflected P goes straight back, and the amplitudes are the
    normal-incidence impedance ratios (Z2 - Z1)/(Z1 + Z2), 2 Z1/(Z1 + Z2).  A normal taken along e3
    instead of the radius gives oblique incidence and S children."""
    O = oracle
    c = np.array([1.0, -2.0, 0.5])
    cp, rho = (2.0, 3.1), (1.2, 2.5)
    model = _spheres(O, c, [1.5], cp=cp, cs=(1.0, 1.6), rho=rho)
    u = np.array([2.0, 1.0, -2.0]) / 3.0
    x = c + 1.5 * u
    st, mt = _beam(O, model, 0, c + 1.7 * u, -u, amps=(0.7 - 0.2j, 0))
    st[0:3] = x
    kids, km = O.shell_event(model, mt, st, 1, rel_min=1e-9)
    got = {("r" if O.meta_layer(m) == 0 else "t") + ("S" if m & 2 else "P"): k for k, m in zip(kids, km)}
    assert set(got) == {"rP", "tP"}
    Z1, Z2 = rho[0] * cp[0], rho[1] * cp[1]
    a = st[42:44].view(complex)[0]
    np.testing.assert_allclose(got["rP"][42:44].view(complex)[0], a * (Z2 - Z1) / (Z1 + Z2), rtol=1e-12)
    np.testing.assert_allclose(got["tP"][42:44].view(complex)[0], a * 2 * Z1 / (Z1 + Z2), rtol=1e-12)
    pin = np.linalg.norm(st[3:6])
    np.testing.assert_allclose(got["rP"][3:6] / pin, u, atol=1e-14)
    np.testing.assert_allclose(got["tP"][3:6] / np.linalg.norm(got["tP"][3:6]), -u, atol=1e-14)


@pytest.mark.parametrize("cls,inward,ang", [(0, True, 0.5), (0, False, 0.4), (2, True, 0.3), (3, False, 0.3),
                                             (1, True, 0.45), (2, False, 0.25)])
def test_sphere_event_children_satisfy_welded_continuity(oracle, cls, inward, ang):
    """A beam meets a sphere (arbitrary centre) at an angle ang from its normal, below every critical angle
    so that all children propagate: the children, in global coordinates, keep displacement and traction
    sigma.n continuous across the tangent plane of the crossing point (n the sphere's normal there), keep
    the tangential part of P and c |P| (Snell), and the reflected ones travel back to the incident side."""
    O = oracle
    c = np.array([0.4, -0.3, 2.0])
    cp, cs, rho = (2.0, 2.6), (1.1, 1.5), (1.3, 1.9)
    model = _spheres(O, c, [1.5], cp=cp, cs=cs, rho=rho)
    u = np.array([-0.36, 0.48, -0.8])                   # unit vector: the crossing point is c + 1.5 u
    x = c + 1.5 * u
    t = np.cross(u, [0.6, 0.0, 0.8])
    t /= np.linalg.norm(t)
    sgn = -1.0 if cls & 1 else 1.0                      # the beam travels along sgn P
    p = sgn * 0.9 * ((-1.0 if inward else 1.0) * math.cos(ang) * u + math.sin(ang) * t)
    lay = 0 if inward else 1
    st, mt = _vector_beam(O, model, cls, x - 0.05 * sgn * np.asarray(p), p)
    assert int(O.meta_layer(mt[0])) == lay
    st = st[0].copy()
    st[0:3] = x
    kids, km = O.shell_event(model, int(mt[0]), st, 1 - lay, rel_min=0.0)
    assert len(kids) == 4
    lam = [r * (a * a - 2 * b * b) for r, a, b in zip(rho, cp, cs)]
    mu = [r * b * b for r, b in zip(rho, cs)]

    def disp(row, m):
        a = row[42:48].copy().view(complex)
        return a[0] * row[3:6] / np.linalg.norm(row[3:6]) if (m & 3) < 2 else a

    U_in = disp(st, int(mt[0]))
    du, dtr = U_in.copy(), _traction_n(lam[lay], mu[lay], st[3:6], U_in, u)
    T_in = dtr.copy()
    cin = (cs if cls >= 2 else cp)[lay] * np.linalg.norm(st[3:6])
    tang = st[3:6] - np.dot(st[3:6], u) * u
    for k, m in zip(kids, km):
        L = int(O.meta_layer(m))
        s = 1.0 if L == lay else -1.0
        U = disp(k, int(m))
        du += s * U
        dtr += s * _traction_n(lam[L], mu[L], k[3:6], U, u)
        np.testing.assert_allclose(k[3:6] - np.dot(k[3:6], u) * u, tang, atol=1e-14)
        np.testing.assert_allclose((cs if m & 2 else cp)[L] * np.linalg.norm(k[3:6]), cin, rtol=1e-13)
        travel = (-1.0 if m & 1 else 1.0) * np.dot(k[3:6], u)       # outward speed of the child
        assert (travel > 0) == (L == 0)
        np.testing.assert_allclose(k[0:3], x, atol=1e-14)
    assert np.linalg.norm(du) <= 1e-12 * np.linalg.norm(U_in), du
    assert np.linalg.norm(dtr) <= 1e-12 * np.linalg.norm(T_in), dtr


def _sphere_vs_plane_errors(O, big):
    """Relative L2 differences (Q, P, dzQ, dzP, amplitudes) between the spherical solve with radius ~big
    about a centre far along the normal n and the tilted-plane solve of the planes n.x = z_i, over
    lineages, after 30 steps of the layered workload; asserts that both have the same lineages."""
    from paper_1810_06760_gb300 import workloads as W
    from tests.helpers import oracle_beams
    nrm = np.array([0.3, -0.4, 0.85])
    nrm = nrm / np.linalg.norm(nrm)
    w = W.layered(nq=2, np_=4, ny=20, nsteps=30, dt=0.1)
    z = np.asarray(w.medium.z_interfaces)
    sph = _spheres(O, (z[0] + big) * nrm, [big, big - (z[1] - z[0])], cp=w.medium.layer_cp,
                   cs=w.medium.layer_cs, rho=w.medium.layer_rho)
    flat, _, obeams = oracle_beams(O, w)
    st0 = np.concatenate([b[1] for b in obeams])
    mt0 = np.concatenate([b[2] for b in obeams])
    mid0 = np.concatenate([np.arange(b[1].shape[0]) for b in obeams])
    Rm = O.layer_frame(nrm)
    # spherical solve in global coordinates (S beams in vector form, layers from the spheres)
    st, mt = O.to_vector_form(st0, mt0)
    mt = (mt & ~np.int32(0xF0)) | (O.shell_layer(sph, st[:, 0:3]).astype(np.int32) << 4)
    path, mid = np.zeros(st.shape[0], dtype=np.int64), mid0.copy()
    for _ in range(w.nsteps):
        st, mt, path, par = O.shell_step(sph, st, mt, path, w.dt, return_parent=True)
        mid = mid[par]
    # tilted planes: the same beams in the layer frame, flat steps, rotated back
    tf, tm = O.rotate_beams(st0, mt0, Rm, z_interfaces=z)
    tpath, tmid = np.zeros(tf.shape[0], dtype=np.int64), mid0.copy()
    for _ in range(w.nsteps):
        tf, tm, tpath, par = O.layered_step(flat, tf, tm, tpath, w.dt, return_parent=True)
        tmid = tmid[par]
    tf, tm = O.rotate_beams(tf, tm, Rm.T)
    key = lambda m, i, p: [((int(a) >> 13) & 3, int(b), int(c)) for a, b, c in zip(m, i, p)]
    ks, kt = key(mt, mid, path), key(tm, tmid, tpath)
    assert len(set(ks)) == len(ks) and set(ks) == set(kt)
    assert len(ks) > 1.5 * st0.shape[0]                 # interfaces were crossed
    it = {k: i for i, k in enumerate(kt)}
    order = [it[k] for k in ks]
    A, B = st, tf[order]
    np.testing.assert_array_equal(mt & 0x6FF3, tm[order] & 0x6FF3)
    return [np.linalg.norm(A[:, sl] - B[:, sl]) / np.linalg.norm(B[:, sl])
            for sl in (slice(0, 3), slice(3, 6), slice(6, 24), slice(24, 42), slice(42, 48))]


def test_spheres_of_large_radius_reduce_to_tilted_planes(oracle):
    """Concentric spheres of radius rho about a centre far along the normal n look, over the beams' paths,
    like the planes n.x = z_i: their gap is |x_perp|^2 / 2 rho and their normals differ by |x_perp| / rho.
    Every lineage of the spherical solve exists in the tilted-plane solve (the pinned rotate_beams + flat
    steps), and their difference falls as 1/rho: tenfold from rho = 1e7 to 1e8 km.  At 1e8 the centres,
    propagation vectors and amplitudes agree to 1e-5; the Jacobians to 2e-3, because a beam meeting an
    interface at grazing incidence (P.n/|P| ~ 0.01 here) takes the jump F with the factor 1/p_n of Eq.
    Inter_DzQDzP, which magnifies the 1/rho tilt of the normal a hundredfold."""
    e7 = _sphere_vs_plane_errors(oracle, 1.0e7)
    e8 = _sphere_vs_plane_errors(oracle, 1.0e8)
    for name, a, b, bar in zip(("Q", "P", "dzQ", "dzP", "a"), e7, e8, (1e-5, 1e-5, 2e-3, 2e-3, 1e-5)):
        assert b < bar, (name, b)
        assert 5.0 < a / b < 20.0, (name, a, b)


# ---------------------------------------------------------------------------------------------
# undulating layers: interfaces x3 = z_i + a_i cos(k1 x1) cos(k2 x2), not parallel to each other
# ---------------------------------------------------------------------------------------------

def _undulating(O, amp, z=(15.0, 35.0), wl=(20.0, 30.0), cp=(5.8, 6.5, 8.04), cs=(3.46, 3.85, 4.47),
                rho=(2.72, 2.92, 3.32)):
    n = len(z) + 1
    return O.Model("layered", z_interfaces=z, layer_cp=cp[:n], layer_cs=cs[:n], layer_rho=rho[:n],
                   layer_shape="undulating", layer_amp=amp, layer_wavelength=wl)


def _disp_rows(st, mt):
    out = np.zeros((st.shape[0], 3), complex)
    for b in range(st.shape[0]):
        P = st[b, 3:6]
        a = st[b, 42:48].copy().view(complex)
        if (mt[b] & 3) < 2:
            out[b] = a[0] * P / np.linalg.norm(P)
        elif mt[b] & 8:
            out[b] = a
        else:
            e = np.array([1.0, 0, 0]) if mt[b] & 4 else np.array([0, 0, 1.0])
            nsh = np.cross(e, P)
            nsh /= np.linalg.norm(nsh)
            out[b] = a[0] * np.cross(nsh, P / np.linalg.norm(P)) + a[1] * nsh
    return out


def test_initial_layers_below_undulating_surfaces(oracle):
    """Beams start in the layer given by the number of interfaces at or above their centre (a centre on an
    interface belongs to the deeper layer), the interfaces' heights varying along x1 and x2."""
    O = oracle
    model = _undulating(O, [3.0, -2.0])
    for x, want in (((0.0, 0.0, 17.9), 0), ((0.0, 0.0, 18.0), 1), ((10.0, 0.0, 12.1), 1), ((0.0, 0.0, 33.5), 2),
                    ((5.0, 7.5, 35.0), 2), ((10.0, 0.0, 36.9), 1)):
        st, mt = _beam(O, model, 0, x, [0.3, 0.2, 0.9])
        assert int(O.meta_layer(mt)) == want, (x, mt)
        assert int(O.surface_layer(model, np.array([x]))[0]) == want


def _surface_solve(O, model, w, nsteps):
    from tests.helpers import oracle_beams
    _, _, obeams = oracle_beams(O, w)
    st = np.concatenate([b[1] for b in obeams])
    mt = np.concatenate([b[2] for b in obeams])
    mid = np.concatenate([np.arange(b[1].shape[0]) for b in obeams])
    mt = (mt & ~np.int32(0xF0)) | (O.surface_layer(model, st[:, 0:3]).astype(np.int32) << 4)
    path = np.zeros(st.shape[0], dtype=np.int64)
    for _ in range(nsteps):
        st, mt, path, par = O.surface_step(model, st, mt, path, w.dt, return_parent=True)
        mid = mid[par]
    return st, mt, mid, path


def _lineage_diff(O, A, B):
    """Relative L2 differences of Q, P, dzQ, dzP and displacement vectors over common lineages."""
    key = lambda m, i, p: [((int(a) >> 13) & 3, int(b), int(c)) for a, b, c in zip(m, i, p)]
    ka, kb = key(A[1], A[2], A[3]), key(B[1], B[2], B[3])
    assert len(set(ka)) == len(ka) and set(ka) == set(kb)
    ib = {k: i for i, k in enumerate(kb)}
    o = [ib[k] for k in ka]
    sa, sb = A[0], B[0][o]
    np.testing.assert_array_equal(A[1] & 0x6FF3, B[1][o] & 0x6FF3)
    errs = [np.linalg.norm(sa[:, sl] - sb[:, sl]) / np.linalg.norm(sb[:, sl])
            for sl in (slice(0, 3), slice(3, 6), slice(6, 24), slice(24, 42))]
    da, db = _disp_rows(sa, A[1]), _disp_rows(sb, B[1][o])
    return errs + [np.linalg.norm(da - db) / np.linalg.norm(db)], len(ka)


def test_flat_undulating_layers_equal_flat_layers(oracle):
    """Zero amplitudes make the undulating solve the flat one: the same lineages after 30 steps and the
    same states to rounding (the crossing by Brent's method on the path instead of the linear formula, the
    event in the identity frame with S amplitudes in vector form)."""
    from paper_1810_06760_gb300 import workloads as W
    from tests.helpers import oracle_beams
    O = oracle
    w = W.layered(nq=2, np_=4, ny=20, nsteps=30, dt=0.1)
    und = _undulating(O, [0.0, 0.0])
    A = _surface_solve(O, und, w, w.nsteps)
    flat, _, obeams = oracle_beams(O, w)
    st = np.concatenate([b[1] for b in obeams])
    mt = np.concatenate([b[2] for b in obeams])
    mid = np.concatenate([np.arange(b[1].shape[0]) for b in obeams])
    path = np.zeros(st.shape[0], dtype=np.int64)
    for _ in range(w.nsteps):
        st, mt, path, par = O.layered_step(flat, st, mt, path, w.dt, return_parent=True)
        mid = mid[par]
    errs, n = _lineage_diff(O, A, (st, mt, mid, path))
    assert n > 1.5 * w.n_beams
    assert max(errs) < 1e-12, errs


def test_undulating_layers_converge_to_flat_with_the_amplitude(oracle):
    """The difference to the flat solve falls linearly with the amplitudes: tenfold from 1e-3 to 1e-4 km
    (the interface heights move by a, their normals tilt by a k), for centres, propagation vectors,
    Jacobians and displacement vectors; lineages are the same."""
    from paper_1810_06760_gb300 import workloads as W
    O = oracle
    w = W.layered(nq=2, np_=4, ny=20, nsteps=30, dt=0.1)
    ref = _surface_solve(O, _undulating(O, [0.0, 0.0]), w, w.nsteps)
    e3, _ = _lineage_diff(O, _surface_solve(O, _undulating(O, [1e-3, -1e-3]), w, w.nsteps), ref)
    e4, _ = _lineage_diff(O, _surface_solve(O, _undulating(O, [1e-4, -1e-4]), w, w.nsteps), ref)
    for a, b in zip(e3, e4):
        assert 6.0 < a / b < 16.0, (e3, e4)
    assert max(e4) < 1e-3


def test_crossing_of_an_undulating_surface(oracle):
    """The crossing lies on the surface and inside the step; an end point short of the surface means no
    crossing; a path leaving upwards crosses the interface above."""
    O = oracle
    model = _undulating(O, [3.0, -2.0])
    q0 = np.array([[4.0, 1.0, 15.0]])
    q1 = q0 + np.array([[0.4, 0.1, 1.2]])
    h = O.surface_height(model, 0, q1)[0]
    assert int(O.surface_layer(model, q0)[0]) == 0 and q1[0, 2] >= h
    th, lb = O.surface_crossing(model, q0, q1, np.array([0]))
    x = q0[0] + th[0] * (q1[0] - q0[0])
    assert 0.0 < th[0] < 1.0 and lb[0] == 1
    assert abs(x[2] - O.surface_height(model, 0, x[None])[0]) < 1e-12
    th, _ = O.surface_crossing(model, q0, q0 + np.array([[0.4, 0.1, 0.2]]), np.array([0]))
    assert np.isnan(th[0])
    q0 = np.array([[2.0, -1.0, 19.0]])
    q1 = q0 + np.array([[0.3, 0.2, -3.0]])
    assert int(O.surface_layer(model, q0)[0]) == 1 and q1[0, 2] < O.surface_height(model, 0, q1)[0]
    th, lb = O.surface_crossing(model, q0, q1, np.array([1]))
    x = q0[0] + th[0] * (q1[0] - q0[0])
    assert lb[0] == 0 and abs(x[2] - O.surface_height(model, 0, x[None])[0]) < 1e-12


@pytest.mark.parametrize("cls,down,ang", [(0, True, 0.4), (2, True, 0.3), (3, False, 0.25), (1, False, 0.35)])
def test_undulating_interface_children_satisfy_welded_continuity(oracle, cls, down, ang):
    """A beam meets an undulating interface where it slopes (normal tilted by ~30 degrees): its children
    keep displacement and traction sigma.n continuous across the tangent plane there, keep the tangential
    part of P and c |P|, and sit on the right sides; a normal taken as e3 instead breaks continuity.  The
    normal of the checks comes from central differences of the height (agreeing with the oracle's own to
    1e-8, hence the 1e-9 bars), so a wrong derivative in the oracle fails here."""
    O = oracle
    cp, cs, rho = (2.0, 2.6), (1.1, 1.5), (1.3, 1.9)
    model = _undulating(O, [3.0], z=(15.0,), wl=(20.0, 30.0), cp=cp, cs=cs, rho=rho)
    x = np.array([5.0, 3.0, 0.0])
    x[2] = O.surface_height(model, 0, x[None])[0]
    # the normal from central differences of the height, not from the oracle's own derivative
    eps = 1e-5
    hx = lambda dx, dy: O.surface_height(model, 0, (x + [dx, dy, 0.0])[None])[0]
    n = np.array([-(hx(eps, 0) - hx(-eps, 0)) / (2 * eps), -(hx(0, eps) - hx(0, -eps)) / (2 * eps), 1.0])
    n /= np.linalg.norm(n)
    assert n[2] < 0.9                                    # a sloping part of the surface
    assert np.linalg.norm(O.surface_normal(model, 0, x) - n) < 1e-8
    t = np.cross(n, [0.0, 1.0, 0.0])
    t /= np.linalg.norm(t)
    sgn = -1.0 if cls & 1 else 1.0
    p = sgn * 0.9 * ((1.0 if down else -1.0) * math.cos(ang) * n + math.sin(ang) * t)
    lay = 0 if down else 1
    st, mt = _vector_beam(O, model, cls, x - 0.05 * sgn * p, p)
    assert int(O.meta_layer(mt[0])) == lay
    st = st[0].copy()
    st[0:3] = x
    kids, km = O.surface_event(model, int(mt[0]), st, 0, 1 - lay, rel_min=0.0)
    assert len(kids) == 4
    lam = [r * (a * a - 2 * b * b) for r, a, b in zip(rho, cp, cs)]
    mu = [r * b * b for r, b in zip(rho, cs)]

    def disp(row, m):
        a = row[42:48].copy().view(complex)
        return a[0] * row[3:6] / np.linalg.norm(row[3:6]) if (m & 3) < 2 else a

    U_in = disp(st, int(mt[0]))
    du, dtr = U_in.copy(), _traction_n(lam[lay], mu[lay], st[3:6], U_in, n)
    T_in = dtr.copy()
    cin = (cs if cls >= 2 else cp)[lay] * np.linalg.norm(st[3:6])
    tang = st[3:6] - np.dot(st[3:6], n) * n
    for k, m in zip(kids, km):
        L = int(O.meta_layer(m))
        s = 1.0 if L == lay else -1.0
        U = disp(k, int(m))
        du += s * U
        dtr += s * _traction_n(lam[L], mu[L], k[3:6], U, n)
        np.testing.assert_allclose(k[3:6] - np.dot(k[3:6], n) * n, tang, atol=1e-9)
        np.testing.assert_allclose((cs if m & 2 else cp)[L] * np.linalg.norm(k[3:6]), cin, rtol=1e-13)
        travel = (-1.0 if m & 1 else 1.0) * np.dot(k[3:6], n)       # speed towards larger depth
        assert (travel > 0) == (L == 1)
    assert np.linalg.norm(du) <= 1e-9 * np.linalg.norm(U_in), du
    assert np.linalg.norm(dtr) <= 1e-9 * np.linalg.norm(T_in), dtr
    # the same event with the normal taken as e3 (a flat reading of the sloping surface) is not welded
    st_l, mt_l = O.to_vector_form(st[None], np.array([mt[0]], dtype=np.int32))
    bad, bm = O.interface_event(model, int(mt_l[0]), st_l[0], 1 - lay, rel_min=0.0)
    dtb = _traction_n(lam[lay], mu[lay], st[3:6], U_in, n)
    for k, m in zip(bad, bm):
        L = int(O.meta_layer(m))
        dtb += (1.0 if L == lay else -1.0) * _traction_n(lam[L], mu[L], k[3:6], disp(k, int(m)), n)
    assert np.linalg.norm(dtb) > 1e-3 * np.linalg.norm(T_in)


def _flux_n(model_cp, model_cs, rho, st, mt, lay, n):
    """rho c |A|^2 |P.n|/|P|: the energy flux of a beam's plane wave through a plane of normal n (per
    omega^2 / 2)."""
    P = st[3:6]
    a = st[42:48].copy().view(complex)
    wave = (mt & 3) >= 2
    A2 = float(np.sum(np.abs(a) ** 2)) if (wave and (mt & 8)) else abs(a[0]) ** 2 + (abs(a[1]) ** 2 if wave else 0.0)
    c = (model_cs if wave else model_cp)[lay]
    return rho[lay] * c * A2 * abs(np.dot(P, n)) / np.linalg.norm(P)


@pytest.mark.parametrize("shape", ["spheres", "undulating"])
@pytest.mark.parametrize("cls,ang", [(0, 0.3), (0, 0.9), (2, 0.2), (3, 0.6), (1, 0.5)])
def test_curved_interface_energy_flux_balance(oracle, shape, cls, ang):
    """At a sphere or a sloping undulating surface, the energy flux of the incident wave through the tangent
    plane equals the sum over the propagating children, below and beyond the critical angles (a
    post-critical child is not created and carries no normal flux)."""
    O = oracle
    cp, cs, rho = (2.0, 2.6), (1.1, 1.5), (1.3, 1.9)
    if shape == "spheres":
        c = np.array([0.4, -0.3, 2.0])
        model = _spheres(O, c, [1.5], cp=cp, cs=cs, rho=rho)
        u = np.array([-0.36, 0.48, -0.8])
        x = c + 1.5 * u
        n = u                                             # outward; layer 0 outside
        inward = -n                                       # towards layer 1
    else:
        model = _undulating(O, [3.0], z=(15.0,), cp=cp, cs=cs, rho=rho)
        x = np.array([5.0, 3.0, 0.0])
        x[2] = O.surface_height(model, 0, x[None])[0]
        n = O.surface_normal(model, 0, x)                 # towards larger x3, layer 1
        inward = n
    t = np.cross(n, [0.0, 1.0, 0.0])
    t /= np.linalg.norm(t)
    sgn = -1.0 if cls & 1 else 1.0
    p = sgn * 0.9 * (math.cos(ang) * inward + math.sin(ang) * t)     # travels from layer 0 into layer 1
    st, mt = _vector_beam(O, model, cls, x - 0.05 * sgn * p, p)
    assert int(O.meta_layer(mt[0])) == 0
    st = st[0].copy()
    st[0:3] = x
    if shape == "spheres":
        kids, km = O.shell_event(model, int(mt[0]), st, 1, rel_min=0.0)
    else:
        kids, km = O.surface_event(model, int(mt[0]), st, 0, 1, rel_min=0.0)
    assert len(kids) >= 2
    e_in = _flux_n(cp, cs, rho, st, int(mt[0]), 0, n)
    e_out = sum(_flux_n(cp, cs, rho, k, int(m), int(O.meta_layer(m)), n) for k, m in zip(kids, km))
    np.testing.assert_allclose(e_out, e_in, rtol=1e-10)


@pytest.mark.parametrize("shape", ["spheres", "undulating"])
def test_curved_interface_children_stay_symplectic(oracle, shape):
    """The children of an event at a sphere or a sloping undulating surface, rotated back to global
    coordinates, keep the Jacobian (dzQ, dzP) symplectic and Z^-1 dzQ symmetric, as at a flat interface:
    rotating the rows of dzQ and dzP by one orthogonal map preserves both, and a rotation applied to one of
    them only would not."""
    O = oracle
    cp, cs, rho = (2.0, 2.6), (1.1, 1.5), (1.3, 1.9)
    if shape == "spheres":
        c = np.array([0.4, -0.3, 2.0])
        model = _spheres(O, c, [1.5], cp=cp, cs=cs, rho=rho)
        n = np.array([-0.36, 0.48, -0.8])
        x = c + 1.5 * n
        inward = -n
    else:
        model = _undulating(O, [3.0], z=(15.0,), cp=cp, cs=cs, rho=rho)
        x = np.array([5.0, 3.0, 0.0])
        x[2] = O.surface_height(model, 0, x[None])[0]
        inward = O.surface_normal(model, 0, x)
    t = np.cross(inward, [0.0, 1.0, 0.0])
    t /= np.linalg.norm(t)
    p = 0.9 * (math.cos(0.35) * inward + math.sin(0.35) * t)
    st, mt = _vector_beam(O, model, 2, x - 0.3 * p, p)
    O.propagate(model, st, mt, 0.05, 6)                 # dzQ, dzP away from their initial values
    st = st[0].copy()
    st[0:3] = x
    if shape == "spheres":
        kids, km = O.shell_event(model, int(mt[0]), st, 1, rel_min=0.0)
    else:
        kids, km = O.surface_event(model, int(mt[0]), st, 0, 1, rel_min=0.0)
    assert len(kids) == 4
    Om = np.block([[np.zeros((3, 3)), np.eye(3)], [-np.eye(3), np.zeros((3, 3))]])
    for k in kids:
        DQ = k[6:24].view(complex).reshape(3, 3)
        DP = k[24:42].view(complex).reshape(3, 3)
        J = np.block([[DQ.real.T, -DQ.imag.T], [DP.real.T, -DP.imag.T]])
        np.testing.assert_allclose(J.T @ Om @ J, Om, atol=1e-11)
        S = np.linalg.solve(DQ + 1j * DP, DQ)
        np.testing.assert_allclose(S, S.T, atol=1e-11)
