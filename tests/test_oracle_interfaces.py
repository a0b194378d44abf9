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
