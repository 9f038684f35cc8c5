"""Pins of the oracle against facts the paper and mathematics fix.

Each test checks the oracle (oracle/) against something other than itself:
closed forms evaluated in 40-digit arithmetic, Gauss's law, reciprocity,
the derivative relation between Eq. 6 and Eq. 5, far-field asymptotics,
values printed in the paper, the isolated-cube capacitance and finite
differences.  None of these touch the CUDA path.
"""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle as O
from paper_2004_02609_gb300 import workloads as W

mp.mp.dps = 40
FOURPI = 4 * mp.pi
CW = {-1: 1, 0: -2, 1: 1}          # second-difference weights


# ---- independent closed forms (4-D corner sums), in 40-digit arithmetic ----
def _log_plus(a, rest2):
    """ln(a + sqrt(a^2 + rest2)), stable for a < 0."""
    r = mp.sqrt(a * a + rest2)
    if a >= 0:
        return mp.log(a + r)
    return mp.log(rest2 / (r - a))


def _F(u, v, h):
    """d^2/du^2 d^2/dv^2 F = 1/sqrt(u^2+v^2+h^2)  (parallel squares)."""
    r = mp.sqrt(u * u + v * v + h * h)
    t = -(u * u + v * v - 2 * h * h) * r / 6
    c1 = (u * u - h * h) / 2 * v
    if c1 != 0:
        t += c1 * _log_plus(v, u * u + h * h)
    c2 = (v * v - h * h) / 2 * u
    if c2 != 0:
        t += c2 * _log_plus(u, v * v + h * h)
    if h != 0 and u * v != 0:
        t -= u * v * h * mp.atan(u * v / (h * r))
    return t


def _Fh(u, v, h):
    """d^2/du^2 d^2/dv^2 Fh = -h / r^3  (h != 0)."""
    r = mp.sqrt(u * u + v * v + h * h)
    t = h * r
    if v != 0:
        t -= h * v * _log_plus(v, u * u + h * h)
    if u != 0:
        t -= h * u * _log_plus(u, v * v + h * h)
    if u * v != 0:
        t -= u * v * mp.atan(u * v / (h * r))
    return t


def _H(p, q, w):
    """d/dp d/dq d^2/dw^2 H = 1/sqrt(p^2+q^2+w^2)  (orthogonal squares)."""
    r = mp.sqrt(p * p + q * q + w * w)
    t = -p * q * r / 3
    if p * q * w != 0:
        t += p * q * w * _log_plus(w, p * p + q * q)
    c = q * (w * w / 2 - q * q / 6)
    if c != 0:
        t += c * _log_plus(p, q * q + w * w)
    c = p * (w * w / 2 - p * p / 6)
    if c != 0:
        t += c * _log_plus(q, p * p + w * w)
    if w != 0 and q != 0:
        t -= w * q * q / 2 * mp.atan(p * w / (q * r))
    if w != 0 and p != 0:
        t -= w * p * p / 2 * mp.atan(q * w / (p * r))
    if w != 0 and p * q != 0:
        t -= w ** 3 / 6 * mp.atan(p * q / (w * r))
    return t


def _Hp(p, q, w):
    """d/dq d^2/dw^2 Hp = 1/r, equal to dH/dp up to terms the corner sum kills."""
    r = mp.sqrt(p * p + q * q + w * w)
    t = -q * r / 2
    if w * q != 0:
        t += w * q * _log_plus(w, p * p + q * q)
    c = (w * w - p * p) / 2
    if c != 0:
        t += c * _log_plus(q, p * p + w * w)
    if w * p != 0:
        t -= w * p * mp.atan(q * w / (p * r))
    return t


def cf_par(kind, h, s, t):
    h, s, t = mp.mpf(h), mp.mpf(s), mp.mpf(t)
    if kind == 1 and h == 0:
        return mp.mpf(0)
    f = _F if kind == 0 else _Fh
    acc = mp.mpf(0)
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            acc += CW[i] * CW[j] * f(s + i, t + j, h)
    return acc / FOURPI


def cf_ort(kind, a, b, c):
    a, b, c = mp.mpf(a), mp.mpf(b), mp.mpf(c)
    f = _H if kind == 0 else _Hp
    acc = mp.mpf(0)
    for s1 in (-1, 1):
        for s2 in (-1, 1):
            for j in (-1, 0, 1):
                acc += s1 * s2 * CW[j] * f(a + s1 * mp.mpf(0.5), b + s2 * mp.mpf(0.5), c + j)
    return acc / FOURPI


PAR_CASES = [(0, 0, 0), (0, 1, 0), (0, 1, 1), (0, 2, 1), (1, 0, 0), (1, 1, 0),
             (1, 1, 1), (2, 0, 1), (3, 2, 0), (5, 4, 3), (0, 3, 7)]
ORT_CASES = [(0.5, 0.5, 0), (0.5, 0.5, 1), (0.5, 1.5, 0), (1.5, 0.5, 0), (1.5, 1.5, 2),
             (0.5, 2.5, 1), (2.5, 0.5, 3), (3.5, 4.5, 2), (0.5, 0.5, 5)]


def _rel(a, b):
    return abs(float(a) - float(b)) / max(abs(float(b)), 1e-30)


def test_self_term_textbook():
    """Galerkin self term of a unit square: 4 ln(1+sqrt 2) - 4/3 (sqrt 2 - 1)."""
    ref = 4 * math.log(1 + math.sqrt(2)) - 4.0 / 3.0 * (math.sqrt(2) - 1)
    assert abs(O.entry(0, 2, 2, (0, 0, 0)) * 4 * math.pi - ref) < 1e-13 * ref


@pytest.mark.parametrize("o", [0, 1, 2])
@pytest.mark.parametrize("h,s,t", PAR_CASES)
def test_parallel_entries_vs_closed_form(o, h, s, t):
    ax = [1, 0, 0][o], [2, 2, 1][o]
    d = [0.0, 0.0, 0.0]
    d[o], d[ax[0]], d[ax[1]] = h, s, t
    for kind in (0, 1):
        ref = cf_par(kind, h, s, t)
        got = O.entry(kind, o, o, d)
        if kind == 1 and h == 0:
            assert got == 0.0
        else:
            assert _rel(got, ref) < 1e-12, (kind, o, h, s, t, got, float(ref))


@pytest.mark.parametrize("pair", [(0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1)])
@pytest.mark.parametrize("a,b,c", ORT_CASES)
def test_orthogonal_entries_vs_closed_form(pair, a, b, c):
    alpha, beta = pair
    gamma = 3 - alpha - beta
    for sa in (1, -1):
        d = [0.0, 0.0, 0.0]
        d[alpha], d[beta], d[gamma] = sa * a, b, c
        for kind in (0, 1):
            ref = cf_ort(kind, sa * a, b, c)
            got = O.entry(kind, alpha, beta, d)
            assert _rel(got, ref) < 1e-12, (kind, pair, sa * a, b, c, got, float(ref))


def test_reciprocity_orthogonal():
    """P'(test k, src l) = P'(test l, src k): the oracle treats the two panels
    differently (closed form inside, quadrature outside)."""
    rng = np.random.default_rng(1)
    for _ in range(12):
        o1, o2 = rng.choice(3, 2, replace=False)
        d = rng.integers(-3, 4, 3).astype(float)
        d[o1] -= 0.5
        d[o2] += 0.5
        a = O.entry(0, o1, o2, d)
        b = O.entry(0, o2, o1, -d)
        assert _rel(a, b) < 1e-12


def _voxel_faces(v):
    """The 6 faces of voxel v (integer lower corner): (orient, centre, outward sign)."""
    out = []
    for o in range(3):
        for side, sg in ((0, -1.0), (1, 1.0)):
            c = np.asarray(v, float) + 0.5
            c[o] = v[o] + side
            out.append((o, c, sg))
    return out


@pytest.mark.parametrize("src_o", [0, 1, 2])
def test_gauss_flux_invariant(src_o):
    """Sum over a voxel's faces of the outward normal derivative of the
    potential of a unit source panel (Eq. 6 entries with outward sign) is 0
    when the source is outside the voxel (including voxels touching it along
    an edge or a corner, where the orthogonal entry is log-singular), and -1/2
    when the source is one of its faces (half the flux enters; PV self term 0)."""
    src_c = np.array([0.5, 0.5, 0.5])
    src_c[src_o] = 0.0                     # source face at the origin plane
    voxels = []
    for dv in [(0, 0, 0), (-1, 0, 0), (0, -1, 0), (0, 0, -1), (1, 1, 0), (1, 0, 1),
               (-1, -1, -1), (2, 0, 0), (0, 2, 1), (1, -1, 1)]:
        voxels.append(tuple(dv))
    for v in voxels:
        tot = 0.0
        own = False
        for (o, c, sg) in _voxel_faces(v):
            if o == src_o and np.allclose(c, src_c):
                own = True
            tot += sg * O.entry(1, o, src_o, c - src_c)
        expect = -0.5 if own else 0.0
        assert abs(tot - expect) < 1e-11, (v, tot, expect)


def test_field_is_derivative_of_potential():
    """E' (Eq. 6) equals the derivative of P' (Eq. 5) along the test normal."""
    rng = np.random.default_rng(2)
    dl = 1e-4
    for _ in range(8):
        ot, os_ = rng.integers(0, 3, 2)
        d = rng.integers(-3, 4, 3).astype(float)
        if ot != os_:
            d[ot] -= 0.5
            d[os_] += 0.5
        if ot == os_ and d[ot] == 0:
            d[ot] = 1.0
        e = np.zeros(3)
        e[ot] = dl
        fd = (O.entry(0, ot, os_, d + e) - O.entry(0, ot, os_, d - e)) / (2 * dl)
        ex = O.entry(1, ot, os_, d)
        assert abs(fd - ex) < 1e-7 * max(abs(ex), 1e-3)


def test_far_field_quadrupole():
    """At distance R, 4 pi P' = 1/R + quadrupole term + O(R^-5): the centre
    difference of two uniform unit squares has covariance diag(1/6) in-plane."""
    for (o, d) in [(2, (30.0, 20.0, 10.0)), (0, (25.0, -30.0, 15.0))]:
        d = np.asarray(d)
        R = np.linalg.norm(d)
        var = np.full(3, 1.0 / 6.0)
        var[o] = 0.0
        quad = (3 * np.sum(var * d * d) - R * R * np.sum(var)) / (2 * R ** 5)
        got = 4 * math.pi * O.entry(0, o, o, d)
        assert abs(got - (1 / R + quad)) < 5e-7 / R


# ---- panel extraction (Sec. II.A/B) ----
def test_sphere_panel_counts_match_paper():
    """Sec. III.A prints N = 2376, 9480, 14760, 59016 for the coated sphere at
    dv = 0.05, 0.025, 0.02, 0.01 m; a voxelisation by voxel centres strictly
    inside each radius reproduces them (tests/golden/sphere_panel_counts.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "sphere_panel_counts.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for n, count in rows:
        w = W.coated_sphere(int(n))
        ps = O.panels(w.labels, w.conductor_id, w.eps_r)
        assert ps.n == int(count)


def test_panel_rules():
    # cube: 6 * a^2 conductor panels, none dielectric
    ps = O.panels(np.zeros((4, 4, 4), np.int32), np.array([0]), np.array([1.0]))
    assert ps.n == 96 and ps.n_diel == 0 and np.all(ps.qscale == 1.0)
    # equal permittivities carry no panel; vacuum-valued dielectric == vacuum
    lab = np.zeros((3, 3, 3), np.int32)
    lab[1, 1, 1] = 1
    ps = O.panels(lab, np.array([-1, -1]), np.array([1.0, 1.0]))
    assert ps.n == 0
    ps = O.panels(lab, np.array([-1, -1]), np.array([2.0, 2.0]))
    assert ps.n == 54 and ps.n_cond == 0       # only the outer boundary
    # conductor inside a dielectric: q_scale = eps of the dielectric side
    ps = O.panels(lab, np.array([-1, 0]), np.array([3.0, 1.0]))
    assert ps.n_cond == 6 and np.all(ps.qscale[ps.kind == 0] == 3.0)
    # I' sign: face normal +x from eps_a (x-) to eps_b (x+)
    lab2 = np.array([[[0, 1]]], np.int32)
    ps = O.panels(lab2, np.array([-1, -1]), np.array([2.0, 5.0]))
    inner = (ps.orient == 0) & (ps.face == 1)
    assert np.isclose(ps.idiag[inner][0], (2.0 + 5.0) / (2 * (2.0 - 5.0)))
    # short circuit
    lab3 = np.array([[[0, 1]]], np.int32)
    with pytest.raises(O.ShortCircuitError):
        O.panels(lab3, np.array([0, 1]), np.array([1.0, 1.0]))


# ---- capacitance (Eq. 8) ----
def test_cube_refinement_approaches_reference_value():
    """Isolated cube of edge a: C = 0.66067 * 4 pi eps0 a.  The piecewise-
    constant Galerkin values increase monotonically with refinement; a
    three-point extrapolation lands within 0.5 %."""
    vals = {}
    for a in (4, 8, 12, 16):
        w = W.cube(a)
        ps = O.panels(w.labels, w.conductor_id, w.eps_r)
        _, Cn, _ = O.capacitance(ps, rtol=1e-11)
        vals[a] = Cn[0, 0] / (4 * math.pi * a)
    seq = [vals[a] for a in (4, 8, 12, 16)]
    assert all(b > a for a, b in zip(seq, seq[1:]))
    assert all(v < 0.66067 for v in seq)
    # fit c_inf + k a^-p through a = 8, 12, 16
    a1, a2, a3 = 8.0, 12.0, 16.0
    f1, f2, f3 = vals[8], vals[12], vals[16]
    from scipy.optimize import brentq
    g = lambda p: (f1 - f2) / (a1 ** -p - a2 ** -p) - (f2 - f3) / (a2 ** -p - a3 ** -p)
    p = brentq(g, 0.3, 3.0)
    k = (f1 - f2) / (a1 ** -p - a2 ** -p)
    cinf = f3 - k * a3 ** -p
    assert abs(cinf - 0.66067) < 0.005 * 0.66067, (cinf, p)


def test_capacitance_matrix_properties():
    """Three conductors in vacuum: C symmetric (to discretisation error),
    C_ii > 0, C_ij < 0, row sums > 0."""
    lab = np.zeros((6, 8, 10), np.int32)
    lab[1:3, 1:4, 1:4] = 1
    lab[1:3, 1:4, 6:9] = 2
    lab[4:6, 4:7, 3:7] = 3
    ps = O.panels(lab, np.array([-1, 0, 1, 2]), np.ones(4))
    _, Cn, _ = O.capacitance(ps, rtol=1e-11)
    assert np.all(np.diag(Cn) > 0)
    off = Cn[~np.eye(3, dtype=bool)]
    assert np.all(off < 0)
    assert np.all(Cn.sum(1) > 0)
    assert np.linalg.norm(Cn - Cn.T) < 1e-2 * np.linalg.norm(Cn)


def test_dielectric_limits():
    """Eq. 7 limits: a coating of eps_r -> infinity makes the coated conductor
    behave as the larger conductor (the dielectric rows force a constant
    potential on the coating surface); eps_r = 1 removes every dielectric panel."""
    big = O.panels(np.zeros((4, 4, 4), np.int32), np.array([0]), np.array([1.0]))
    _, Cbig, _ = O.capacitance(big, rtol=1e-11)
    lab = np.zeros((4, 4, 4), np.int32)
    lab[1:3, 1:3, 1:3] = 1
    coat = O.panels(lab, np.array([-1, 0]), np.array([1e7, 1.0]))
    _, Cc, _ = O.capacitance(coat, rtol=1e-11)
    # the continuum limit is exact; the discrete dielectric rows (a normal-
    # derivative condition) and conductor rows (a potential condition) agree
    # to discretisation error only
    assert abs(Cc[0, 0] - Cbig[0, 0]) < 0.03 * Cbig[0, 0]
    coat4 = O.panels(lab, np.array([-1, 0]), np.array([1e4, 1.0]))
    _, Cc4, _ = O.capacitance(coat4, rtol=1e-11)
    assert abs(Cc4[0, 0] - Cc[0, 0]) < 1e-3 * Cc[0, 0]     # the limit is reached
    plain = O.panels(lab, np.array([-1, 0]), np.array([1.0, 1.0]))
    assert plain.n_diel == 0
    # a dielectric coating raises the capacitance monotonically with eps_r
    prev = O.capacitance(plain, rtol=1e-11)[1][0, 0]
    for e in (2.0, 4.0, 16.0):
        cur = O.capacitance(O.panels(lab, np.array([-1, 0]), np.array([e, 1.0])), rtol=1e-11)[1][0, 0]
        assert cur > prev
        prev = cur


def test_coated_sphere_analytic():
    """Sec. III.A: C = 4 pi eps0 eps_r r_d r_c / ((r_d - r_c) + eps_r r_c)
    for the coated sphere; at dv = 0.05 m the staircase error is a few %."""
    w = W.coated_sphere(20, 2.0)
    ps = O.panels(w.labels, w.conductor_id, w.eps_r)
    C, _, _ = O.capacitance(ps, voxel_size=w.voxel_size, rtol=1e-10)
    rc, rd, er = 0.25, 0.5, 2.0
    ref = 4 * math.pi * O.EPS0 * er * rd * rc / ((rd - rc) + er * rc)
    assert abs(C[0, 0] - ref) < 0.05 * ref


def test_preconditioner_blocks_invert_their_boxes():
    """Eq. 14: R A restricted to a small box's conductor panels is the
    identity; dielectric rows are scaled by 1/I'."""
    lab = np.zeros((8, 16, 16), np.int32)
    lab[3:5, 2:14, 2:14] = 1
    lab[1:3, 2:14, 2:14] = 2
    lab[5:7, 2:14, 2:14] = 3
    ps = O.panels(lab, np.array([-1, -1, 0, 1]), np.array([1.0, 3.9, 1, 1]))
    A = O.dense_matrix(ps, rtol=1e-10)
    R = O.precond_matrix(ps, A, nv=5, kind="bdd")
    RA = R @ A
    box = O.panel_boxes(ps, 5)
    cond = ps.kind == 0
    for b in np.unique(box[cond]):
        S = np.nonzero(cond & (box == b))[0]
        assert np.allclose(RA[np.ix_(S, S)], np.eye(len(S)), atol=1e-10)
    diel = np.nonzero(~cond)[0]
    # A_kk = I'_k + E'_kk with E'_kk = 0 (principal value), so (R A)_kk = 1
    assert np.allclose(np.diag(RA)[diel], 1.0, atol=1e-12)
    assert O.unique_box_patterns(ps, 5) >= 1


@pytest.mark.parametrize("nx,ny,expect_boxes,expect_unique", [(20, 5, 4, 3), (20, 20, 16, 9)])
def test_unique_box_patterns_hand_counted(nx, ny, expect_boxes, expect_unique):
    """Sec. II.D (ii): a full conductor slab nx x ny x 1, boxes of 5 voxels.

    Panels: x-faces at i = 0 and i = nx, y-faces at j = 0 and j = ny, z-faces
    at k = 0 and k = 1 over the whole slab.  A face on the far boundary of its
    own axis (i = nx, j = ny, k = 1) joins the last box along that axis.  Along
    x the boxes fall into three classes: the first holds the i = 0 x-faces at
    local x 0, the last holds the i = nx x-faces at local x 5, the middle ones
    hold none; the same three classes along y (when ny > 5).  z-faces and the
    z extent are identical in every box.  So a 4 x 1 row of boxes has the
    patterns {first, middle, middle, last}: 3 unique; a 4 x 4 array has
    3 x 3 = 9 unique patterns among its 16 boxes."""
    lab = np.zeros((1, ny, nx), np.int32)
    ps = O.panels(lab, np.array([0]), np.array([1.0]))
    assert ps.n == 2 * ny + 2 * nx + 2 * nx * ny
    box = O.panel_boxes(ps, 5)
    assert len(np.unique(box)) == expect_boxes
    assert O.unique_box_patterns(ps, 5) == expect_unique


def _three_panel_set():
    """Three z-normal panels on a 10 x 5 x 1 grid: panel 0 at z-face (1,1,0)
    and panel 1 at (3,2,1) lie in box 0 (x in [0,5)), panel 2 at (7,0,0) in
    box 1; panel 1 is a dielectric row with I' = 2.5."""
    fx, fy = 10, 5                                   # z-face grid is 10 x 5 x 2
    face = np.array([1 + fx * (1 + fy * 0), 3 + fx * (2 + fy * 1), 7 + fx * (0 + fy * 0)], np.int32)
    n = 3
    ps = O.PanelSet(10, 5, 1, np.full(n, 2, np.int8), face, np.array([0, 1, 0], np.int8),
                    np.array([0, -1, 0], np.int16), np.array([0.0, 2.5, 0.0]), np.array([1.0, 0.0, 1.0]),
                    np.zeros(n, np.int32), np.zeros(n, np.int32), 1, centers=np.zeros((n, 3)))
    A = np.array([[2.0, 1.0, 0.5], [1.0, 4.0, 1.0], [0.5, 1.0, 8.0]])
    return ps, A


def test_preconditioner_variants_by_hand():
    """Eq. 14 and the conventional preconditioners of Sec. III.A on a
    three-panel case worked by hand (A = [[2,1,.5],[1,4,1],[.5,1,8]]):
    diag = diag(1/2, 1/4, 1/8); bd = inv([[2,1],[1,4]]) = [[4,-1],[-1,2]]/7 on
    box 0 and 1/8 on box 1; bdd = 1/2 and 1/8 on the conductor rows (each
    alone in its box) and 1/I' = 0.4 on the dielectric row; none = I."""
    ps, A = _three_panel_set()
    assert list(O.panel_boxes(ps, 5)) == [0, 0, 1]
    np.testing.assert_allclose(O.precond_matrix(ps, A, 5, "diag"), np.diag([0.5, 0.25, 0.125]),
                               rtol=0, atol=1e-15)
    bd = np.array([[4 / 7, -1 / 7, 0], [-1 / 7, 2 / 7, 0], [0, 0, 1 / 8]])
    np.testing.assert_allclose(O.precond_matrix(ps, A, 5, "bd"), bd, rtol=0, atol=1e-15)
    np.testing.assert_allclose(O.precond_matrix(ps, A, 5, "bdd"), np.diag([0.5, 0.4, 0.125]),
                               rtol=0, atol=1e-15)
    np.testing.assert_array_equal(O.precond_matrix(ps, A, 5, "none"), np.eye(3))


def test_oracle_gradient_matches_finite_differences():
    """The oracle's adjoint dC/d(eps) against central differences of its own
    capacitance (step 1e-4) on a tiny grid with distinct permittivities."""
    rng = np.random.default_rng(3)
    n = 4
    lab = np.arange(n ** 3, dtype=np.int32).reshape(n, n, n)
    lab[1:3, 1:3, 0:2] = n ** 3
    cid = np.full(n ** 3 + 1, -1, np.int32)
    cid[-1] = 0
    eps = np.concatenate([1.5 + rng.random(n ** 3), [1.0]])
    G = np.array([[1.0]])
    g, C = O.capacitance_grad(lab, cid, eps, G, rtol=1e-12)
    for v in rng.choice(np.unique(lab[lab < n ** 3]), 6, replace=False):
        ep, em = eps.copy(), eps.copy()
        h = 1e-4
        ep[v] += h
        em[v] -= h
        Cp = O.capacitance(O.panels(lab, cid, ep), rtol=1e-12)[0][0, 0]
        Cm = O.capacitance(O.panels(lab, cid, em), rtol=1e-12)[0][0, 0]
        fd = (Cp - Cm) / (2 * h)
        assert abs(fd - g[v]) < 1e-3 * abs(g).max(), (v, fd, g[v])


def test_equal_eps_faces_hand_counted():
    """Faces between equal permittivities carry no panel: two voxels of eps 3
    share one such face (the interior x-face); at eps 1 all 11 faces of the
    pair are, the 10 boundary faces included (vacuum outside); a conductor
    side never counts."""
    lab = np.zeros((1, 1, 2), np.int32)
    ef = O.equal_eps_faces(lab, np.array([-1]), np.array([3.0]))
    assert len(ef["orient"]) == 1 and ef["orient"][0] == 0 and ef["face"][0] == 1
    assert ef["label_a"][0] == 0 and ef["label_b"][0] == 0
    np.testing.assert_array_equal(ef["center"][0], [1.0, 0.5, 0.5])
    ef = O.equal_eps_faces(lab, np.array([-1]), np.array([1.0]))
    assert len(ef["orient"]) == 11
    assert sorted(np.bincount(ef["orient"], minlength=3)) == [3, 4, 4]
    assert np.count_nonzero((ef["label_a"] < 0) | (ef["label_b"] < 0)) == 10
    lab2 = np.array([[[0, 1]]], np.int32)
    ef = O.equal_eps_faces(lab2, np.array([-1, 0]), np.array([1.0, 1.0]))
    assert len(ef["orient"]) == 5 and np.all(ef["label_a"] != 1) and np.all(ef["label_b"] != 1)


def test_oracle_gradient_at_equal_permittivity_faces():
    """Voxels whose faces join equal permittivities (no panel there): the
    oracle's adjoint gradient, which adds the limit of Eq. 7 for those faces,
    against central differences of its own capacitance (step 1e-4).  Without
    that term the two disagree by up to several times the gradient."""
    rng = np.random.default_rng(1)
    nx, ny, nz = 5, 4, 3
    nv = nx * ny * nz
    lab = np.arange(nv, dtype=np.int32).reshape(nz, ny, nx)
    lab[0:2, 0:2, 0:2] = nv
    lab[1:3, 2:4, 3:5] = nv + 1
    cid = np.full(nv + 2, -1, np.int32)
    cid[nv], cid[nv + 1] = 0, 1
    eps = np.concatenate([1.5 + 4 * rng.random(nv), [1.0, 1.0]])
    eps[: nv // 2] = 3.0                      # half of the voxels share one value
    G = np.array([[0.3, 1.0], [0.0, -0.5]])
    g, _ = O.capacitance_grad(lab, cid, eps, G, rtol=1e-12)
    free = [v for v in range(nv) if np.any(lab == v)]
    picks = [v for v in free if v < nv // 2][:4] + [v for v in free if v >= nv // 2][:2]
    h = 1e-4
    for v in picks:
        ep, em = eps.copy(), eps.copy()
        ep[v] += h
        em[v] -= h
        Cp = O.capacitance(O.panels(lab, cid, ep), rtol=1e-12)[0]
        Cm = O.capacitance(O.panels(lab, cid, em), rtol=1e-12)[0]
        fd = float(np.sum(G * (Cp - Cm))) / (2 * h)
        assert abs(fd - g[v]) <= 1e-6 * abs(fd) + 1e-9 * np.max(np.abs(g)), (v, fd, g[v])


def test_tucker_roundtrip():
    """Eq. 13: with full ranks the restore reproduces the tensor; truncated,
    the Frobenius error stays within tol."""
    rng = np.random.default_rng(5)
    x = np.arange(12)[:, None, None] + 0.5
    y = np.arange(10)[None, :, None] + 0.5
    z = np.arange(6)[None, None, :] + 0.5
    X = 1.0 / np.sqrt(x * x + y * y + z * z) + 1e-3 * rng.standard_normal((12, 10, 6))
    S, U1, U2, U3 = O.tucker_hosvd(X, 0.0)
    assert np.allclose(O.tucker_expand(S, U1, U2, U3), X, rtol=0, atol=1e-12)
    for tol in (1e-2, 1e-4):
        S, U1, U2, U3 = O.tucker_hosvd(X, tol)
        err = np.linalg.norm(O.tucker_expand(S, U1, U2, U3) - X)
        assert err <= tol * np.linalg.norm(X) * (1 + 1e-9)
