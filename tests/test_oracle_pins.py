"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test states what it pins.  None of them re-derives the oracle's own formula:
they use closed forms, an independent adaptive quadrature (QUADPACK) on the real
frequency axis, physical relations (causality, fluctuation-dissipation, conjugation
and crossing symmetry), exactness properties, and a brute-force evaluation of the
general leg-index bubble formula with explicit spin sums.
"""

import os

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import oracle as O
import seeded as S

G_TINY = dict(n1=11, n2w=7, n2v=7, n3w=5, n3v=5)
G_SMALL = dict(n1=31, n2w=9, n2v=9, n3w=7, n3v=7)


def _blocks(r):
    """Parity blocks of a K1 4x4 matrix: (row pair, col pair) parities per component.
    a: rows (a1', a2), cols (a2', a1); p: rows (a1', a2'), cols (a1, a2)."""
    out = {}
    for c in range(16):
        b1p, b2p, b1, b2 = (c >> 3) & 1, (c >> 2) & 1, (c >> 1) & 1, c & 1
        if r == 0:
            key = ((b1p + b2) % 2, (b2p + b1) % 2)
        else:
            key = ((b1p + b2p) % 2, (b1 + b2) % 2)
        out.setdefault(key, []).append(c)
    return out


def _quad_c(f, a=-np.inf, b=np.inf, **kw):
    re = quad(lambda e: f(e).real, a, b, epsabs=1e-15, epsrel=1e-13, limit=800, **kw)[0]
    im = quad(lambda e: f(e).imag, a, b, epsabs=1e-15, epsrel=1e-13, limit=800, **kw)[0]
    return re + 1j * im


def _spec(e, D):
    return D / np.pi / (e * e + D * D)


def pi_R_ph(om, D, T):
    """Retarded particle-hole bubble of G^R = 1/(v + i D) with the dv/(2 pi i) measure:
    -int de A(e) tanh(e/2T) [1/(e - w - iD) + 1/(e + w + iD)] (real-axis QUADPACK)."""
    return _quad_c(lambda e: -_spec(e, D) * np.tanh(e / (2 * T)) * (1 / (e - om - 1j * D) + 1 / (e + om + 1j * D)))


def pi_R_pp(om, D, T):
    """Retarded particle-particle bubble: int dv/(2 pi i) [G^K(w/2+v) G^R(w/2-v) + G^R G^K],
    written with e = w/2 + v as -int de A(e) tanh(e/2T) * 2 / (w - e + iD)."""
    return _quad_c(lambda e: -_spec(e, D) * np.tanh(e / (2 * T)) * 2.0 / (om - e + 1j * D))


@pytest.mark.parametrize("r", [0, 1])
def test_pt2_k1_matches_independent_bubble(r):
    """PT2 (Sec. III.A.2): B_r(Gamma0, Gamma0) has only K1; its retarded parity block is
    (U/2)^2 times the textbook retarded bubble computed by QUADPACK on the real axis;
    the all-classical block vanishes (causality); FDR and conjugation relate the rest."""
    U, D, T = 1.0, 1.0, 0.1
    V = O.Vertex(G_SMALL, U=U, has_R=True)
    P = O.Prop(Delta=D, T=T)
    B = O.bubble_class(V, V, P, r, "K1", 1001)
    w = O.grid(G_SMALL["n1"])
    bl = _blocks(r)
    ee, eo, oe, oo = bl[(0, 0)], bl[(0, 1)], bl[(1, 0)], bl[(1, 1)]
    for i in (3, 9, 15, 18, 24):
        om = w[i]
        ref = (U / 2) ** 2 * (pi_R_ph(om, D, T) if r == 0 else pi_R_pp(om, D, T))
        # every component of a parity block is the same number (Gamma0 depends on parity only)
        for blk in (eo, oe, oo):
            assert np.allclose(B[i, blk], B[i, blk[0]], rtol=0, atol=1e-15)
        Rt, Ad, Kd = B[i, oe[0]], B[i, eo[0]], B[i, oo[0]]
        assert abs(Rt - ref) <= 1e-9 * abs(ref), (om, Rt, ref)
        assert np.abs(B[i, ee]).max() <= 1e-12 * abs(ref)                       # causality
        assert abs(Ad - np.conj(Rt)) <= 1e-13 * abs(ref)                        # K1^A = (K1^R)*
        # bosonic FDR: K1^K = coth(w/2T) (K1^R - K1^A)  (Sec. II.E.2, K1 relation)
        assert abs(np.tanh(om / (2 * T)) * Kd - (Rt - Ad)) <= 1e-9 * abs(ref)
        # the printed form: Im K1^R = -(i/2) tanh(w/2T) K1^K
        assert abs(Rt.imag - (-0.5j * np.tanh(om / (2 * T)) * Kd).real) <= 1e-9 * abs(ref)


def test_pt2_structure_and_t_channel_zero():
    """Bare x bare bubble: only K1 survives (K2, K2', K3 exactly 0); the t-channel up-down
    PT2 bubble vanishes exactly because Gamma0^{upup} = 0."""
    V = O.Vertex(G_TINY, U=2.0, has_R=True)
    P = O.Prop(Delta=1.0, T=0.05)
    for r in range(3):
        B = O.bubble_all(V, V, P, r, 201)
        for c in ("K2", "K2p", "K3"):
            assert np.abs(B[c]).max() == 0.0
        if r == 2:
            assert np.abs(B["K1"]).max() == 0.0
        else:
            assert np.abs(B["K1"]).max() > 1e-3


def test_pt2_t_channel_upup_by_crossing():
    """Crossing of the PT2 vertex: the up-up vertex Gamma(1'2'|12) - Gamma(1'2'|21) of
    a + p bubbles.  The t-channel bubble of Gamma0 with the up-up spin sum (computed by
    the brute-force general formula below) must equal minus the exchanged a-bubble."""
    D, T, U = 1.0, 0.1, 1.0
    V = O.Vertex(G_TINY, U=U, has_R=True)
    P = O.Prop(Delta=D, T=T)
    om, v, vp = 0.7, -0.4, 1.3
    x = np.linspace(-0.97, 0.97, 9)
    # brute force t-bubble of the up-up component at t-variables (om, v, vp)
    bt = np.array([_brute_integrand(V, V, P, 2, om, v, vp, xi, spins=(0, 0, 0, 0)) for xi in x])
    # exchanged a-bubble: legs of t-variables, exchange 1<->2, a-variables of that
    L = _legs(2, om, v, vp)
    Ls = [L[0], L[1], L[3], L[2]]
    wa, va, vpa = _chan(0, Ls)
    ba = O.integrand(V, V, P, 0, O.SEL_FULL, O.SEL_FULL, wa, va, vpa, x)
    perm = [8 * ((c >> 3) & 1) + 4 * ((c >> 2) & 1) + 2 * (c & 1) + ((c >> 1) & 1) for c in range(16)]
    # the exchanged a-diagram integrates over the same v'' with the same measure
    assert np.allclose(bt, -ba[:, perm], rtol=0, atol=1e-14 * np.abs(ba).max())


@pytest.mark.parametrize("r", [0, 1, 2])
def test_conjugation_and_crossing_of_seeded_bubble(r):
    """The 1-loop bubble of a conjugation- and crossing-symmetric vertex inherits both
    symmetries (Sec. II.G.3) exactly (roundoff), for every class."""
    V = O.Vertex(G_TINY, U=1.0, has_R=True, channels=S.seeded_vertex(G_TINY, 1.0, seed=7))
    P = O.Prop(Delta=1.0, T=0.1)
    B = O.bubble_all(V, V, P, r, 201)
    cls = (B["K1"], B["K2"], B["K2p"], B["K3"])
    sc = max(np.abs(a).max() for a in cls)
    for a, b in zip(cls, S.conj_image(r, cls)):
        assert np.abs(a - b).max() <= 1e-13 * sc
    for a, b in zip(cls, S.cross_image(r, cls)):
        assert np.abs(a - b).max() <= 1e-13 * sc


@pytest.mark.parametrize("r", [0, 1, 2])
def test_class_split_sums_to_unsplit(r):
    """K1 + K2 + K2' + K3 at one (w, v, v') equals the contraction of the full vertices
    (linearity of the class split, Sec. II.C.1)."""
    V = O.Vertex(G_TINY, U=1.0, has_R=True, channels=S.seeded_vertex(G_TINY, 1.0, seed=11))
    P = O.Prop(Delta=1.0, T=0.1)
    f = np.array([[0.3, -1.1, 2.2], [-2.0, 0.5, 0.5], [0.0, 7.0, -0.2]])
    tot = 0
    for ls, rs in O.CLASS_SEL.values():
        tot = tot + O.bubble_points(V, V, P, r, ls, rs, 201, f)
    full = O.bubble_points(V, V, P, r, O.SEL_FULL, O.SEL_FULL, 201, f)
    assert np.abs(tot - full).max() <= 1e-14 * np.abs(full).max()


def test_bilinearity():
    """B(a G + b G', G2) = a B(G, G2) + b B(G', G2) for the reducible parts."""
    g = G_TINY
    c1, c2 = S.seeded_vertex(g, 1.0, seed=1), S.seeded_vertex(g, 1.0, seed=2)
    a, b = 0.7 - 0.2j, -1.3
    mix = {c: tuple(a * x + b * y for x, y in zip(c1[c], c2[c])) for c in c1}
    V1, V2, V12 = (O.Vertex(g, channels=c) for c in (c1, c2, mix))
    W = O.Vertex(g, U=1.0, has_R=True, channels=S.seeded_vertex(g, 1.0, seed=3))
    P = O.Prop(Delta=1.0, T=0.2)
    for r in range(3):
        B1, B2, B12 = (O.bubble_all(X, W, P, r, 101) for X in (V1, V2, V12))
        for k in B1:
            ref = a * B1[k] + b * B2[k]
            assert np.abs(B12[k] - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1e-30)


def test_interpolation_exact_at_nodes_and_linear_in_x():
    """linear_on_aux interpolation (Sec. II.G.7): exact at grid nodes, exact for data
    linear in x between nodes, and zero at v = +-inf."""
    g = G_TINY
    z = lambda shp: np.zeros(shp, dtype=complex)
    n = g["n3v"]
    xg = -1 + 2 * (np.arange(n) + 1) / (n + 1)
    wx = -1 + 2 * (np.arange(g["n3w"]) + 1) / (g["n3w"] + 1)
    K3 = (1.0 + 2.0 * wx[:, None, None] - 0.5 * xg[None, :, None] + 3.0 * xg[None, None, :])[..., None] \
        * np.arange(1, 17)[None, None, None, :]
    ch = {0: (z((g["n1"], 16)), z((g["n2w"], g["n2v"], 16)), z((g["n2w"], g["n2v"], 16)), K3.astype(complex))}
    V = O.Vertex(g, channels=ch)
    w3, v3 = O.grid(g["n3w"]), O.grid(n)
    # nodes
    f = np.array([[w3[1], v3[2], v3[4]], [w3[3], v3[0], v3[1]]])
    got = O.vertex_eval(V, 0, 0, 0, O.SEL_FULL, f)
    assert np.allclose(got[0], K3[1, 2, 4], rtol=1e-14)
    assert np.allclose(got[1], K3[3, 0, 1], rtol=1e-14)
    # between nodes (inside the grid), data linear in x is reproduced
    xs = np.array([[wx[1] * 0.3 + wx[2] * 0.7, xg[3] * 0.5 + xg[4] * 0.5, xg[0] * 0.9 + xg[1] * 0.1]])
    f = 5.0 * np.tan(np.pi * xs / 2)
    got = O.vertex_eval(V, 0, 0, 0, O.SEL_FULL, f)
    ref = (1.0 + 2.0 * xs[0, 0] - 0.5 * xs[0, 1] + 3.0 * xs[0, 2]) * np.arange(1, 17)
    assert np.allclose(got[0], ref, rtol=1e-12)
    # beyond the last node the class decays linearly in x to zero at x = 1
    got = O.vertex_eval(V, 0, 0, 0, O.SEL_FULL, np.array([[w3[1], v3[2], np.inf]]))
    assert np.abs(got).max() == 0.0


def test_gl5_rule_exactness():
    """Composite 5-point Gauss-Lobatto: sum of weights 2; exact for piecewise polynomials
    of degree <= 7 on each panel; endpoints included (Sec. II.G.5 rule family)."""
    for Nq in (5, 21, 1001):
        x, w = O.gl5_rule(Nq)
        assert abs(w.sum() - 2.0) < 1e-13
        assert x[0] == -1.0 and x[-1] == 1.0
        for d in range(8):
            # every panel integrates polynomials of degree <= 7 exactly, hence any
            # global polynomial of that degree
            exact = 2.0 / (d + 1) if d % 2 == 0 else 0.0
            assert abs((w * (0.3 + x) ** d).sum() - ((1.3 ** (d + 1) - (-0.7) ** (d + 1)) / (d + 1))) < 1e-12, (Nq, d)
    x, w = O.gl5_rule(5)
    assert abs((w * x ** 8).sum() - 2.0 / 9) > 1e-3          # degree 8 is not exact on one panel


def test_kronrod_rules_match_printed_nodes():
    """GL4 / GLK7 / GLK13 rules derived from the nodes printed in Sec. II.G.5 (golden
    fixture): derived nodes agree with all printed digits, weights are positive, and the
    rules are exact to degrees 5, 9 and 19."""
    path = os.path.join(os.path.dirname(__file__), "golden", "gl_kronrod_nodes.txt")
    printed = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            val, rule = line.split()
            printed.setdefault(rule, []).append(float(val))
    R = O.lobatto_kronrod_rules()
    kron = sorted(set(np.round(R["x13"], 12)) - set(np.round(R["x7"], 12)))
    assert np.allclose(sorted(kron), sorted(printed["GLK13"]), atol=6e-7)
    assert np.allclose(sorted(R["x7"][R["w4"] != 0]), sorted(printed["GL4"]), atol=6e-7)
    assert np.allclose(sorted(R["x7"]), sorted(printed["GL4"] + printed["GLK7"]), atol=6e-7)
    assert (R["w13"] > 0).all() and (R["w7"] > 0).all()
    for name, xs, ws, deg in (("GL4", R["x7"], R["w4"], 5), ("GLK7", R["x7"], R["w7"], 9),
                              ("GLK13", R["x13"], R["w13"], 19)):
        for d in range(deg + 1):
            exact = 2.0 / (d + 1) if d % 2 == 0 else 0.0
            assert abs((ws * xs ** d).sum() - exact) < 1e-12, (name, d)


def test_fixed_rule_vs_adaptive_brute_force():
    """Brute force on a tiny grid: the fixed composite GL5 result agrees with the paper's
    adaptive GL4/GLK7 (GLK13 error scale) integrator at tight tolerance, and the
    agreement improves with Nq (this measures the fixed rule's quadrature error)."""
    g = dict(n1=11, n2w=7, n2v=7, n3w=5, n3v=5)
    V = O.Vertex(g, U=1.0, has_R=True, channels=S.seeded_vertex(g, 1.0, seed=5))
    P = O.Prop(Delta=1.0, T=0.5)
    r = 0
    f = O.class_freqs(g, "K3")[::17]
    ref, n = O.bubble_points_adaptive(V, V, P, r, O.SEL_NU, O.SEL_NU, f, eps=1e-11)
    assert n > 0
    errs = []
    for Nq in (201, 801, 3201):
        got = O.bubble_points(V, V, P, r, O.SEL_NU, O.SEL_NU, Nq, f)
        errs.append(np.abs(got - ref).max() / np.abs(ref).max())
    assert errs[-1] < 1e-5
    assert errs[0] > errs[1] > errs[2]


def test_propagator_sum_rule_kk_fdr():
    """G^R of the flat-band model: spectral sum rule (Sec. II.E.4), Kramers-Kronig
    (Sec. II.E.3) and the FDR G^K = 2i tanh(v/2T) Im G^R (Sec. II.E.2); also with a
    Sigma table the Dyson G satisfies the same FDR when Sigma^K obeys it."""
    P = O.Prop(Delta=1.0, T=0.1)
    A = lambda v: -O.prop_eval(P, 0, np.atleast_1d(v))[:, 0, 1].imag / np.pi
    s = quad(lambda v: A(v)[0], -np.inf, np.inf, epsabs=1e-13, limit=400)[0]
    assert abs(s - 1.0) < 1e-10
    for w0 in (-1.3, 0.2, 2.5):
        pv = quad(lambda v: -np.pi * A(v)[0], -200, 200, weight="cauchy", wvar=w0, limit=400)[0]
        tail = quad(lambda v: -np.pi * A(v)[0] / (v - w0), 200, np.inf)[0] + \
            quad(lambda v: -np.pi * A(v)[0] / (v - w0), -np.inf, -200)[0]
        re = O.prop_eval(P, 0, np.array([w0]))[0, 0, 1].real
        assert abs(re - (pv + tail) / np.pi) < 1e-8
    v = np.linspace(-7, 7, 41)
    M = O.prop_eval(P, 0, v)
    assert np.allclose(M[:, 0, 0], 2j * np.tanh(v / 0.2) * M[:, 0, 1].imag, atol=1e-15)
    assert np.allclose(M[:, 1, 0], np.conj(M[:, 0, 1])) and np.all(M[:, 1, 1] == 0)
    # with a causal Sigma table whose Keldysh part obeys the FDR
    n = 41
    sg = O.grid(n)
    sR = S.seeded_sigma(n, seed=4)
    sK = 2j * np.tanh(sg / 0.2) * sR.imag
    P2 = O.Prop(Delta=1.0, T=0.1, sigR=sR, sigK=sK)
    M = O.prop_eval(P2, 0, sg)
    assert np.allclose(M[:, 0, 0], 2j * np.tanh(sg / 0.2) * M[:, 0, 1].imag, atol=1e-14)
    # single-scale propagator of the hybridisation flow: S^R = -i (G^R)^2 = dG^R/dDelta
    Pp, Pm = O.Prop(Delta=1.0 + 1e-6, T=0.1), O.Prop(Delta=1.0 - 1e-6, T=0.1)
    Sfd = (O.prop_eval(Pp, 0, v) - O.prop_eval(Pm, 0, v)) / 2e-6
    Sm = O.prop_eval(P, 1, v)
    assert np.allclose(Sm, Sfd, atol=1e-8)


# ---------------------------------------------------------------------------------
# brute-force general formula with explicit spins (used by two pins)
# ---------------------------------------------------------------------------------
def _legs(r, w, v, vp):
    if r == 0:
        return [v + w / 2, vp - w / 2, vp + w / 2, v - w / 2]
    if r == 1:
        return [w / 2 + v, w / 2 - v, w / 2 + vp, w / 2 - vp]
    return [v - w / 2, vp + w / 2, v + w / 2, vp - w / 2]


def _chan(r, L):
    if r == 0:
        return L[0] - L[3], (L[0] + L[3]) / 2, (L[2] + L[1]) / 2
    if r == 1:
        return L[0] + L[1], (L[0] - L[1]) / 2, (L[2] - L[3]) / 2
    return L[1] - L[3], (L[0] + L[2]) / 2, (L[1] + L[3]) / 2


def _gamma_ud(V, L):
    """Full up-down vertex at legs L (any parametrisation: use a-variables)."""
    return O.vertex_eval(V, 0, 0, 0, O.SEL_FULL, np.array([_chan(0, L)]))[0]


def _kswap12(vec):
    return vec[[8 * ((c >> 3) & 1) + 4 * ((c >> 2) & 1) + 2 * (c & 1) + ((c >> 1) & 1) for c in range(16)]]


def _gamma_spin(V, L, s):
    """Vertex component with spins s = (s1', s2', s1, s2) (0 up, 1 down) from the up-down
    one by SU(2) and crossing (Sec. II.G.3)."""
    s1p, s2p, s1, s2 = s
    Ls = [L[0], L[1], L[3], L[2]]
    if s1p == s1 and s2p == s2:
        if s1p != s2p:
            return _gamma_ud(V, L)
        return _gamma_ud(V, L) - _kswap12(_gamma_ud(V, Ls))
    if s1p == s2 and s2p == s1 and s1p != s2p:
        return -_kswap12(_gamma_ud(V, Ls))
    return np.zeros(16, dtype=complex)


def _brute_integrand(V1, V2, P, r, w, v, vp, x, spins=(0, 1, 0, 1)):
    """J(x) * sum over internal spins and Keldysh indices of the general bubble formula
    a: I(1'4'|32) G(3|3') G(4|4') G(3'2'|14); p: 1/2 I(1'2'|34) G G G(3'4'|12);
    t: -I(4'2'|32) G G G(1'3'|14) (internal legs 3, 4; G diagonal in spin)."""
    A = 5.0
    nu = A * np.tan(np.pi * x / 2)
    J = A * np.pi / 2 / np.cos(np.pi * x / 2) ** 2
    l1p, l2p, l1, l2 = _legs(r, w, v, vp)
    s1p, s2p, s1, s2 = spins
    if r == 1:
        n3, n4 = w / 2 + nu, w / 2 - nu
    else:
        n3, n4 = nu + w / 2, nu - w / 2
    G3 = O.prop_eval(P, 0, np.array([n3]))[0]
    G4 = O.prop_eval(P, 0, np.array([n4]))[0]
    out = np.zeros(16, dtype=complex)
    for s3 in (0, 1):
        for s4 in (0, 1):
            if r == 0:
                Lv = _gamma_spin(V1, [l1p, n4, n3, l2], (s1p, s4, s3, s2))
                Rv = _gamma_spin(V2, [n3, l2p, l1, n4], (s3, s2p, s1, s4))
            elif r == 1:
                Lv = _gamma_spin(V1, [l1p, l2p, n3, n4], (s1p, s2p, s3, s4))
                Rv = _gamma_spin(V2, [n3, n4, l1, l2], (s3, s4, s1, s2))
            else:
                # Gamma1 is the vertex on the external legs 1', 1 (it carries v),
                # Gamma2 the one on legs 2', 2 (it carries v')
                Lv = _gamma_spin(V1, [l1p, n3, l1, n4], (s1p, s3, s1, s4))   # (1'3'|14)
                Rv = _gamma_spin(V2, [n4, l2p, n3, l2], (s4, s2p, s3, s2))   # (4'2'|32)
            for o in range(16):
                a1p, a2p, a1, a2 = (o >> 3) & 1, (o >> 2) & 1, (o >> 1) & 1, o & 1
                acc = 0
                for b3 in (0, 1):
                    for b3p in (0, 1):
                        for b4 in (0, 1):
                            for b4p in (0, 1):
                                g = G3[b3, b3p] * G4[b4, b4p]
                                if g == 0:
                                    continue
                                if r == 0:
                                    li = 8 * a1p + 4 * b4p + 2 * b3 + a2
                                    ri = 8 * b3p + 4 * a2p + 2 * a1 + b4
                                    acc += Lv[li] * g * Rv[ri]
                                elif r == 1:
                                    li = 8 * a1p + 4 * a2p + 2 * b3 + b4
                                    ri = 8 * b3p + 4 * b4p + 2 * a1 + a2
                                    acc += Lv[li] * g * Rv[ri]
                                else:
                                    ii = 8 * b4p + 4 * a2p + 2 * b3 + a2    # (4'2'|32)
                                    gi = 8 * a1p + 4 * b3p + 2 * a1 + b4    # (1'3'|14)
                                    acc += Lv[gi] * g * Rv[ii]
                out[o] += acc
    pref = {0: 1.0, 1: 0.5, 2: -1.0}[r]
    return pref * J * out


@pytest.mark.parametrize("r", [0, 1, 2])
def test_channel_form_equals_general_spin_formula(r):
    """The channel/spin-reduced integrand of the oracle equals the general leg-index
    formula with explicit internal spin sums (SU(2) + crossing for the spin components).
    For p the two spin terms are equal after v'' -> -v'', so the +-v'' pair is compared."""
    g = G_TINY
    ch = S.seeded_vertex(g, 1.0, seed=13)
    V1 = O.Vertex(g, U=1.0, has_R=True, channels=ch)
    ch2 = S.seeded_vertex(g, 1.0, seed=14)
    V2 = O.Vertex(g, U=1.0, has_R=True, channels=ch2)
    P = O.Prop(Delta=1.0, T=0.1)
    w, v, vp = 0.9, -0.3, 1.7
    xs = np.array([-0.8, -0.35, 0.05, 0.4, 0.77])
    orc = O.integrand(V1, V2, P, r, O.SEL_FULL, O.SEL_FULL, w, v, vp, xs) * (1.0 if r != 2 else -1.0)
    bru = np.array([_brute_integrand(V1, V2, P, r, w, v, vp, x) for x in xs])
    if r == 1:
        orc = orc + (O.integrand(V1, V2, P, r, O.SEL_FULL, O.SEL_FULL, w, v, vp, -xs))
        bru = bru + np.array([_brute_integrand(V1, V2, P, r, w, v, vp, -x) for x in xs])
    assert np.allclose(orc, bru, rtol=0, atol=1e-13 * np.abs(bru).max())


def test_quadrature_convergence_smooth_integrand():
    """Grid convergence: the PT2 bubble's integrand is smooth in x, so the fixed-rule error
    falls monotonically with Nq and quickly once the peaks at v'' = +-w/2 (width Delta)
    are resolved by the tan-map panels; at large |w| they sit where the x-grid is
    coarse, which is why the paper prefers an adaptive rule (Sec. II.G.5)."""
    V = O.Vertex(G_SMALL, U=1.0, has_R=True)
    P = O.Prop(Delta=1.0, T=0.1)
    f = O.class_freqs(G_SMALL, "K1")[::5]
    ref = O.bubble_points(V, V, P, 0, O.SEL_ZERO, O.SEL_ZERO, 8001, f)
    sc = np.abs(ref).max()
    e = [np.abs(O.bubble_points(V, V, P, 0, O.SEL_ZERO, O.SEL_ZERO, n, f) - ref).max() / sc
         for n in (101, 401, 1601, 3201)]
    assert e[0] > e[1] > e[2] > e[3]
    assert e[3] < 1e-5 and e[2] < 1e-3


@pytest.mark.parametrize("r", [0, 1, 2])
def test_multiloop_left_part_has_no_k1_k2p(r):
    """Multiloop left correction gamma-dot_rbar o Pi o Gamma (Sec. III.C): its left vertex
    is the sum over the channels other than r, so no part of it is r-reducible with bare
    legs on the left: the output has no K1 and no K2' class.  In the t channel this needs
    the up-up component built channel by channel (crossing partner a <-> t)."""
    g = G_TINY
    dot = S.seeded_vertex(g, 0.5, seed=4)
    inc = tuple(c for c in range(3) if c != r)
    Vd = O.Vertex(g, channels=dot, include=inc)
    V = O.Vertex(g, U=1.0, has_R=True, channels=S.seeded_vertex(g, 1.0, seed=5))
    P = O.Prop(Delta=1.0, T=0.1)
    B = O.bubble_all(Vd, V, P, r, 101, pi_kind=O.PI_GG)
    assert np.abs(B["K1"]).max() == 0.0 and np.abs(B["K2p"]).max() == 0.0
    assert np.abs(B["K2"]).max() > 0 and np.abs(B["K3"]).max() > 0
    # right correction Gamma o Pi o gamma-dot_rbar: no K1 and no K2
    B = O.bubble_all(V, Vd, P, r, 101)
    assert np.abs(B["K1"]).max() == 0.0 and np.abs(B["K2"]).max() == 0.0


def test_third_order_k1_is_the_ladder_of_a_repulsive_coupling():
    """K1 of the parquet solution at w = 0 to third order in U (a fit over three small
    couplings): the third-order term is the ladder R Pi K1^(2) with R = -U/2, so its ratio to
    the second-order term is -Pi_r(0)/2 with the textbook bubbles (particle-hole for a,
    particle-particle for p) — the transverse-spin channel enhanced and the pairing channel
    suppressed, as a repulsive U requires.  The ratio is odd in the bare vertex's sign, so
    this pins that sign (C2) through the vertex alone."""
    CLS = ("K1", "K2", "K2p", "K3")
    g = dict(n1=21, n2w=7, n2v=6, n3w=5, n3v=4)
    nq, D, T = 81, 1.0, 0.2
    P = O.Prop(Delta=D, T=T)

    def parquet(U, iters=40, mix=0.7):
        gam = {c: [np.zeros(O.class_shape(g, k), dtype=np.complex128) for k in CLS] for c in range(3)}
        for _ in range(iters):
            Gam = O.Vertex(g, U=U, has_R=True, channels=gam)
            new = {r: O.bubble_all(O.Vertex(g, U=U, has_R=True, channels=gam,
                                            include=[c for c in range(3) if c != r]), Gam, P, r, nq)
                   for r in range(3)}
            gam = {c: [(1 - mix) * gam[c][k] + mix * new[c][CLS[k]] for k in range(4)] for c in range(3)}
        return gam

    Us = np.array([0.025, 0.05, 0.1])
    w0 = g["n1"] // 2
    sols = [parquet(U) for U in Us]
    for r, pi in ((0, pi_R_ph(0.0, D, T)), (1, pi_R_pp(0.0, D, T))):
        vals = np.array([s[r][0][w0][1].real / U ** 2 for s, U in zip(sols, Us)])   # component (c c|c q)
        c4, c3, c2 = np.polyfit(Us, vals, 2)
        assert abs(c3 / c2 / (-pi.real / 2) - 1) <= 2e-3, (r, c3 / c2, -pi.real / 2)


def test_parquet_classes_keep_the_bare_vertex_keldysh_structure():
    """The bare vertex depends on the parity of the quantum indices only, and the bubble passes
    that on: in the parquet solution each K1 parity block carries one number (4 distinct
    components of 16) and K2, K2' pair their components up to sign (8 distinct), K3 keeps all
    16, exactly, in every channel."""
    CLS = ("K1", "K2", "K2p", "K3")
    g = dict(n1=13, n2w=7, n2v=6, n3w=5, n3v=4)
    nq, U = 41, 1.0
    P = O.Prop(Delta=1.0, T=0.2)
    gam = {c: [np.zeros(O.class_shape(g, k), dtype=np.complex128) for k in CLS] for c in range(3)}
    for _ in range(25):
        Gam = O.Vertex(g, U=U, has_R=True, channels=gam)
        new = {r: O.bubble_all(O.Vertex(g, U=U, has_R=True, channels=gam, include=[c for c in range(3) if c != r]),
                               Gam, P, r, nq) for r in range(3)}
        gam = {c: [0.5 * gam[c][k] + 0.5 * new[c][CLS[k]] for k in range(4)] for c in range(3)}

    def distinct(X):
        X = X.reshape(-1, 16)
        tol = 1e-13 * np.abs(X).max()
        groups = []
        for c in range(16):
            if not any(min(np.abs(X[:, c] - X[:, q]).max(), np.abs(X[:, c] + X[:, q]).max()) <= tol for q in groups):
                groups.append(c)
        return len(groups)

    for r in range(3):
        assert [distinct(gam[r][k]) for k in range(4)] == [4, 8, 8, 16], r
    # the structure is exact and without signs: with each channel's leg pairs (a: (1', 2),
    # (1, 2'); p: (1', 2'), (1, 2); t: (1', 1), (2', 2)) K1 depends on the two pairs'
    # parities, K2 on the left pair and the right parity, K2' on the left parity and the
    # right pair; a plausible slip (the pairs of another channel) breaks it
    pairs = {0: ((0, 3), (2, 1)), 1: ((0, 1), (2, 3)), 2: ((0, 2), (1, 3))}

    def key(pr, k, c):
        b = ((c >> 3) & 1, (c >> 2) & 1, (c >> 1) & 1, c & 1)
        L, R = (b[pr[0][0]], b[pr[0][1]]), (b[pr[1][0]], b[pr[1][1]])
        return [((L[0] ^ L[1]), (R[0] ^ R[1])), (L, R[0] ^ R[1]), (L[0] ^ L[1], R), (L, R)][k]

    def residual(X, pr, k):
        X = X.reshape(-1, 16)
        rep = {}
        for c in range(16):
            rep.setdefault(key(pr, k, c), c)
        return max(np.abs(X[:, c] - X[:, rep[key(pr, k, c)]]).max() for c in range(16)) / np.abs(X).max()

    for r in range(3):
        for k in range(3):
            assert residual(gam[r][k], pairs[r], k) == 0.0, (r, k)
        wrong = pairs[(r + 1) % 3]
        assert max(residual(gam[r][k], wrong, k) for k in range(3)) > 1e-3, r
