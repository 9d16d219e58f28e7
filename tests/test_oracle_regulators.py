"""Pins of the oracle's flow-scheme propagators (Sec. III.C.2), independent of its code:

- S = dG/dLambda at fixed Sigma, for the hybridisation (Lambda = Delta), interaction
  (Lambda = lam) and temperature (Lambda = T) flows, against central finite differences of
  the oracle's own G in Lambda — all four Keldysh entries, with and without a Sigma table;
- the interaction flow at Sigma = 0 scales the propagator, G_lam = lam G_1, so every bubble
  with Pi = G G is lam^2 times the lam = 1 bubble, and Pi-dot = G S + S G = 2 lam G_1 G_1
  (S = G_1), tails included: exact identities of the whole integrand chain;
- the temperature flow's S^R vanishes and S^K is i Delta v |G^R|^2 / (T^2 cosh^2(v / 2T))."""

import numpy as np
import pytest

import seeded as S
from oracle import oracle as O

V = np.array([-40.0, -3.1, -0.7, -0.05, 0.0, 0.02, 0.4, 1.9, 7.5, 120.0])


def _sig(n=21):
    return S.seeded_sigma(n, seed=5, scale=0.3)


@pytest.mark.parametrize("reg,par", [(O.REG_DELTA, "Delta"), (O.REG_U, "lam"), (O.REG_T, "T")])
@pytest.mark.parametrize("with_sigma", [False, True])
def test_single_scale_is_derivative_of_G(reg, par, with_sigma):
    base = dict(Delta=0.8, T=0.2, eps=0.15, lam=0.7)
    sig = dict(sigR=_sig(), sigK=1j * np.abs(_sig()).astype(np.complex128)) if with_sigma else {}
    h = 1e-5 * base[par]

    def G(delta):
        kw = dict(base)
        kw[par] += delta
        return O.prop_eval(O.Prop(Delta=kw["Delta"], T=kw["T"], eps=kw["eps"], reg=reg, lam=kw["lam"], **sig), 0, V)

    fd = (G(h) - G(-h)) / (2 * h)
    s = O.prop_eval(O.Prop(reg=reg, **base, **sig), 1, V)
    scale = np.abs(fd).max()
    assert np.abs(s - fd).max() <= 1e-7 * scale, (reg, np.abs(s - fd).max(), scale)
    assert np.all(s[:, 1, 1] == 0)


def test_interaction_flow_scales_the_bubble():
    g = dict(n1=11, n2w=7, n2v=6, n3w=5, n3v=4)
    ch = S.seeded_vertex(g, 1.0, seed=31)
    Vx = O.Vertex(g, U=1.0, has_R=True, channels=ch)
    lam = 0.63
    P1 = O.Prop(Delta=1.0, T=0.1, reg=O.REG_U, lam=1.0)
    Pl = O.Prop(Delta=1.0, T=0.1, reg=O.REG_U, lam=lam)
    for r in range(3):
        b1 = O.bubble_all(Vx, Vx, P1, r, 41)
        bl = O.bubble_all(Vx, Vx, Pl, r, 41)
        bd = O.bubble_all(Vx, Vx, Pl, r, 41, pi_kind=O.PI_GS)
        for k in b1:
            m = np.abs(b1[k]).max()
            assert np.abs(bl[k] - lam ** 2 * b1[k]).max() <= 1e-12 * m, (r, k)
            assert np.abs(bd[k] - 2 * lam * b1[k]).max() <= 1e-12 * m, (r, k)


def test_temperature_flow_single_scale_closed_form():
    D, T = 0.9, 0.15
    s = O.prop_eval(O.Prop(Delta=D, T=T, reg=O.REG_T), 1, V)
    gr = 1.0 / (V + 1j * D)
    e = np.exp(-np.abs(V) / T)                              # sech^2(v/2T) = 4 e / (1 + e)^2
    ref = 1j * D * V * np.abs(gr) ** 2 * 4 * e / (1 + e) ** 2 / T ** 2
    assert np.all(s[:, 0, 1] == 0) and np.all(s[:, 1, 0] == 0)
    assert np.allclose(s[:, 0, 0], ref, rtol=1e-13, atol=1e-300)


@pytest.mark.parametrize("reg,par", [(O.REG_DELTA, "Delta"), (O.REG_U, "lam"), (O.REG_T, "T")])
def test_katanin_substitution_is_the_total_derivative(reg, par):
    """With Sigma(Lambda) = Sigma0 + Lambda Sigma1 the Katanin-substituted single-scale
    propagator S + G Sigma1 G is the total derivative dG/dLambda (chain rule)."""
    base = dict(Delta=0.8, T=0.2, eps=0.15, lam=0.7)
    s0R, s1R = _sig(), S.seeded_sigma(21, seed=9, scale=0.2)
    s0K, s1K = 1j * np.abs(s0R).astype(np.complex128), 0.5j * np.abs(s1R).astype(np.complex128)
    h = 1e-5 * base[par]

    def G(delta):
        kw = dict(base)
        kw[par] += delta
        lam_tot = kw[par]
        return O.prop_eval(O.Prop(Delta=kw["Delta"], T=kw["T"], eps=kw["eps"], reg=reg, lam=kw["lam"],
                                  sigR=s0R + lam_tot * s1R, sigK=s0K + lam_tot * s1K), 0, V)

    fd = (G(h) - G(-h)) / (2 * h)
    L = base[par]
    kat = O.prop_eval(O.Prop(reg=reg, **base, sigR=s0R + L * s1R, sigK=s0K + L * s1K, dsigR=s1R, dsigK=s1K), 1, V)
    assert np.abs(kat - fd).max() <= 1e-7 * np.abs(fd).max(), (reg, np.abs(kat - fd).max())


def test_no_flow_scheme_gives_the_change_of_G_along_dsigma():
    """REG_NONE (S = 0): with dSigma tables, the substituted single-scale line is the
    directional derivative of the Dyson propagator, d/de G[Sigma + e dSigma] at e = 0
    (central differences of the oracle's own G), and the Pi-dot bubble built from it is the
    derivative of the G G bubble along dSigma; without tables the line vanishes."""
    s0R, dR = _sig(), S.seeded_sigma(21, seed=13, scale=0.2)
    s0K, dK = 1j * np.abs(s0R).astype(np.complex128), 0.3j * np.abs(dR).astype(np.complex128) - 0.1 * dR
    base = dict(Delta=0.8, T=0.2, eps=0.15)
    h = 1e-5

    def G(e):
        return O.prop_eval(O.Prop(**base, sigR=s0R + e * dR, sigK=s0K + e * dK), 0, V)

    fd = (G(h) - G(-h)) / (2 * h)
    line = O.prop_eval(O.Prop(**base, reg=O.REG_NONE, sigR=s0R, sigK=s0K, dsigR=dR, dsigK=dK), 1, V)
    assert np.abs(line - fd).max() <= 1e-7 * np.abs(fd).max(), np.abs(line - fd).max()
    assert np.all(O.prop_eval(O.Prop(**base, reg=O.REG_NONE, sigR=s0R, sigK=s0K), 1, V) == 0)
    # the bubble: Pi-dot with S = G dSigma G is d/de of B(Gamma, Gamma; G G) along dSigma
    g = dict(n1=9, n2w=5, n2v=4, n3w=3, n3v=4)
    ch = S.seeded_vertex(g, 1.0, seed=21)
    Vx = O.Vertex(g, U=1.0, has_R=True, channels=ch)
    he = 1e-4

    def B(e):
        return O.bubble_all(Vx, Vx, O.Prop(**base, sigR=s0R + e * dR, sigK=s0K + e * dK), 0, 41)

    bp, bm = B(he), B(-he)
    dot = O.bubble_all(Vx, Vx, O.Prop(**base, reg=O.REG_NONE, sigR=s0R, sigK=s0K, dsigR=dR, dsigK=dK), 0, 41,
                       pi_kind=O.PI_GS)
    for name in ("K1", "K2", "K2p", "K3"):
        ref = (bp[name] - bm[name]) / (2 * he)
        assert np.abs(dot[name] - ref).max() <= 1e-6 * np.abs(ref).max(), name
