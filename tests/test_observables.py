"""Susceptibilities from K1 (observables), on the oracle's vertices (CPU): at second order
they are the textbook bare bubbles (χ_± = χ_c = −Π_ph/2, χ_pair = Π_pp/2) with the bosonic
FDR; at first order in U they are the ladders χ0 ± U χ0² (transverse spin enhanced, pairing
and charge suppressed by a repulsive U)."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2405_20996_gb300.observables import charge_susceptibility_from_K1, susceptibility_from_K1
from test_oracle_pins import pi_R_ph, pi_R_pp

CLS = ("K1", "K2", "K2p", "K3")


def test_second_order_is_the_bare_bubble_with_the_fdr():
    g = dict(n1=31, n2w=9, n2v=9, n3w=7, n3v=7)
    U, D, T = 0.7, 1.0, 0.1
    V = O.Vertex(g, U=U, has_R=True)
    P = O.Prop(Delta=D, T=T)
    w = O.grid(g["n1"])
    for r, ref_of in ((0, lambda om: -pi_R_ph(om, D, T) / 2), (1, lambda om: pi_R_pp(om, D, T) / 2)):
        chiR, chiK = susceptibility_from_K1(O.bubble_class(V, V, P, r, "K1", 1001), r, U)
        for i in (4, 11, 15, 20, 27):
            ref = ref_of(w[i])
            assert abs(chiR[i] - ref) <= 1e-9 * abs(ref), (r, w[i], chiR[i], ref)
            # bosonic FDR: chi^K = coth(w/2T) (chi^R - chi^A), chi^A = (chi^R)*
            assert abs(np.tanh(w[i] / (2 * T)) * chiK[i] - (chiR[i] - np.conj(chiR[i]))) <= 1e-9 * abs(ref)
        assert chiR[15].real > 0                                   # static limit positive
    Ka = O.bubble_class(V, V, P, 0, "K1", 1001)
    chiR, chiK = charge_susceptibility_from_K1(O.bubble_class(V, V, P, 2, "K1", 1001), Ka, U)
    for i in (4, 11, 15, 20, 27):
        ref = -pi_R_ph(w[i], D, T) / 2
        assert abs(chiR[i] - ref) <= 1e-9 * abs(ref), (w[i], chiR[i], ref)
        assert abs(np.tanh(w[i] / (2 * T)) * chiK[i] - (chiR[i] - np.conj(chiR[i]))) <= 1e-9 * abs(ref)


def test_first_order_is_the_ladder():
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
    cases = [(lambda s, U, r=r: susceptibility_from_K1(s[r][0], r, U)[0][w0].real, sign, chi0)
             for r, sign, chi0 in ((0, 1.0, -pi_R_ph(0.0, D, T).real / 2), (1, -1.0, pi_R_pp(0.0, D, T).real / 2))]
    cases.append((lambda s, U: charge_susceptibility_from_K1(s[2][0], s[0][0], U)[0][w0].real, -1.0,
                  -pi_R_ph(0.0, D, T).real / 2))
    for r, (get, sign, chi0) in enumerate(cases):
        chi = np.array([get(s, U) for s, U in zip(sols, Us)])
        c2, c1, c0 = np.polyfit(Us, chi, 2)
        assert abs(c0 / chi0 - 1) <= 1e-3, (r, c0, chi0)
        assert abs(c1 / (sign * chi0 ** 2) - 1) <= 2e-3, (r, c1, sign * chi0 ** 2)


def test_rejects_the_t_channel_and_zero_coupling():
    K1 = np.zeros((5, 16), dtype=np.complex128)
    with pytest.raises(ValueError):
        susceptibility_from_K1(K1, 2, 1.0)
    with pytest.raises(ValueError):
        susceptibility_from_K1(K1, 0, 0.0)
