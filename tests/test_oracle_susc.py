"""Pins of the oracle's leg-contraction susceptibility (oracle_susc.chi_legs):

- no vertex: the bare bubble closed at both ends, χ0, is the textbook bare susceptibility
  (−Π_ph/2 transverse spin, Π_pp/2 pairing, by an independent spectral integral);
- bare vertex Γ = R at coupling U: the chain R̂ Π R Π R̂ gives the first-order ladder
  χ = χ0 + s U χ0² (s = +1 spin, −1 pairing) exactly, up to the quadrature-level causality
  of Π (converging fast in Nq; 1e-10 at Nq = 1281);
- on a converged parquet solution the leg contraction and the K1 route (susceptibility from
  the vertex's own K1) agree to the discretisation of the vertex classes, closer on finer
  grids (the two are equivalent for a converged parquet vertex, Sec. II.E.5)."""

import numpy as np
import pytest

from oracle import oracle as O
from oracle import oracle_susc as OS
from paper_2405_20996_gb300.observables import susceptibility_from_K1
from test_oracle_pins import pi_R_ph, pi_R_pp

CLS = ("K1", "K2", "K2p", "K3")


def test_no_vertex_gives_the_bare_susceptibility():
    g = dict(n1=31, n2w=7, n2v=6, n3w=5, n3v=4)
    D, T = 1.0, 0.1
    P = O.Prop(Delta=D, T=T)
    w = O.grid(g["n1"])
    for r, ref_of in ((0, lambda om: -pi_R_ph(om, D, T) / 2), (1, lambda om: pi_R_pp(om, D, T) / 2)):
        chiR, chiK = OS.chi_legs(O.Vertex(g), P, r, 1001)
        for i in (4, 11, 15, 20, 27):
            ref = ref_of(w[i])
            assert abs(chiR[i] - ref) <= 1e-9 * abs(ref), (r, w[i], chiR[i], ref)
            assert abs(np.tanh(w[i] / (2 * T)) * chiK[i] - (chiR[i] - np.conj(chiR[i]))) <= 1e-9 * abs(ref)


@pytest.mark.parametrize("r,s", [(0, 1.0), (1, -1.0)])
def test_bare_vertex_gives_the_first_order_ladder(r, s):
    g = dict(n1=21, n2w=7, n2v=6, n3w=5, n3v=4)
    P = O.Prop(Delta=1.0, T=0.2)
    nq = 1281
    c0, _ = OS.chi_legs(O.Vertex(g), P, r, nq)
    for U in (0.3, 1.1):
        cR, _ = OS.chi_legs(O.Vertex(g, U=U, has_R=True), P, r, nq)
        ref = c0 + s * U * c0 ** 2
        assert np.abs(cR - ref).max() <= 1e-10 * np.abs(ref).max(), (U, np.abs(cR - ref).max())
    # a plausible mistake fails it: the chain without its bare bubble, or the wrong sign
    cR, _ = OS.chi_legs(O.Vertex(g, U=0.3, has_R=True), P, r, nq)
    assert np.abs(cR - (c0 - s * 0.3 * c0 ** 2)).max() > 1e-3 * np.abs(c0).max()


def _parquet(g, nq, U, P, mix=0.6, tol=1e-13, iters=300):
    gam = {c: [np.zeros(O.class_shape(g, k), dtype=np.complex128) for k in CLS] for c in range(3)}
    for _ in range(iters):
        Gam = O.Vertex(g, U=U, has_R=True, channels=gam)
        new = {r: O.bubble_all(O.Vertex(g, U=U, has_R=True, channels=gam, include=[c for c in range(3) if c != r]),
                               Gam, P, r, nq) for r in range(3)}
        change = max(np.abs(new[c][CLS[k]] - gam[c][k]).max() for c in range(3) for k in range(4))
        gam = {c: [(1 - mix) * gam[c][k] + mix * new[c][CLS[k]] for k in range(4)] for c in range(3)}
        if change <= tol:
            break
    return gam


def test_leg_contraction_agrees_with_k1_on_the_parquet_solution():
    P = O.Prop(Delta=1.0, T=0.2)
    U, nq = 1.0, 81
    dev = []
    for g in (dict(n1=21, n2w=7, n2v=6, n3w=5, n3v=4), dict(n1=21, n2w=13, n2v=13, n3w=9, n3v=9)):
        gam = _parquet(g, nq, U, P)
        V = O.Vertex(g, U=U, has_R=True, channels=gam)
        d = 0.0
        for r in (0, 1):
            cl, _ = OS.chi_legs(V, P, r, nq)
            ck, _ = susceptibility_from_K1(gam[r][0], r, U)
            d = max(d, np.abs(cl - ck).max() / np.abs(ck).max())
        dev.append(d)
    print("leg contraction vs K1 on the parquet solution: %.2e (coarse), %.2e (finer grids)" % tuple(dev))
    assert dev[0] <= 5e-3 and dev[1] < 0.7 * dev[0], dev
