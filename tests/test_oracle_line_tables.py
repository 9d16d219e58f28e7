"""Pins of the oracle's tabulated lines (G or S given as tables instead of computed from the
model and Sigma; the bubble's propagator pair, Sec. II.C.5, and the loop's line, Sec. II.D.2),
independent of its table code:

- tables sampled from the model's own lines at the table's grid nodes reproduce those lines
  at the nodes exactly (all four Keldysh entries of G, of S, of S with the Katanin term and of
  the line with one dSigma insertion): the entry layout, the advanced part as the conjugate and
  the node positions;
- tables linear in x are read exactly at any x between nodes, and fall linearly to 0 between
  the outermost node and x = +-1 (the reading of every table of the method);
- a bubble built from tables sampled from the analytic lines converges to the bubble of the
  analytic lines at second order in the table spacing (Pi = G G and Pi-dot = G S + S G)."""

import numpy as np
import pytest

import seeded as S
from oracle import oracle as O

MODEL = dict(Delta=0.9, T=0.15, eps=0.1)


def _lines(P, v, which):
    m = O.prop_eval(P, which, v)
    return m[:, 0, 1], m[:, 0, 0]           # retarded, Keldysh


@pytest.mark.parametrize("with_sigma", [False, True])
def test_tables_sampled_at_nodes_reproduce_the_lines(with_sigma):
    sig = S.seeded_sigma(17, seed=3, scale=0.25)
    kw = dict(sigR=sig, sigK=1j * np.abs(sig).astype(np.complex128)) if with_sigma else {}
    dsig = S.seeded_sigma(13, seed=8, scale=0.1)
    model = O.Prop(**MODEL, **kw, dsigR=dsig, dsigK=0.5j * np.abs(dsig).astype(np.complex128))
    n, A = 37, 3.0
    v = O.grid(n, A)
    gR, gK = _lines(model, v, 0)
    sR, sK = _lines(O.Prop(**MODEL, **kw), v, 1)          # S without the Katanin term
    tab = O.Prop(**MODEL, dsigR=dsig, dsigK=0.5j * np.abs(dsig).astype(np.complex128),
                 gtR=gR, gtK=gK, A_gt=A, stR=sR, stK=sK, A_st=A)
    for which in (0, 1, 2):
        want = O.prop_eval(model, which, v)
        got = O.prop_eval(tab, which, v)
        scale = np.abs(want).max()
        assert np.abs(got - want).max() <= 1e-14 * scale, which
        assert np.all(got[:, 1, 1] == 0)
        assert np.array_equal(got[:, 1, 0], np.conj(got[:, 0, 1]))


def test_linear_tables_are_read_exactly():
    n, A = 23, 4.0
    xn = -1.0 + 2.0 * (np.arange(n) + 1) / (n + 1)
    a, b, c, d = 0.3 - 0.2j, 1.1 + 0.4j, -0.05j, 0.7 + 0.0j
    tab = O.Prop(**MODEL, gtR=a + b * xn, gtK=c + d * xn, A_gt=A)
    rng = np.random.default_rng(11)
    x = rng.uniform(xn[0], xn[-1], 40)
    R, K = _lines(tab, A * np.tan(np.pi * x / 2), 0)
    assert np.abs(R - (a + b * x)).max() <= 1e-13
    assert np.abs(K - (c + d * x)).max() <= 1e-13
    # outer intervals: linear between the last node and 0 at x = +-1
    xo = np.array([0.5 * (xn[-1] + 1.0), 0.5 * (xn[0] - 1.0)])
    R, _ = _lines(tab, A * np.tan(np.pi * xo / 2), 0)
    want = np.array([(a + b * xn[-1]) * (1.0 - xo[0]) / (1.0 - xn[-1]),
                     (a + b * xn[0]) * (xo[1] + 1.0) / (xn[0] + 1.0)])
    assert np.abs(R - want).max() <= 1e-13


def test_bubble_from_sampled_tables_converges_at_second_order():
    g = dict(n1=9, n2w=5, n2v=5, n3w=3, n3v=3)
    Vx = O.Vertex(g, U=1.0, has_R=True)                      # bare vertex: second order
    nq = 201
    exact = O.Prop(**MODEL)
    errs = {O.PI_GG: [], O.PI_GS: []}
    for n in (101, 201, 401):
        v = O.grid(n, 5.0)
        gR, gK = _lines(exact, v, 0)
        sR, sK = _lines(exact, v, 1)
        tab = O.Prop(**MODEL, gtR=gR, gtK=gK, stR=sR, stK=sK)
        for pk in errs:
            for r in (0, 1):
                want = O.bubble_class(Vx, Vx, exact, r, "K1", nq, pi_kind=pk)
                got = O.bubble_class(Vx, Vx, tab, r, "K1", nq, pi_kind=pk)
                errs[pk].append(np.abs(got - want).max() / np.abs(want).max())
    for pk, e in errs.items():
        e = np.array(e).reshape(3, 2)                          # [table size][channel]
        assert np.all(e[1] < e[0] / 3.0) and np.all(e[2] < e[1] / 3.0), (pk, e)
        assert e[2].max() < 2e-3, (pk, e)
