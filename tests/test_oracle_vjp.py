"""Pins of the oracle's vector-jacobian product of the bubble (real-embedding gradients,
bar(z) = dL/dRe z + i dL/dIm z for a real loss L).

- Vertex gradients: the bubble is linear in each vertex's stored classes, so the adjoint
  identity  sum conj(gbar) . B(dGamma) = sum conj(grad) . dGamma  holds exactly (to
  roundoff) for any gbar and any perturbation dGamma, where B(dGamma) is the forward
  oracle evaluated on the perturbation alone (no bare part).  A dropped term, a wrong
  component map, a wrong interpolation corner or a missing up-up exchange fails it.
- G^R gradient: the level eps and the hybridisation Delta enter the bubble only through
  G^R at the sample frequencies (G^A = G^R*, G^K = tanh(v/2T)(G^R - G^A) without a
  self-energy), with dG^R/deps = (G^R)^2 and dG^R/dDelta = -i (G^R)^2; the chain rule
  through the gradient table must reproduce central finite differences of the forward.
"""
import numpy as np
import pytest

import seeded as S
from oracle import oracle as O

G = dict(n1=9, n2w=5, n2v=5, n3w=3, n3v=5)
NQ = 21
U, DELTA, T = 1.3, 1.0, 0.15


def _cgauss(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def _perturbation(seed):
    rng = np.random.default_rng(seed)
    return {c: tuple(_cgauss(rng, O.class_shape(G, k)) for k in O.CLASSES) for c in range(3)}


def _inner(a, b):
    return np.vdot(np.asarray(a).ravel(), np.asarray(b).ravel())   # sum conj(a) b


def _grad_dot(grad, pert):
    return sum(_inner(grad[c][k], pert[c][k]) for c in range(3) for k in range(4))


@pytest.mark.parametrize("r", [0, 1, 2])
@pytest.mark.parametrize("cls", ["K1", "K2", "K2p", "K3"])
def test_vertex_vjp_adjoint_identity(r, cls):
    ch = S.seeded_vertex(G, U, seed=3)
    ch2 = S.seeded_vertex(G, U, seed=4)
    include = (0, 1, 2)
    V1 = O.Vertex(G, U=U, has_R=True, channels=ch, include=include)
    V2 = O.Vertex(G, U=U, has_R=True, channels=ch2, include=include)
    P = O.Prop(Delta=DELTA, T=T)
    rng = np.random.default_rng(11 + r)
    gbar = _cgauss(rng, O.class_shape(G, cls))
    gl, gr, _ = O.bubble_vjp(V1, V2, P, r, cls, NQ, gbar)
    for side in ("left", "right"):
        pert = _perturbation(100 + r + (side == "right"))
        Vp = O.Vertex(G, U=0.0, has_R=False, channels=pert, include=include)
        Bv = O.bubble_class(Vp, V2, P, r, cls, NQ) if side == "left" else O.bubble_class(V1, Vp, P, r, cls, NQ)
        lhs = _inner(gbar, Bv)
        rhs = _grad_dot(gl if side == "left" else gr, pert)
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-30), (side, lhs, rhs)


@pytest.mark.parametrize("r", [0, 2])
def test_vertex_vjp_channel_subset_vertex(r):
    """Multiloop L-part input (only the channels other than r): the up-up component
    still reads the crossing partners; the adjoint identity must hold for it too."""
    ch = S.seeded_vertex(G, U, seed=5)
    include = tuple(c for c in range(3) if c != r)
    V1 = O.Vertex(G, U=0.0, has_R=False, channels=ch, include=include)
    V2 = O.Vertex(G, U=U, has_R=True, channels=S.seeded_vertex(G, U, seed=6))
    P = O.Prop(Delta=DELTA, T=T)
    gbar = _cgauss(np.random.default_rng(7), O.class_shape(G, "K3"))
    gl, _, _ = O.bubble_vjp(V1, V2, P, r, "K3", NQ, gbar, want_right=False)
    pert = _perturbation(200 + r)
    Vp = O.Vertex(G, U=0.0, has_R=False, channels=pert, include=include)
    lhs = _inner(gbar, O.bubble_class(Vp, V2, P, r, "K3", NQ))
    rhs = _grad_dot(gl, pert)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _sample_freqs(r, cls, nq):
    """Frequencies of the two propagators at every [w index][node][side] sample."""
    x, _ = O.gl5_rule(nq)
    w = O.grid(O.class_shape(G, cls)[0])
    with np.errstate(over="ignore"):
        vpp = 5.0 * np.tan(np.pi * x / 2)
    W, X = np.meshgrid(w, vpp, indexing="ij")
    if r == 1:
        a3, a4 = W / 2 + X, W / 2 - X
    else:
        a3, a4 = X + W / 2, X - W / 2
    return np.stack([a3, a4], axis=-1), np.abs(x) < 1.0


@pytest.mark.parametrize("r", [0, 1, 2])
@pytest.mark.parametrize("cls", ["K1", "K2", "K3"])
def test_gr_vjp_matches_finite_differences(r, cls):
    ch = S.seeded_vertex(G, U, seed=8)
    V = O.Vertex(G, U=U, has_R=True, channels=ch)
    eps0 = 0.07
    gbar = _cgauss(np.random.default_rng(21 + r), O.class_shape(G, cls))
    _, _, ggr = O.bubble_vjp(V, V, O.Prop(Delta=DELTA, T=T, eps=eps0), r, cls, NQ, gbar, want_left=False,
                             want_right=False, want_gr=True)
    a, interior = _sample_freqs(r, cls, NQ)

    def loss(eps, Delta):
        B = O.bubble_class(V, V, O.Prop(Delta=Delta, T=T, eps=eps), r, cls, NQ)
        return float(np.real(_inner(gbar, B)))

    h = 1e-4
    with np.errstate(all="ignore"):
        GR = 1.0 / (a - eps0 + 1j * DELTA)
    GR = np.where(interior[None, :, None], GR, 0.0)
    for name, dG, fd in (
            ("eps", GR ** 2, (loss(eps0 + h, DELTA) - loss(eps0 - h, DELTA)) / (2 * h)),
            ("Delta", -1j * GR ** 2, (loss(eps0, DELTA + h) - loss(eps0, DELTA - h)) / (2 * h))):
        chain = float(np.real(_inner(ggr, dG)))
        assert abs(chain - fd) <= 2e-7 * max(abs(fd), 1e-12) + 1e-12, (name, chain, fd)


def test_gr_vjp_rows_follow_the_bosonic_index():
    """A gradient on one bosonic frequency of K1 touches only that row of the table."""
    V = O.Vertex(G, U=U, has_R=True, channels=S.seeded_vertex(G, U, seed=9))
    gbar = np.zeros(O.class_shape(G, "K1"), dtype=np.complex128)
    gbar[3] = _cgauss(np.random.default_rng(1), 16)
    _, _, ggr = O.bubble_vjp(V, V, O.Prop(Delta=DELTA, T=T), 0, "K1", NQ, gbar, want_left=False,
                             want_right=False, want_gr=True)
    assert np.abs(ggr[3]).max() > 0
    assert np.abs(np.delete(ggr, 3, axis=0)).max() == 0
    # the tail nodes (v'' = +-inf) carry no propagator dependence
    assert np.abs(ggr[:, [0, -1]]).max() == 0
