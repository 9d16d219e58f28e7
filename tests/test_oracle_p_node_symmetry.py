"""Pin of the node symmetry of the p-channel K1 integrand that the mixed path uses to sum the
nodes v'' >= 0 only (Sec. II.C.1 crossing, reading C12): for a crossing-symmetric vertex
bubbled with itself, the integrand of the K1 class at -v'' is the one at v'' with the two
indices of both output pairs exchanged, (a1' a2' | a1 a2) -> (a2' a1' | a2 a1), for Pi = G G
and Pi-dot = G S + S G, at any model (no particle-hole symmetry needed).  The same relation
fails for the a channel and for the p channel without the exchange, so the pin discriminates."""

import numpy as np
import pytest

import seeded as S
from oracle import oracle as O

G = dict(n1=13, n2w=9, n2v=8, n3w=5, n3v=6)


def _integrands(r, pi_kind, w, xs):
    ch = S.seeded_vertex(G, 1.3, seed=91)          # conjugation- and crossing-symmetric
    V = O.Vertex(G, U=1.3, has_R=True, channels=ch)
    P = O.Prop(Delta=0.8, T=0.12, eps=0.3)
    return (O.integrand(V, V, P, r, O.SEL_ZERO, O.SEL_ZERO, w, 0.0, 0.0, xs, pi_kind=pi_kind),
            O.integrand(V, V, P, r, O.SEL_ZERO, O.SEL_ZERO, w, 0.0, 0.0, -xs, pi_kind=pi_kind))


@pytest.mark.parametrize("pi_kind", [O.PI_GG, O.PI_GS])
@pytest.mark.parametrize("w", [0.0, 0.7, -2.3])
def test_p_channel_k1_integrand_at_minus_node_is_the_pair_exchanged_one(pi_kind, w):
    xs = np.array([0.0, 0.11, 0.37, 0.62, 0.9, 1.0])
    plus, minus = _integrands(1, pi_kind, w, xs)
    scale = np.abs(plus).max()
    assert scale > 0
    assert np.abs(minus - plus[:, S.PERM_X]).max() <= 1e-13 * scale
    assert np.abs(minus - plus).max() > 1e-3 * scale          # the exchange is needed


def test_relation_does_not_hold_in_the_a_channel():
    xs = np.array([0.11, 0.37, 0.62, 0.9])
    plus, minus = _integrands(0, O.PI_GG, 0.7, xs)
    assert np.abs(minus - plus[:, S.PERM_X]).max() > 1e-3 * np.abs(plus).max()
