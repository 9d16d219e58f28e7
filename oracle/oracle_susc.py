"""Susceptibilities from the full vertex by contracting pairs of external legs (the paper's
post-processing, Sec. II.E.5), written out on the oracle's bubbles (TEST INFRASTRUCTURE:
only tests use this module; it shares no code with the CUDA library or its Python package).

The a-channel susceptibility is drawn as the bare bubble closed at both ends plus a bubble,
the full vertex and a bubble, closed at both ends; p likewise.  Closing a pair of legs with a
unit bare vertex R̂ (the bare vertex at U = 1: -1/2 on the Keldysh components with an odd
number of quantum indices) turns both into bubble chains of channel r whose vertices at the
ends are local, so only their K1 class survives:

    K1_r[ R̂ Π R̂ + R̂ Π Γ Π R̂ ] = K1_r[ B_r(R̂, R̂) + B_r(R̂, X) ],   X = B_r(Γ, R̂),

where X has only K1 and K2 (its right vertex is bare) and enters B_r(R̂, X) as a channel-r
vertex (R0 = X_K1 + X_K2(ω, v'')).  The susceptibility is read off this K1 exactly as from
the vertex's own K1 at U = 1 (observables.susceptibility_from_K1's normalisation):
χ_a = -2 K1, χ_p = +2 K1 on the retarded and Keldysh components.  Defined here for the a
(transverse spin) and p (pairing) channels.
"""

import numpy as np

from . import oracle as O

CLS = ("K1", "K2", "K2p", "K3")
# representative components of the retarded and Keldysh blocks, and the normalisation
_COMP = {0: (1, 3), 1: (8, 9)}
_SCALE = {0: -2.0, 1: 2.0}


def chi_from_k1(K1, r):
    """(χ^R, χ^K) of channel r (0 or 1) from a K1 array [n1][16] of a chain closed by R̂."""
    cR, cK = _COMP[r]
    return _SCALE[r] * K1[:, cR], _SCALE[r] * K1[:, cK]


def legs_k1(V, P, r, nq):
    """K1 of R̂ Π R̂ + R̂ Π Γ Π R̂ in channel r (V: the vertex Γ as an oracle Vertex)."""
    g = V.grids
    Rh = O.Vertex(g, U=1.0, has_R=True)
    X = O.bubble_all(V, Rh, P, r, nq, classes=("K1", "K2"))
    VX = O.Vertex(g, channels={r: (X["K1"], X["K2"], None, None)}, include=(r,))
    return O.bubble_class(Rh, Rh, P, r, "K1", nq) + O.bubble_class(Rh, VX, P, r, "K1", nq)


def chi_legs(V, P, r, nq):
    """(χ^R, χ^K) on the K1 grid from the full vertex V by the leg contraction."""
    if r not in _COMP:
        raise ValueError("the leg contraction is written out for the a and p channels")
    return chi_from_k1(legs_k1(V, P, r, nq), r)
