"""Pin of the symmetry image that relates the right and left multiloop parts (Sec. II.G.3
symmetries; Sec. III.C parts): for a conjugation- and crossing-symmetric Γ and X,

    B_r(Γ, X) = I_r[B_r(X, Γ)],

with I_r the conjugation (a, p: (w, v, v') -> (w, v', v), Keldysh (a1'a2'|a1a2) -> (a1a2|a1'a2'),
complex conjugate, sign (-1)^(1+Σa)) or, for t, the conjugation after crossing (the same w,
v <-> v', Keldysh permutation of both maps).  K2 and K2' trade places.  Checked on the oracle
for every channel and class, with X a channel subset (the multiloop γ_rbar)."""

import numpy as np
import pytest

import seeded as S
from oracle import oracle as O

G = dict(n1=11, n2w=7, n2v=6, n3w=5, n3v=4)
NQ = 41


def perm_c(c):                       # conjugation: (a1'a2'|a1a2) -> (a1a2|a1'a2')
    return ((c & 3) << 2) | (c >> 2)


def perm_x(c):                       # crossing: (a1'a2'|a1a2) -> (a2'a1'|a2a1)
    return (((c >> 2) & 1) << 3) | (((c >> 3) & 1) << 2) | ((c & 1) << 1) | ((c >> 1) & 1)


def sign_c(c):                       # (-1)^(1 + number of quantum indices + 4)
    return 1.0 if bin(c).count("1") % 2 else -1.0


def image(r, cls):
    """{K1, K2, K2p, K3} of I_r[B]."""
    p = [perm_x(perm_c(c)) if r == 2 else perm_c(c) for c in range(16)]
    sg = np.array([sign_c(c) for c in range(16)])
    f = lambda a: sg * np.conj(a[..., p])
    return {"K1": f(cls["K1"]), "K2": f(cls["K2p"]), "K2p": f(cls["K2"]),
            "K3": f(np.swapaxes(cls["K3"], 1, 2))}


@pytest.mark.parametrize("r", [0, 1, 2])
def test_right_part_is_the_image_of_the_left_part(r):
    gam = S.seeded_vertex(G, 1.0, seed=51)
    x = S.seeded_vertex(G, 0.4, seed=52)
    P = O.Prop(Delta=1.0, T=0.1)
    Gv = O.Vertex(G, U=1.0, has_R=True, channels=gam)
    Xv = O.Vertex(G, has_R=False, channels=x, include=[c for c in range(3) if c != r])
    L = O.bubble_all(Xv, Gv, P, r, NQ)
    R = O.bubble_all(Gv, Xv, P, r, NQ)
    I = image(r, L)
    for k in ("K1", "K2", "K2p", "K3"):
        m = max(np.abs(R[k]).max(), 1e-300)
        assert np.abs(I[k] - R[k]).max() <= 1e-12 * max(m, np.abs(L["K3"]).max()), (r, k)
    assert np.abs(R["K2p"]).max() > 0 and np.abs(R["K3"]).max() > 0
