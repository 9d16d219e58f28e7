"""Point evaluation of the full vertex (kb_vertex_eval): the GPU value of a seeded vertex at
arbitrary points — on and between grid points, beyond the grid ends, at infinite
arguments, both spin components, every channel's variables, complex128 and complex64
classes, a channel-subset slot — equals the oracle's evaluation; and the t-channel slice at
zero transfer frequency."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import RAGGED
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _points(rng, n):
    f = rng.standard_normal((n, 3)) * np.array([4.0, 3.0, 3.0])
    f[:5] *= 200.0                                                  # far beyond the grids
    f[5, 1] = np.inf
    f[6, 0] = -np.inf
    g = O.grid(RAGGED["grids"]["n3v"])
    f[7] = (0.0, g[2], g[-3])                                       # grid points
    return f


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("include", [(0, 1, 2), (0, 2)])
def test_vertex_eval_matches_oracle(dtype, include):
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=71)
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch, dtype=dtype, include=include)
    if dtype == torch.complex64:
        ch = {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}
    V = O.Vertex(g, U=cfg["U"], has_R=True, channels=ch, include=include)
    f = _points(np.random.default_rng(3), 257)
    for r in range(3):
        for uu in (0, 1):
            got = e.vertex_eval(0, r, f, spin_uu=uu).cpu().numpy()
            ref = O.vertex_eval(V, r, uu, 0, O.SEL_FULL, f)
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), (r, uu)
    e.close()


def test_t_channel_slice_at_zero_transfer():
    """The slice (w_t = 0, v, v') of a vertex with only the bare part is -U/2 on the
    components with an odd number of quantum indices, everywhere; with classes it matches
    the oracle on a grid of (v, v')."""
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    e.set_vertex(0, U=cfg["U"], has_R=True)
    v = np.linspace(-6, 6, 13)
    f = np.array([(0.0, a, b) for a in v for b in v])
    got = e.vertex_eval(0, 2, f).cpu().numpy()
    odd = np.array([bin(c).count("1") % 2 for c in range(16)], dtype=float)
    assert np.allclose(got, -0.5 * cfg["U"] * odd[None, :], rtol=0, atol=1e-15)
    ch = S.seeded_vertex(g, cfg["U"], seed=72)
    e.set_vertex(1, U=cfg["U"], has_R=True, channels=ch)
    got = e.vertex_eval(1, 2, f).cpu().numpy()
    ref = O.vertex_eval(O.Vertex(g, U=cfg["U"], has_R=True, channels=ch), 2, 0, 0, O.SEL_FULL, f)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    e.close()
