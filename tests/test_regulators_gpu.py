"""Flow schemes of the single-scale propagator on the GPU (kb_set_regulator, Sec. III.C.2):
the interaction and temperature flows, Π = G G and Π-dot = G S + S G, FP64 (<= 1e-10) and
mixed (<= 1e-6) against the oracle with the same scheme, every channel and class; bad
scheme arguments are refused."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CLS, RAGGED, rel_err
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _run(cfg, reg, lam, pi_kind, precision):
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=61)
    dt = torch.complex64 if precision == "mixed" else torch.complex128
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    e.set_regulator(reg, lam)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch, dtype=dt, symmetric=True)
    e.alloc_out(1)
    out = {}
    for r in range(3):
        e.bubble(r, 0, 0, 1, pi_kind=pi_kind, precision=precision)
        torch.cuda.synchronize()
        out[r] = {k: v.cpu().numpy() for k, v in e.out(1, r).items()}
    e.close()
    if precision == "mixed":
        ch = {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}
    return out, ch


@pytest.mark.parametrize("reg,lam", [(1, 0.7), (2, 1.0)])
@pytest.mark.parametrize("pi_kind", [0, 1])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_flow_scheme_bubbles_match_oracle(reg, lam, pi_kind, precision, tol):
    cfg = RAGGED
    got, ch = _run(cfg, reg, lam, pi_kind, precision)
    V = O.Vertex(cfg["grids"], U=cfg["U"], has_R=True, channels=ch)
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], reg=reg, lam=lam)
    for r in range(3):
        ref = O.bubble_all(V, V, P, r, cfg["nq"], pi_kind=pi_kind)
        for k in CLS:
            if np.abs(ref[k]).max() == 0:
                assert np.abs(got[r][k]).max() <= 1e-14, (r, k)
            else:
                assert rel_err(got[r][k], ref[k]) <= tol, (r, k, rel_err(got[r][k], ref[k]))


def test_bad_regulator_arguments_refused():
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine
    e = Engine(RAGGED["grids"], RAGGED["nq"])
    L = kb.lib()
    assert L.kb_set_regulator(e.ctx, 7, 1.0) == kb.KB_ERR_ARG
    assert L.kb_set_regulator(e.ctx, kb.KB_REG_U, 0.0) == kb.KB_ERR_ARG
    e.set_model(1.0, 0.0)
    assert L.kb_set_regulator(e.ctx, kb.KB_REG_T, 1.0) == kb.KB_ERR_ARG          # T = 0
    e.set_model(1.0, 0.1)
    e.set_regulator(kb.KB_REG_T)
    assert L.kb_set_model(e.ctx, 1.0, 0.0, 0.0) == kb.KB_ERR_ARG
    e.close()


@pytest.mark.parametrize("reg", [0, 1, 3])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_katanin_substitution_matches_oracle(reg, precision, tol):
    """Π-dot with G-dot = S + G dΣ G (self-energy and its derivative as tables) against the
    oracle with the same tables; reg 3 (no flow parameter, S = 0) leaves G dΣ G alone, the
    change of G along dΣ."""
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    sigR = S.seeded_sigma(31, seed=3, scale=0.3)
    sigK = 1j * np.abs(sigR).astype(np.complex128)
    dsigR = S.seeded_sigma(25, seed=4, scale=0.2)
    dsigK = 0.5j * np.abs(dsigR).astype(np.complex128)
    ch = S.seeded_vertex(g, cfg["U"], seed=62)
    dt = torch.complex64 if precision == "mixed" else torch.complex128
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    e.set_regulator(reg, 0.8)
    e.set_self_energy(sigR, sigK)
    e.set_self_energy_derivative(dsigR, dsigK, A_dsig=4.0)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch, dtype=dt, symmetric=True)
    e.alloc_out(1)
    if precision == "mixed":
        ch = {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}
    V = O.Vertex(g, U=cfg["U"], has_R=True, channels=ch)
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], reg=reg, lam=0.8, sigR=sigR, sigK=sigK, dsigR=dsigR, dsigK=dsigK,
               A_dsig=4.0)
    for r in range(3):
        e.bubble(r, 0, 0, 1, pi_kind=1, precision=precision)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in e.out(1, r).items()}
        ref = O.bubble_all(V, V, P, r, cfg["nq"], pi_kind=1)
        for k in CLS:
            assert rel_err(got[k], ref[k]) <= tol, (r, k, rel_err(got[k], ref[k]))
    e.close()
