"""Multiloop parts through the same bubble (Sec. III.C): the right part R = B_r(Γ, γ̇_r̄)
with the derivative of the channels other than r on the right, and the central part
C = B_r(Γ, L) whose right vertex is the left part L = B_r(γ̇_r̄, Γ) computed before —
a vertex with channel r only and no bare part.  GPU (FP64 and mixed) against the oracle on
the ragged grids; the chain L -> C runs on each side separately."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CLS, RAGGED, rel_err
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _engine(cfg):
    from paper_2405_20996_gb300.engine import Engine
    e = Engine(cfg["grids"], cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    return e


def _c64(ch):
    return {c: tuple(a.astype(np.complex64) for a in v) for c, v in ch.items()}


def _as128(ch):
    return {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}


def _check(got, ref, tol):
    for k in CLS:
        if np.abs(ref[k]).max() == 0:
            assert np.abs(got[k]).max() == 0, k
        else:
            assert rel_err(got[k], ref[k]) <= tol, (k, rel_err(got[k], ref[k]))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
@pytest.mark.parametrize("r", [0, 2])
def test_right_part(r, precision, tol):
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=81)
    dot = S.seeded_vertex(g, 0.4, seed=82)
    inc = tuple(c for c in range(3) if c != r)
    dt = torch.complex64
    e = _engine(cfg)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=_c64(ch), dtype=dt)
    e.set_vertex(1, has_R=False, channels=_c64(dot), dtype=dt, include=inc)
    e.alloc_out(2, channels=(r,))
    e.bubble(r, 0, 1, 2, precision=precision)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in e.out(2, r).items()}
    V = O.Vertex(g, U=cfg["U"], has_R=True, channels=_as128(ch))
    Vd = O.Vertex(g, has_R=False, channels=_as128(dot), include=inc)
    ref = O.bubble_all(V, Vd, O.Prop(Delta=cfg["Delta"], T=cfg["T"]), r, cfg["nq"])
    _check(got, ref, tol)


@pytest.mark.parametrize("r", [0, 1, 2])
def test_left_then_central_part_fp64(r):
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=83)
    dot = S.seeded_vertex(g, 0.4, seed=84)
    inc = tuple(c for c in range(3) if c != r)
    e = _engine(cfg)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch)
    e.set_vertex(1, has_R=False, channels=dot, include=inc)
    e.alloc_out(2, channels=(r,))
    e.bubble(r, 1, 0, 2)                       # L = B_r(γ̇_r̄, Γ)
    kbmod = __import__("paper_2405_20996_gb300.kb", fromlist=["kb"])
    kbmod.kb_set_vertex_channels(e.ctx, 2, 1 << r)   # L as a vertex: channel r only, no bare part
    e.alloc_out(3, channels=(r,))
    e.bubble(r, 0, 2, 3)                       # C = B_r(Γ, L)
    torch.cuda.synchronize()
    gotL = {k: v.cpu().numpy() for k, v in e.out(2, r).items()}
    gotC = {k: v.cpu().numpy() for k, v in e.out(3, r).items()}
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"])
    V = O.Vertex(g, U=cfg["U"], has_R=True, channels=ch)
    Vd = O.Vertex(g, has_R=False, channels=dot, include=inc)
    refL = O.bubble_all(Vd, V, P, r, cfg["nq"])
    VL = O.Vertex(g, has_R=False, channels={r: tuple(refL[k] for k in CLS)}, include=(r,))
    refC = O.bubble_all(V, VL, P, r, cfg["nq"])
    _check(gotL, refL, 1e-10)
    _check(gotC, refC, 1e-10)
