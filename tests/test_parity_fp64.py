"""Parity of the plain FP64 CUDA path (through the C ABI) with the FP64 CPU oracle,
element by element, relative max-norm per class <= 1e-10."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CFG0, CLS, RAGGED, oracle_vertex, rel_err, seeded_inputs
from oracle import oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-10


def engine_for(cfg):
    from paper_2405_20996_gb300.engine import Engine
    e = Engine(cfg["grids"], cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    return e


def run_gpu(e, ch_in, r, U, pi_kind=0, dtype=torch.complex128, left=None, right=None, has_R=True):
    e.set_vertex(0, U=U, has_R=has_R, channels=ch_in, dtype=dtype)
    if left is not None:
        e.set_vertex(1, U=U, has_R=left[1], channels=left[0], dtype=dtype, include=left[2])
    e.alloc_out(2, channels=(r,))
    e.bubble(r, 1 if left is not None else 0, 0, 2, pi_kind=pi_kind)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in e.out(2, r).items()}


@pytest.mark.parametrize("r", [0, 1, 2])
def test_ragged_all_channels(r):
    cfg = RAGGED
    ch = seeded_inputs(cfg, seed=21)
    e = engine_for(cfg)
    got = run_gpu(e, ch, r, cfg["U"])
    V = oracle_vertex(cfg, ch)
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"])
    ref = O.bubble_all(V, V, P, r, cfg["nq"])
    for k in CLS:
        assert rel_err(got[k], ref[k]) <= TOL, (r, k, rel_err(got[k], ref[k]))


def test_cfg0_a_channel_full():
    """Plain FP64 a-channel one-loop bubble on the small workload (K1 101, K2 21x21,
    K3 15^3, 1001 nodes, complex128)."""
    cfg = CFG0
    ch = seeded_inputs(cfg, seed=0)
    e = engine_for(cfg)
    got = run_gpu(e, ch, 0, cfg["U"])
    V = oracle_vertex(cfg, ch)
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"])
    ref = O.bubble_all(V, V, P, 0, cfg["nq"])
    for k in CLS:
        assert rel_err(got[k], ref[k]) <= TOL, (k, rel_err(got[k], ref[k]))


@pytest.mark.parametrize("r", [0, 2])
def test_pi_dot_sigma_table_and_loop_part_slots(r):
    """Pi-dot = G S + S G with a tabulated self-energy (Dyson in FP64), left vertex an
    r-irreducible vertex without R (the multiloop 'L' part) and complex64 inputs."""
    cfg = dict(RAGGED, T=0.07)
    g = cfg["grids"]
    ch = seeded_inputs(cfg, seed=3)
    dot = S.seeded_vertex(g, 0.5, seed=4)
    inc = tuple(c for c in range(3) if c != r)        # gamma-dot of the channels other than r
    sg = O.grid(33)
    sR = S.seeded_sigma(33, seed=9)
    sK = 2j * np.tanh(sg / (2 * cfg["T"])) * sR.imag
    e = engine_for(cfg)
    e.set_self_energy(sR, sK)
    ch32 = {c: tuple(a.astype(np.complex64) for a in v) for c, v in ch.items()}
    dot32 = {c: tuple(a.astype(np.complex64) for a in v) for c, v in dot.items()}
    got = run_gpu(e, ch32, r, cfg["U"], pi_kind=1, dtype=torch.complex64, left=(dot32, False, inc))
    cast = lambda d: {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in d.items()}
    V = oracle_vertex(cfg, cast(ch))
    Vd = O.Vertex(g, U=cfg["U"], has_R=False, channels=cast(dot), include=inc)
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], sigR=sR, sigK=sK)
    ref = O.bubble_all(Vd, V, P, r, cfg["nq"], pi_kind=O.PI_GS)
    assert np.abs(ref["K1"]).max() == 0.0 and np.abs(ref["K2p"]).max() == 0.0   # L part: no K1, K2'
    for k in CLS:
        if np.abs(ref[k]).max() == 0:
            assert np.abs(got[k]).max() == 0
        else:
            assert rel_err(got[k], ref[k]) <= TOL, (k, rel_err(got[k], ref[k]))


def test_alpha_beta_and_pt2():
    """out <- alpha B + beta out, and the PT2 bubble of the bare vertex."""
    cfg = RAGGED
    e = engine_for(cfg)
    e.set_vertex(0, U=cfg["U"], has_R=True)
    e.alloc_out(2, channels=(1,))
    for k, t in e.out(2, 1).items():
        t.copy_(torch.full_like(t, 0.5 - 0.25j))
    e.bubble(1, 0, 0, 2, alpha=2.0, beta=-1.0)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in e.out(2, 1).items()}
    V = O.Vertex(cfg["grids"], U=cfg["U"], has_R=True)
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"])
    ref = O.bubble_all(V, V, P, 1, cfg["nq"])
    for k in CLS:
        want = 2.0 * ref[k] - (0.5 - 0.25j)
        assert rel_err(got[k], want) <= TOL


def test_degenerate_sizes():
    """Single-point grids and the smallest quadrature (one panel, 5 nodes)."""
    cfg = dict(grids=dict(n1=1, n2w=1, n2v=1, n3w=1, n3v=1), nq=5, U=1.0, Delta=1.0, T=0.3)
    ch = seeded_inputs(cfg, seed=8)
    for r in range(3):
        e = engine_for(cfg)
        got = run_gpu(e, ch, r, cfg["U"])
        V = oracle_vertex(cfg, ch)
        ref = O.bubble_all(V, V, O.Prop(Delta=1.0, T=0.3), r, 5)
        for k in CLS:
            assert rel_err(got[k], ref[k]) <= TOL


def test_invalid_arguments_return_errors():
    from paper_2405_20996_gb300 import kb
    e = engine_for(RAGGED)
    with pytest.raises(kb.KBError) as ei:
        kb.kb_bubble(e.ctx, 3, 0, 0, 0)
    assert ei.value.status == kb.KB_ERR_ARG
    with pytest.raises(kb.KBError) as ei:
        kb.kb_bubble(e.ctx, 0, 5, 5, 6)           # slots never set
    assert ei.value.status == kb.KB_ERR_STATE
    with pytest.raises(kb.KBError):
        kb.kb_set_grids(e.ctx, 10, 10, 10, 10, 10, 100)   # nq not 4P+1
