"""Tabulated lines on the GPU (kb_set_propagator_table: G or S given as tables instead of
computed from the model and Sigma): bubbles with Pi = G G and Pi-dot = G S + S G, FP64
(<= 1e-10) and mixed (<= 1e-6), and the self-energy loop (<= 1e-11) against the oracle with
the same tables, every channel and class; an S table with the model's G and the Katanin term;
refusals (S line undefined with a tabulated G, the G^R gradient, bad arguments); removing the
tables gives back the model's bubble bit for bit."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CLS, RAGGED, rel_err
from oracle import oracle as O

pytestmark = pytest.mark.gpu

N_TAB, A_TAB = 57, 3.0


def _tables(cfg, which, seed):
    """Lines of the model on the table grid plus a seeded perturbation, so that the tables
    are not the model's own lines."""
    v = O.grid(N_TAB, A_TAB)
    m = O.prop_eval(O.Prop(Delta=cfg["Delta"], T=cfg["T"]), which, v)
    d = S.seeded_sigma(N_TAB, seed=seed, scale=0.05, A=A_TAB)
    return m[:, 0, 1] + d, m[:, 0, 0] + 1j * np.abs(d)


def _engine(cfg, ch, dt, g_tab=None, s_tab=None, dsig=None):
    from paper_2405_20996_gb300.engine import Engine
    e = Engine(cfg["grids"], cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    if g_tab is not None:
        e.set_propagator_table("G", *g_tab, A_tab=A_TAB)
    if s_tab is not None:
        e.set_propagator_table("S", *s_tab, A_tab=A_TAB)
    if dsig is not None:
        e.set_self_energy_derivative(*dsig, A_dsig=4.0)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch, dtype=dt, symmetric=True)
    e.alloc_out(1)
    return e


def _as_stored(ch, precision):
    if precision != "mixed":
        return ch
    return {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}


@pytest.mark.parametrize("pi_kind", [0, 1])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_bubbles_with_tabulated_lines_match_oracle(pi_kind, precision, tol):
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=71)
    gt, st = _tables(cfg, 0, 21), _tables(cfg, 1, 22)
    dt = torch.complex64 if precision == "mixed" else torch.complex128
    e = _engine(cfg, ch, dt, g_tab=gt, s_tab=st)
    V = O.Vertex(g, U=cfg["U"], has_R=True, channels=_as_stored(ch, precision))
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], gtR=gt[0], gtK=gt[1], A_gt=A_TAB, stR=st[0], stK=st[1], A_st=A_TAB)
    for r in range(3):
        e.bubble(r, 0, 0, 1, pi_kind=pi_kind, precision=precision)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in e.out(1, r).items()}
        ref = O.bubble_all(V, V, P, r, cfg["nq"], pi_kind=pi_kind)
        for k in CLS:
            assert rel_err(got[k], ref[k]) <= tol, (r, k, rel_err(got[k], ref[k]))
    e.close()


def test_s_table_with_model_G_and_katanin_term_matches_oracle():
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=72)
    st = _tables(cfg, 1, 23)
    dsR = S.seeded_sigma(25, seed=4, scale=0.2)
    dsig = (dsR, 0.5j * np.abs(dsR).astype(np.complex128))
    e = _engine(cfg, ch, torch.complex128, s_tab=st, dsig=dsig)
    V = O.Vertex(g, U=cfg["U"], has_R=True, channels=ch)
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], stR=st[0], stK=st[1], A_st=A_TAB, dsigR=dsig[0], dsigK=dsig[1],
               A_dsig=4.0)
    for r in range(3):
        e.bubble(r, 0, 0, 1, pi_kind=1, precision="fp64")
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in e.out(1, r).items()}
        ref = O.bubble_all(V, V, P, r, cfg["nq"], pi_kind=1)
        for k in CLS:
            assert rel_err(got[k], ref[k]) <= 1e-10, (r, k, rel_err(got[k], ref[k]))
    e.close()


@pytest.mark.parametrize("line", [0, 1])
def test_loop_with_tabulated_lines_matches_oracle(line):
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=73)
    gt, st = _tables(cfg, 0, 24), _tables(cfg, 1, 25)
    e = _engine(cfg, ch, torch.complex128, g_tab=gt, s_tab=st)
    nus = np.array([-6.0, -1.3, -0.2, 0.0, 0.45, 2.2, 11.0])
    got = e.loop(0, nus, line=line).cpu().numpy()
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], gtR=gt[0], gtK=gt[1], A_gt=A_TAB, stR=st[0], stK=st[1], A_st=A_TAB)
    ref = O.loop(O.Vertex(g, U=cfg["U"], has_R=True, channels=ch), P, cfg["nq"], nus, which=line)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), np.abs(got - ref).max()
    e.close()


def test_refusals_and_removal():
    from paper_2405_20996_gb300 import kb
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=74)
    e = _engine(cfg, ch, torch.complex128)
    e.bubble(0, 0, 0, 1, pi_kind=0, precision="fp64")
    torch.cuda.synchronize()
    before = {k: v.cpu().numpy().copy() for k, v in e.out(1, 0).items()}
    L = kb.lib()
    r = np.zeros(2 * N_TAB)
    p = r.ctypes.data
    assert L.kb_set_propagator_table(e.ctx, 5, N_TAB, A_TAB, p, None) == kb.KB_ERR_ARG
    assert L.kb_set_propagator_table(e.ctx, kb.KB_PROP_G, 0, A_TAB, p, None) == kb.KB_ERR_ARG
    assert L.kb_set_propagator_table(e.ctx, kb.KB_PROP_G, N_TAB, 0.0, p, None) == kb.KB_ERR_ARG
    bad = r.copy()
    bad[3] = np.nan
    assert L.kb_set_propagator_table(e.ctx, kb.KB_PROP_G, N_TAB, A_TAB, bad.ctypes.data, None) == kb.KB_ERR_ARG
    gt = _tables(cfg, 0, 26)
    e.set_propagator_table("G", *gt, A_tab=A_TAB)
    with pytest.raises(kb.KBError) as x:
        e.bubble(0, 0, 0, 1, pi_kind=1, precision="fp64")
    assert x.value.status == kb.KB_ERR_STATE
    with pytest.raises(kb.KBError) as x:
        e.loop(0, [0.5], line=1)
    assert x.value.status == kb.KB_ERR_STATE
    with pytest.raises(kb.KBError) as x:
        e.bubble_vjp(0, 0, 0, 1, grad_gr=e.gr_tables())
    assert x.value.status == kb.KB_ERR_UNSUPPORTED
    e.bubble(0, 0, 0, 1, pi_kind=0, precision="fp64")
    torch.cuda.synchronize()
    with_tab = {k: v.cpu().numpy().copy() for k, v in e.out(1, 0).items()}
    assert max(rel_err(with_tab[k], before[k]) for k in CLS) > 1e-3      # the table is used
    e.set_propagator_table("G", None)
    e.bubble(0, 0, 0, 1, pi_kind=0, precision="fp64")
    torch.cuda.synchronize()
    for k in CLS:
        assert np.array_equal(e.out(1, 0)[k].cpu().numpy(), before[k]), k
    e.close()
