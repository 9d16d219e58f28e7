"""Multiloop vertex step (Sec. III.C) as one step graph: the one-loop bubble with the
single-scale pair, then the left, central and right parts of each loop order, slot
additions and joins between orders.

- the FP64 graph equals the same loop-order recursion run on the oracle's bubbles (every
  order, every channel and class, <= 1e-10), and the accumulated derivative equals the sum
  of the orders;
- the graph replay equals the same entries launched eagerly on one stream, bit for bit
  (FP64 and mixed);
- the mixed graph stays within 1e-5 of the FP64 graph at every order (c64-rounded inputs
  on both sides)."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CLS, RAGGED, rel_err
from oracle import oracle as O

pytestmark = pytest.mark.gpu

TINY = dict(grids=dict(n1=13, n2w=7, n2v=6, n3w=5, n3v=4), nq=41, U=1.0, Delta=1.0, T=0.1)


def _step(cfg, vertex, n_loops, precision):
    from paper_2405_20996_gb300.multiloop import MultiloopStep
    return MultiloopStep(cfg["grids"], cfg["nq"], cfg["U"], cfg["Delta"], cfg["T"], vertex, n_loops=n_loops,
                         precision=precision)


def _orders(ml):
    return [{r: {k: v.cpu().numpy().astype(np.complex128) for k, v in ml.order(l, r).items()} for r in range(3)}
            for l in range(1, ml.n_loops + 1)]


def _c64(ch):
    return {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}


def _oracle_orders(cfg, vertex, n_loops):
    g, nq = cfg["grids"], cfg["nq"]
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"])
    Gam = O.Vertex(g, U=cfg["U"], has_R=True, channels=vertex)
    tup = lambda d: tuple(d[k] for k in CLS)
    orders = [{r: O.bubble_all(Gam, Gam, P, r, nq, pi_kind=O.PI_GS) for r in range(3)}]
    lefts = {}
    for l in range(2, n_loops + 1):
        prev = {c: tup(orders[-1][c]) for c in range(3)}
        cur, new_lefts = {}, {}
        for r in range(3):
            bar = O.Vertex(g, has_R=False, channels=prev, include=[c for c in range(3) if c != r])
            Lr = O.bubble_all(bar, Gam, P, r, nq)
            Rr = O.bubble_all(Gam, bar, P, r, nq)
            tot = {k: Lr[k] + Rr[k] for k in CLS}
            if l >= 3:
                Lv = O.Vertex(g, has_R=False, channels={r: tup(lefts[r])}, include=[r])
                Cr = O.bubble_all(Gam, Lv, P, r, nq)
                tot = {k: tot[k] + Cr[k] for k in CLS}
            cur[r], new_lefts[r] = tot, Lr
        orders.append(cur)
        lefts = new_lefts
    return orders


def _compare(got, ref, tol):
    for l, (go, ro) in enumerate(zip(got, ref), start=1):
        for r in range(3):
            for k in CLS:
                if np.abs(ro[r][k]).max() == 0:
                    assert np.abs(go[r][k]).max() <= 1e-14, (l, r, k)
                else:
                    e = rel_err(go[r][k], ro[r][k])
                    assert e <= tol, (l, r, k, e)


def test_fp64_step_matches_oracle_recursion():
    cfg = TINY
    vertex = S.seeded_vertex(cfg["grids"], cfg["U"], seed=91)
    ml = _step(cfg, vertex, 4, "fp64")
    ml.zero()
    ml.run()
    torch.cuda.synchronize()
    got = _orders(ml)
    ref = _oracle_orders(cfg, vertex, 4)
    _compare(got, ref, 1e-10)
    for r in range(3):
        for k, v in ml.derivative(r).items():
            assert rel_err(v.cpu().numpy(), sum(o[r][k] for o in got)) <= 1e-14
    ml.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_equals_eager(precision):
    cfg = RAGGED
    vertex = S.seeded_vertex(cfg["grids"], cfg["U"], seed=92)
    ml = _step(cfg, vertex, 5, precision)
    ml.zero()
    ml.run()
    torch.cuda.synchronize()
    a = _orders(ml)
    ta = {r: {k: v.cpu().numpy() for k, v in ml.derivative(r).items()} for r in range(3)}
    ml.zero()
    for o in ml.orders:
        for t in o.values():
            t.fill_(1.0)                      # the eager run must overwrite every order
    ml.run_eager()
    torch.cuda.synchronize()
    b = _orders(ml)
    for l in range(ml.n_loops):
        for r in range(3):
            for k in CLS:
                assert np.array_equal(a[l][r][k], b[l][r][k]), (l + 1, r, k)
    for r in range(3):
        for k, v in ml.derivative(r).items():
            assert np.array_equal(v.cpu().numpy(), ta[r][k]), (r, k)
    assert ml.bubbles_per_step() == 3 * (1 + 2 + 3 * (ml.n_loops - 2))
    ml.close()


def test_mixed_step_tracks_fp64():
    cfg = RAGGED
    vertex = _c64(S.seeded_vertex(cfg["grids"], cfg["U"], seed=93))
    mm = _step(cfg, vertex, 6, "mixed")
    mf = _step(cfg, vertex, 6, "fp64")
    for m in (mm, mf):
        m.zero()
        m.run()
    torch.cuda.synchronize()
    _compare(_orders(mm), _orders(mf), 1e-5)
    mm.close()
    mf.close()
