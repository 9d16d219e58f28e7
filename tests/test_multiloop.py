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
    assert ml.parts_per_step() == 3 * (1 + 2 + 3 * (ml.n_loops - 2))
    assert ml.bubbles_per_step() == ml.parts_per_step() - 3          # order 2's right parts as images
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


def test_record_cache_matches_gather_and_goes_stale():
    """kb_vertex_cache: the K2 (left) and K2' (right) contractions of a cached vertex agree with
    the gathering kernels to FP32 rounding (same records, another summation order), the K3
    class from its cached tiles is bit-identical; any change of the slot makes the cache
    stale (then unused)."""
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    gam = S.seeded_vertex(g, cfg["U"], seed=94)
    y = S.seeded_vertex(g, 0.3, seed=95)
    outs = {}
    for use_cache in (False, True):
        for r in range(3):
            e = Engine(g, cfg["nq"])
            e.set_model(cfg["Delta"], cfg["T"])
            e.set_vertex(0, U=cfg["U"], has_R=True, channels=gam, dtype=torch.complex64, symmetric=True)
            # a channel-r-only vertex (like the left part that the central part reads): its
            # r-independent part is not zero, so every class of both bubbles is computed
            e.set_vertex(1, has_R=False, channels={r: y[r]}, dtype=torch.complex64, include=[r])
            e.alloc_out(2, channels=(r,), dtype=torch.complex64)
            e.alloc_out(3, channels=(r,), dtype=torch.complex64)
            if use_cache:
                kb.kb_vertex_cache(e.ctx, 0, r, 15, torch.cuda.current_stream().cuda_stream)
            kb.kb_profile_enable(e.ctx, True)
            e.bubble(r, 1, 0, 2, precision="mixed")          # Γ on the right: its K2' records
            e.bubble(r, 0, 1, 3, precision="mixed")          # Γ on the left: its K2 records
            torch.cuda.synchronize()
            prof = kb.kb_profile_read(e.ctx)
            names = set(prof)
            kb.kb_profile_enable(e.ctx, False)
            assert ({"k_mx_k2c", "k_mx_k2pc"} <= names) == use_cache, names
            # K3: Γ's tiles come from the cache, only Y's are built
            ntile = 1 if use_cache else 2
            assert prof["k_mx_tile3_left"][1] == prof["k_mx_tile3_right"][1] == ntile, prof
            outs[(use_cache, r)] = {s: {k: t.cpu().numpy() for k, t in e.out(s, r).items()} for s in (2, 3)}
            if use_cache:
                # re-attaching a class of the cached slot makes the cache stale
                t = e.tensors[0][(0, 0)]
                kb.kb_set_vertex_class(e.ctx, 0, 0, 0, t.data_ptr(), kb.KB_DT_C64)
                kb.kb_profile_enable(e.ctx, True)
                e.bubble(r, 0, 1, 3, precision="mixed")
                torch.cuda.synchronize()
                names = set(kb.kb_profile_read(e.ctx))
                assert "k_mx_k2" in names and "k_mx_k2c" not in names, names
                kb.kb_vertex_uncache(e.ctx, 0)
            e.close()
    for r in range(3):
        for s in (2, 3):
            for k in CLS:
                a, b = outs[(False, r)][s][k], outs[(True, r)][s][k]
                assert np.abs(a).max() > 0, (r, s, k)
                if k in ("K1", "K3"):
                    assert np.array_equal(a, b), (r, s, k)          # not touched by the cache
                else:
                    assert rel_err(b.astype(np.complex128), a.astype(np.complex128)) <= 1e-6, (r, s, k)


def test_cached_multiloop_step_matches_uncached():
    cfg = RAGGED
    vertex = S.seeded_vertex(cfg["grids"], cfg["U"], seed=96)
    from paper_2405_20996_gb300.multiloop import MultiloopStep
    res = []
    for cache in (False, True):
        ml = MultiloopStep(cfg["grids"], cfg["nq"], cfg["U"], cfg["Delta"], cfg["T"], vertex, n_loops=4,
                           precision="mixed", cache=cache)
        assert ml.cached == ({0: 15, 1: 15, 2: 15} if cache else {})
        ml.zero()
        ml.run()
        torch.cuda.synchronize()
        res.append(_orders(ml))
        ml.close()
    _compare(res[1], res[0], 2e-6)


def test_parts_of_a_vertex_without_channel_r_skip_the_zero_classes():
    """A left vertex with no bare part and without channel r (the multiloop left part
    B_r(gamma_rbar, Gamma)) has L0 = 0, so K1 and K2' are zero; the right part has R0 = 0, so
    K1 and K2 are zero.  The mixed path writes beta * out for them without computing; the
    other classes match the FP64 path."""
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    gam = _c64(S.seeded_vertex(g, cfg["U"], seed=97))
    x = _c64(S.seeded_vertex(g, 0.3, seed=98))
    for r in range(3):
        res = {}
        for prec, dt in (("mixed", torch.complex64), ("fp64", torch.complex128)):
            e = Engine(g, cfg["nq"])
            e.set_model(cfg["Delta"], cfg["T"])
            e.set_vertex(0, U=cfg["U"], has_R=True, channels=gam, dtype=dt)
            e.set_vertex(1, has_R=False, channels=x, dtype=dt, include=[c for c in range(3) if c != r])
            for o in (2, 3):
                e.alloc_out(o, channels=(r,), dtype=torch.complex128)
                for t in e.tensors[o].values():
                    t.fill_(7.0)                     # beta = 0.5 keeps half of it where B = 0
            kb.kb_profile_enable(e.ctx, True)
            e.bubble(r, 1, 0, 2, beta=0.5, precision=prec)     # left part
            e.bubble(r, 0, 1, 3, beta=0.5, precision=prec)     # right part
            torch.cuda.synchronize()
            names = kb.kb_profile_read(e.ctx)
            res[prec] = {o: {k: t.cpu().numpy() for k, t in e.out(o, r).items()} for o in (2, 3)}
            if prec == "mixed":
                assert names.get("k_mx_k2", (0, 0))[1] == 1 and names.get("k_mx_k2p", (0, 0))[1] == 1, names
                assert "k_mx_k1" not in names, names
            e.close()
        for o, zero in ((2, ("K1", "K2p")), (3, ("K1", "K2"))):
            for k in CLS:
                m, f = res["mixed"][o][k], res["fp64"][o][k]
                if k in zero:
                    assert np.all(m == 3.5) and np.allclose(f, 3.5, rtol=0, atol=1e-12), (r, o, k)
                else:
                    assert rel_err(m - 3.5, f - 3.5) <= 1e-6, (r, o, k, rel_err(m - 3.5, f - 3.5))
