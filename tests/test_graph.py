"""Step graphs: bubbles of two parameter points (different grids, models and precisions,
a loop-part bubble among them) captured into one CUDA graph; every replay reproduces the
eager calls bit for bit, launch accounting follows the replays, and the result matches the
oracle on sampled points."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CLS, RAGGED, rel_err
from oracle import oracle as O

pytestmark = pytest.mark.gpu

EVEN = dict(grids=dict(n1=36, n2w=12, n2v=10, n3w=8, n3v=10), nq=161, U=2.5, Delta=1.0, T=0.03)


def _engine(cfg):
    from paper_2405_20996_gb300.engine import Engine
    e = Engine(cfg["grids"], cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    return e


def _snapshot(e, slot, chans):
    return {(c, k): e.tensors[slot][(c, k)].clone() for c in chans for k in range(4)}


def test_graph_replays_match_eager_two_points():
    from paper_2405_20996_gb300.engine import StepGraph
    A, B = RAGGED, EVEN
    ea, eb = _engine(A), _engine(B)
    cha = S.seeded_vertex(A["grids"], A["U"], seed=70)
    chb = S.seeded_vertex(B["grids"], B["U"], seed=71)
    dot = S.seeded_vertex(A["grids"], 0.4, seed=72)
    ea.set_vertex(0, U=A["U"], has_R=True, channels=cha)
    ea.set_vertex(1, U=0.0, has_R=False, channels=dot, include=(1, 2))     # L-part input of the a channel
    ea.alloc_out(2, channels=(0, 1, 2))
    ea.alloc_out(3, channels=(0,))
    eb.set_vertex(0, U=B["U"], has_R=True, channels=chb, dtype=torch.complex64, symmetric=True)
    eb.alloc_out(1, channels=(0, 2), dtype=torch.complex64)
    descs = [ea.desc(0, 0, 0, 2), ea.desc(1, 0, 0, 2), ea.desc(2, 0, 0, 2),
             ea.desc(0, 1, 0, 3, pi_kind=1, alpha=0.5),
             eb.desc(0, 0, 0, 1, precision="mixed"), eb.desc(2, 0, 0, 1, precision="mixed")]

    def eager():
        for d, e in zip(descs, [ea] * 4 + [eb] * 2):
            e.bubble(d.channel, d.slot_left, d.slot_right, d.out_slot, pi_kind=d.pi_kind, class_mask=d.class_mask,
                     alpha=d.alpha, beta=d.beta, precision="fp64" if d.precision == 0 else "mixed")
        torch.cuda.synchronize()
        return _snapshot(ea, 2, (0, 1, 2)), _snapshot(ea, 3, (0,)), _snapshot(eb, 1, (0, 2))

    ref = eager()
    for e in (ea, eb):
        for slot in e.tensors:
            if slot != 0 and not (e is ea and slot == 1):
                for t in e.tensors[slot].values():
                    t.zero_()
    g = StepGraph(descs)
    n0a, n0b = ea.launches(), eb.launches()
    for rep in range(2):
        g.launch()
        torch.cuda.synchronize()
        got = (_snapshot(ea, 2, (0, 1, 2)), _snapshot(ea, 3, (0,)), _snapshot(eb, 1, (0, 2)))
        for a, b in zip(got, ref):
            for key in b:
                assert torch.equal(a[key], b[key]), (rep, key)
    assert (ea.launches() - n0a) + (eb.launches() - n0b) == 2 * g.kernels()
    # spot check against the oracle: K2 of point B's t channel (mixed tolerance)
    Vb = O.Vertex(B["grids"], U=B["U"], has_R=True,
                  channels={c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in chb.items()})
    ref_b = O.bubble_class(Vb, Vb, O.Prop(Delta=B["Delta"], T=B["T"]), 2, "K2", B["nq"])
    assert rel_err(got[2][(2, 1)].cpu().numpy(), ref_b) <= 1e-6
    g.close()


def test_graph_rejects_bad_descriptor():
    import paper_2405_20996_gb300.kb as kb
    e = _engine(RAGGED)
    e.set_vertex(0, U=1.0, has_R=True, channels=S.seeded_vertex(RAGGED["grids"], 1.0, seed=1))
    e.alloc_out(1, channels=(0,))
    d = e.desc(0, 0, 0, 1)
    d.channel = 5
    with pytest.raises(kb.KBError) as ex:
        kb.kb_graph_create([d])
    assert ex.value.status == kb.KB_ERR_ARG
    d = e.desc(1, 0, 0, 1)          # output class of channel p not attached: fails inside the capture
    with pytest.raises(kb.KBError):
        kb.kb_graph_create([d])
    # the context still works eagerly afterwards
    e.bubble(0, 0, 0, 1)
    torch.cuda.synchronize()


def test_autotuned_contraction_matches_and_tunes_once():
    """kb_set_autotune: the first mixed bubble of a shape times several split-K factors
    (extra k_tc_k3 launches), later ones reuse the choice; the output agrees with the
    untuned bubble to the FP32 segment-sum rounding; a step graph tunes before capturing."""
    import numpy as np
    import torch
    import seeded as S
    from helpers import rel_err
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine, StepGraph
    cfg = dict(grids=dict(n1=37, n2w=13, n2v=11, n3w=9, n3v=11), nq=201, U=1.5, Delta=1.0, T=0.2)
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=41)
    outs = []
    for tune in (False, True):
        e = Engine(g, cfg["nq"])
        e.set_model(cfg["Delta"], cfg["T"])
        e.set_autotune(tune)
        e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch, dtype=torch.complex64, symmetric=True)
        e.alloc_out(1)
        counts = []
        for rep in range(2):
            kb.kb_profile_enable(e.ctx, True)
            e.bubble(2, 0, 0, 1, precision="mixed")
            torch.cuda.synchronize()
            counts.append(kb.kb_profile_read(e.ctx)["k_tc_k3"][1])
            kb.kb_profile_enable(e.ctx, False)
        outs.append({k: v.cpu().numpy() for k, v in e.out(1, 2).items()})
        if tune:
            assert counts[0] > counts[1], counts          # tuning launches only the first time
            gr = StepGraph([e.desc(r, 0, 0, 1, precision="mixed") for r in range(3)])
            gr.launch()
            torch.cuda.synchronize()
            gr.close()
        else:
            assert counts[0] == counts[1], counts
        e.close()
    for k in outs[0]:
        assert rel_err(outs[1][k], outs[0][k]) <= 1e-6, k


def test_graph_of_32_uneven_points_matches_oracle():
    """The batch of the 32-point workload, scaled down so that the oracle computes every
    class in full: 32 parameter points with U/Delta uniform in [0.5, 3], T log-uniform in
    [0.005, 0.5] and K3 grids n^3 with n drawn from {3, 5, 7, 9, 11} (K2 (2n-1)^2, K1 5n-4),
    the one-loop bubble of all three channels of each in mixed precision, as one step graph
    with one branch per point.  Every class of every channel of every point is within 1e-6 of
    the oracle (on the same complex64 vertex), and a replay equals the eager calls bit for bit."""
    from paper_2405_20996_gb300.engine import Engine, StepGraph
    rng = np.random.default_rng(2025)
    nq = 81
    pts = []
    for i in range(32):
        n = int(rng.choice([3, 5, 7, 9, 11]))
        Ui = float(rng.uniform(0.5, 3.0))
        Ti = float(10 ** rng.uniform(np.log10(0.005), np.log10(0.5)))
        g = dict(n1=5 * n - 4, n2w=2 * n - 1, n2v=2 * n - 1, n3w=n, n3v=n)
        ch = S.seeded_vertex(g, Ui, seed=5000 + i)
        e = Engine(g, nq)
        e.set_model(1.0, Ti)
        e.set_vertex(0, U=Ui, has_R=True, channels=ch, dtype=torch.complex64, symmetric=True)
        e.alloc_out(1, dtype=torch.complex64)
        pts.append((e, g, Ui, Ti, ch))
    descs = [e.desc(r, 0, 0, 1, precision="mixed") for e, *_ in pts for r in range(3)]
    for e, *_ in pts:
        for r in range(3):
            e.bubble(r, 0, 0, 1, precision="mixed")
    torch.cuda.synchronize()
    eager = [_snapshot(e, 1, (0, 1, 2)) for e, *_ in pts]
    for e, *_ in pts:
        for t in e.tensors[1].values():
            t.zero_()
    gr = StepGraph(descs)
    gr.launch()
    torch.cuda.synchronize()
    worst, where = 0.0, None
    for (e, g, Ui, Ti, ch), ref_e in zip(pts, eager):
        got = _snapshot(e, 1, (0, 1, 2))
        for key in ref_e:
            assert torch.equal(got[key], ref_e[key]), key
        ch64 = {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}
        V = O.Vertex(g, U=Ui, has_R=True, channels=ch64)
        P = O.Prop(Delta=1.0, T=Ti)
        for r in range(3):
            ref = O.bubble_all(V, V, P, r, nq)
            for k, name in enumerate(CLS):
                err = rel_err(got[(r, k)].cpu().numpy(), ref[name])
                if err > worst:
                    worst, where = err, (g["n3v"], round(Ui, 3), round(Ti, 4), "apt"[r], name)
                assert err <= 1e-6, (g["n3v"], Ui, Ti, r, name, err)
    print("32 uneven points: worst class error %.2e at (n3, U, T, channel, class) = %s" % (worst, where))
    gr.close()
    for e, *_ in pts:
        e.close()
