"""The t-channel bubble in its SU(2) form (kb_bubble_t_su2 + kb_t_su2_finish): K3 from the
density contraction −Γ^d Π_t Γ^d (Γ^d = Γ_uu + Γ_ud, one spin record per side) and the
a-channel bubble with legs 1 and 2 exchanged, B_t = ½ B^d + ½ X[B_a] (Sec. II.G.3 symmetries
of the spin sums):

- eager calls on odd and even grids: every class of channel t equals the oracle's t bubble
  (tolerance of the mixed path, 1e-6);
- the same three entries in a step graph (the finish waiting for the a context's branch)
  equal the eager calls;
- at the benchmark size the K3 class equals the ordinary mixed t bubble (1e-6);
- a slot not declared symmetric is refused."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CLS
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _engines(grids, nq, U, D, T, ch64):
    from paper_2405_20996_gb300.engine import Engine
    ea = Engine(grids, nq)
    et = Engine(grids, nq)
    for e in (ea, et):
        e.set_model(D, T)
    ea.set_vertex(0, U=U, has_R=True, channels=ch64, dtype=torch.complex64, symmetric=True)
    et.share_slot(0, ea, 0, U=U, has_R=True, symmetric=True)
    ea.alloc_out(1, channels=(0,), dtype=torch.complex64)
    et.alloc_out(1, channels=(2,), dtype=torch.complex64)
    return ea, et


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("grids", [dict(n1=21, n2w=9, n2v=9, n3w=7, n3v=7), dict(n1=20, n2w=8, n2v=10, n3w=6, n3v=8)])
def test_t_su2_matches_oracle(grids):
    nq, U, D, T = 81, 1.0, 1.0, 0.1
    ch = S.seeded_vertex(grids, U, seed=11)
    ch64 = {c: tuple(a.astype(np.complex64) for a in v) for c, v in ch.items()}
    ea, et = _engines(grids, nq, U, D, T, ch64)
    ea.bubble(0, 0, 0, 1, precision="mixed")
    et.bubble_t_su2(0, 1)
    et.t_su2_finish(1, ea.out(1, 0)["K3"])
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in et.out(1, 2).items()}
    V = O.Vertex(grids, U=U, has_R=True,
                 channels={c: tuple(a.astype(np.complex128) for a in v) for c, v in ch64.items()})
    ref = O.bubble_all(V, V, O.Prop(Delta=D, T=T), 2, nq)
    for name in CLS:
        assert _rel(got[name], ref[name]) <= 1e-6, (grids, name, _rel(got[name], ref[name]))
    ea.close()
    et.close()


def test_t_su2_step_graph_equals_eager():
    from paper_2405_20996_gb300.engine import StepGraph
    grids = dict(n1=21, n2w=9, n2v=9, n3w=7, n3v=9)
    nq, U, D, T = 81, 1.0, 1.0, 0.1
    ch = S.seeded_vertex(grids, U, seed=12)
    ch64 = {c: tuple(a.astype(np.complex64) for a in v) for c, v in ch.items()}
    ea, et = _engines(grids, nq, U, D, T, ch64)
    ea.bubble(0, 0, 0, 1, precision="mixed")
    et.bubble_t_su2(0, 1)
    et.t_su2_finish(1, ea.out(1, 0)["K3"])
    torch.cuda.synchronize()
    eager = {k: v.clone() for k, v in et.out(1, 2).items()}
    for v in et.out(1, 2).values():
        v.zero_()
    g = StepGraph([ea.desc(0, 0, 0, 1, precision="mixed"), et.desc_t_su2(0, 1), et.desc_t_su2_finish(1, ea, 1)])
    g.launch()
    torch.cuda.synchronize()
    for k, v in et.out(1, 2).items():
        assert torch.equal(v, eager[k]), k
    ea.close()
    et.close()


def test_t_su2_full_size_equals_the_ordinary_t_bubble():
    from paper_2405_20996_gb300.engine import Engine
    grids = dict(n1=401, n2w=101, n2v=101, n3w=51, n3v=51)
    nq, U, D, T = 4001, 2.0, 1.0, 0.05
    ch = S.seeded_vertex(grids, U, seed=13)
    ch64 = {c: tuple(a.astype(np.complex64) for a in v) for c, v in ch.items()}
    ea, et = _engines(grids, nq, U, D, T, ch64)
    ea.bubble(0, 0, 0, 1, precision="mixed")
    et.bubble_t_su2(0, 1)
    et.t_su2_finish(1, ea.out(1, 0)["K3"])
    torch.cuda.synchronize()
    su2 = et.out(1, 2)["K3"].cpu().numpy()
    ref_e = Engine(grids, nq)
    ref_e.set_model(D, T)
    ref_e.share_slot(0, ea, 0, U=U, has_R=True, symmetric=True)
    ref_e.alloc_out(1, channels=(2,), dtype=torch.complex64)
    ref_e.bubble(2, 0, 0, 1, precision="mixed")
    torch.cuda.synchronize()
    ref = ref_e.out(1, 2)["K3"].cpu().numpy()
    assert _rel(su2, ref) <= 1e-6, _rel(su2, ref)
    for e in (ea, et, ref_e):
        e.close()


def test_t_su2_refuses_a_slot_not_declared_symmetric():
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine
    grids = dict(n1=21, n2w=9, n2v=9, n3w=7, n3v=7)
    e = Engine(grids, 81)
    e.set_model(1.0, 0.1)
    ch = S.seeded_vertex(grids, 1.0, seed=14)
    e.set_vertex(0, U=1.0, has_R=True, channels={c: tuple(a.astype(np.complex64) for a in v) for c, v in ch.items()},
                 dtype=torch.complex64, symmetric=False)
    e.alloc_out(1, channels=(2,), dtype=torch.complex64)
    with pytest.raises(kb.KBError):
        e.bubble_t_su2(0, 1)
    e.close()
