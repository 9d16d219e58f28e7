"""Failure detection without a GPU fault:

- a bounded device-side wait that runs out (a one-CTA kernel waiting on a shared-memory
  barrier nothing arrives on, with a short test budget) is reported by kb_check_device as
  KB_ERR_TIMEOUT, the report is cleared once read, and the context keeps working;
- a workspace allocation that fails (injected on the host) returns KB_ERR_OOM before anything
  of that call is launched, and the next call succeeds;
- a step graph refuses to launch once a context's workspace was replaced after the capture
  (its kernels address the old buffer), and a new graph works."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CLS, RAGGED, rel_err
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _engine(cfg=RAGGED, dtype=torch.complex128, seed=91):
    from paper_2405_20996_gb300.engine import Engine
    e = Engine(cfg["grids"], cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    ch = S.seeded_vertex(cfg["grids"], cfg["U"], seed=seed)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch, dtype=dtype)
    e.alloc_out(1, dtype=dtype)
    return e, ch


def test_bounded_wait_runs_out_and_is_reported():
    from paper_2405_20996_gb300 import kb
    e, ch = _engine()
    kb.kb_check_device(e.ctx)                              # nothing pending
    kb.kb_set_wait_budget(e.ctx, 2_000_000)                # ~1 ms at the SM clock
    n0 = e.launches()
    kb.kb_check_wait(e.ctx)
    assert e.launches() == n0 + 1
    with pytest.raises(kb.KBError) as ex:
        kb.kb_check_device(e.ctx)
    assert ex.value.status == kb.KB_ERR_TIMEOUT
    kb.kb_check_device(e.ctx)                              # read once, then cleared
    kb.kb_set_wait_budget(e.ctx, 0)
    # the context still computes correctly
    e.bubble(0, 0, 0, 1)
    kb.kb_check_device(e.ctx)
    V = O.Vertex(RAGGED["grids"], U=RAGGED["U"], has_R=True, channels=ch)
    ref = O.bubble_class(V, V, O.Prop(Delta=RAGGED["Delta"], T=RAGGED["T"]), 0, "K2", RAGGED["nq"])
    assert rel_err(e.out(1, 0)["K2"].cpu().numpy(), ref) <= 1e-10
    e.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_injected_allocation_failure(precision):
    from paper_2405_20996_gb300 import kb
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    e, ch = _engine(dtype=dt, seed=92)
    assert kb.kb_workspace_bytes(e.ctx) == 0
    kb.kb_inject_alloc_failures(e.ctx, 1)
    n0 = e.launches()
    with pytest.raises(kb.KBError) as ex:
        e.bubble(2, 0, 0, 1, precision=precision)
    assert ex.value.status == kb.KB_ERR_OOM
    assert "injected" in str(ex.value)
    assert e.launches() == n0                              # nothing of the failed call ran
    assert kb.kb_workspace_bytes(e.ctx) == 0
    e.bubble(2, 0, 0, 1, precision=precision)              # the hook is used up
    kb.kb_check_device(e.ctx)
    assert kb.kb_workspace_bytes(e.ctx) > 0
    if precision == "mixed":
        ch = {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}
    V = O.Vertex(RAGGED["grids"], U=RAGGED["U"], has_R=True, channels=ch)
    ref = O.bubble_class(V, V, O.Prop(Delta=RAGGED["Delta"], T=RAGGED["T"]), 2, "K1", RAGGED["nq"])
    assert rel_err(e.out(1, 2)["K1"].cpu().numpy(), ref) <= (1e-10 if precision == "fp64" else 1e-6)
    e.close()


def test_graph_refuses_after_workspace_change():
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import StepGraph
    e, ch = _engine(seed=93)
    g = StepGraph([e.desc(1, 0, 0, 1, class_mask=1 << kb.KB_K1)])       # small workspace: K1 only
    g.launch()
    torch.cuda.synchronize()
    k1 = e.out(1, 1)["K1"].clone()
    before = kb.kb_workspace_bytes(e.ctx)
    e.bubble(1, 0, 0, 1)                                   # all classes: the workspace grows
    torch.cuda.synchronize()
    assert kb.kb_workspace_bytes(e.ctx) > before
    with pytest.raises(kb.KBError) as ex:
        g.launch()
    assert ex.value.status == kb.KB_ERR_STATE
    g.close()
    g2 = StepGraph([e.desc(1, 0, 0, 1, class_mask=1 << kb.KB_K1)])
    g2.launch()
    torch.cuda.synchronize()
    assert torch.equal(e.out(1, 1)["K1"], k1)
    g2.close()
    e.close()
