"""Run in a child process with KB_CHECKED=1 (tests/test_checked_gpu.py): the bounds-checked
library variant through the C ABI on ragged and even grids — the FP64 and mixed bubbles of
every channel and class (the K2 gather, the tile gathers, K1), the self-energy loop, the
vertex evaluation and both adjoints — each followed by kb_check_device, which reports any
vertex record index from a frequency lookup that fell outside its class; spot parity with
the oracle on the checked library.  Prints one line "checked run ok: ..." on success."""

import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import seeded as S  # noqa: E402
from helpers import CLS, RAGGED, rel_err  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2405_20996_gb300 import kb  # noqa: E402
from paper_2405_20996_gb300.engine import Engine  # noqa: E402

EVEN = dict(grids=dict(n1=16, n2w=10, n2v=8, n3w=6, n3v=8), nq=81, U=1.0, Delta=1.0, T=0.1)


def run(cfg, seed):
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=seed)
    c64 = {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"], 0.1)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch)
    e.set_vertex(1, U=cfg["U"], has_R=True, channels=c64, dtype=torch.complex64)
    e.set_vertex(2, U=cfg["U"], has_R=True, channels=c64, dtype=torch.complex64, symmetric=True)
    e.alloc_out(3)
    e.alloc_out(4, dtype=torch.complex64)
    e.alloc_out(5, dtype=torch.complex64)
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], eps=0.1)
    checks = 0
    for r in range(3):
        e.bubble(r, 0, 0, 3)
        e.bubble(r, 1, 1, 4, precision="mixed")
        e.bubble(r, 2, 2, 5, precision="mixed")          # symmetric mode: K2 gather + symmetry images
        kb.kb_check_device(e.ctx)
        checks += 3
        for k, name in ((1, "K2"), (3, "K3")):
            ref = O.bubble_class(O.Vertex(g, U=cfg["U"], has_R=True, channels=ch), O.Vertex(g, U=cfg["U"], has_R=True, channels=ch),
                                 P, r, name, cfg["nq"])
            ref64 = O.bubble_class(O.Vertex(g, U=cfg["U"], has_R=True, channels=c64), O.Vertex(g, U=cfg["U"], has_R=True, channels=c64),
                                   P, r, name, cfg["nq"])
            assert rel_err(e.out(3, r)[name].cpu().numpy(), ref) <= 1e-10, (r, name)
            assert rel_err(e.out(4, r)[name].cpu().numpy(), ref64) <= 1e-6, (r, name)
            assert rel_err(e.out(5, r)[name].cpu().numpy(), ref64) <= 1e-6, (r, name)
    nus = np.linspace(-8.0, 8.0, 17)
    e.loop(0, nus)
    e.loop(0, nus, single_scale=True, ud_only=True)
    e.vertex_eval(0, 2, [[0.3, -1.0, 2.5], [0.0, 40.0, -0.2], [-3.0, 0.1, 0.1]])
    kb.kb_check_device(e.ctx)
    checks += 1
    # adjoints (gradient slots complex128)
    for s in (6, 7):
        e.alloc_out(s)
    for r in range(3):
        e.bubble_vjp(r, 0, 0, 3, grad_left=6, grad_right=6, grad_gr=e.gr_tables())
        e.bubble_vjp(r, 1, 1, 4, grad_left=7, grad_right=7, grad_gr=e.gr_tables(), precision="mixed")
        kb.kb_check_device(e.ctx)
        checks += 2
    e.close()
    return checks


def main():
    assert kb.lib().kb_build_checked() == 1, "not the bounds-checked library"
    n = run(RAGGED, 11) + run(EVEN, 12)
    print("checked run ok: %d checks, no out-of-range record access" % n)


if __name__ == "__main__":
    main()
