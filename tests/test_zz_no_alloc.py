"""The allocation-free entry point kb_bubble_fp64_noalloc.

Some callers cannot call cudaMalloc: their device memory is owned by a pool or a host
program that reserved it all, or they must not trigger an allocation in the middle of
their own work.  For them the library offers one entry point whose scratch lives in a
fixed device array inside the library image.  This test calls it through the C ABI twice
in a row and compares each result with the ordinary kb_bubble (FP64) result; it also
checks that a problem too large for the fixed array is refused without running anything.
It is collected last so that a failure here never hides another test's result.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from helpers import CLS, RAGGED, rel_err, seeded_inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _desc(kb, tensors, has_R, U, include=(0, 1, 2)):
    d = kb.kb_vertex_desc()
    d.has_R, d.U, d.channels = int(has_R), U, sum(1 << c for c in include)
    for (ch, k), t in tensors.items():
        d.cls[ch][k] = t.data_ptr()
        d.dtype[ch][k] = kb.KB_DT_C128 if t.dtype == torch.complex128 else kb.KB_DT_C64
    return d


def test_noalloc_matches_kb_bubble_twice():
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    ch = seeded_inputs(cfg, seed=31)
    eng = Engine(g, cfg["nq"])
    eng.set_model(cfg["Delta"], cfg["T"])
    eng.set_vertex(0, U=cfg["U"], has_R=True, channels=ch)
    eng.alloc_out(1)
    gd = kb.kb_grid_desc(g["n1"], g["n2w"], g["n2v"], g["n3w"], g["n3v"], cfg["nq"], 5.0)
    desc = _desc(kb, eng.tensors[0], True, cfg["U"])
    stream = torch.cuda.current_stream().cuda_stream
    for r in range(3):
        eng.bubble(r, 0, 0, 1)
        torch.cuda.synchronize()
        ref = {k: v.cpu().numpy() for k, v in eng.out(1, r).items()}
        shapes = eng.class_shapes()
        for call in range(2):
            for k, name in enumerate(CLS):
                out = torch.full(shapes[name], 3.0 + 1.0j, dtype=torch.complex128, device="cuda")
                st = kb.kb_bubble_fp64_noalloc(gd, cfg["Delta"], cfg["T"], 0.0, desc, desc, r, kb.KB_PI_GG, k,
                                               out.data_ptr(), kb.KB_DT_C128, 1.0, 0.0, stream)
                assert st == kb.KB_OK
                torch.cuda.synchronize()
                got = out.cpu().numpy()
                assert rel_err(got, ref[name]) <= TOL, (r, name, call, rel_err(got, ref[name]))
    eng.close()


def test_noalloc_rejects_oversized_problem():
    from paper_2405_20996_gb300 import kb
    gd = kb.kb_grid_desc(401, 101, 101, 51, 51, 4001, 5.0)
    d = kb.kb_vertex_desc()
    d.has_R, d.U, d.channels = 1, 1.0, 7
    out = torch.zeros((51, 51, 51, 16), dtype=torch.complex128, device="cuda")
    st = kb.kb_bubble_fp64_noalloc(gd, 1.0, 0.1, 0.0, d, d, 0, kb.KB_PI_GG, kb.KB_K3, out.data_ptr(),
                                   kb.KB_DT_C128, 1.0, 0.0, 0)
    assert st == kb.KB_ERR_TOO_LARGE
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
