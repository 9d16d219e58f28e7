"""Parity of the mixed-precision CUDA path (FP32 gather with double-float frequencies,
3xTF32 tcgen05 contraction for K3, FP64 propagators/Pi/tail) with the FP64 CPU oracle and
with the plain FP64 GPU path: relative max-norm per class <= 1e-6."""

import os

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CFG1, CLS, RAGGED, oracle_vertex, rel_err, seeded_inputs
from oracle import oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-6


def c64(ch):
    return {c: tuple(a.astype(np.complex64) for a in v) for c, v in ch.items()}


def c64_as_128(ch):
    return {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}


def gpu_bubble(cfg, ch, r, precision, pi_kind=0, left=None, sigma=None, out_dtype=torch.complex128, mask=0xF,
               symmetric=False):
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine
    e = Engine(cfg["grids"], cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    if sigma is not None:
        e.set_self_energy(*sigma)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=c64(ch), dtype=torch.complex64, symmetric=symmetric)
    sl = 0
    if left is not None:
        e.set_vertex(1, U=cfg["U"], has_R=False, channels=c64(left[0]), dtype=torch.complex64, include=left[1])
        sl = 1
    e.alloc_out(2, channels=(r,), dtype=out_dtype)
    e.bubble(r, sl, 0, 2, pi_kind=pi_kind, precision=precision, class_mask=mask)
    kb.kb_check_device(e.ctx)
    out = {k: v.cpu().numpy() for k, v in e.out(2, r).items()}
    e.close()
    return out


@pytest.mark.parametrize("r", [0, 1, 2])
def test_mixed_ragged_vs_oracle(r):
    cfg = RAGGED
    ch = seeded_inputs(cfg, seed=41)
    got = gpu_bubble(cfg, ch, r, "mixed")
    V = oracle_vertex(cfg, c64_as_128(ch))
    ref = O.bubble_all(V, V, O.Prop(Delta=cfg["Delta"], T=cfg["T"]), r, cfg["nq"])
    for k in CLS:
        assert rel_err(got[k], ref[k]) <= TOL, (r, k, rel_err(got[k], ref[k]))


@pytest.mark.parametrize("r", [0, 2])
def test_mixed_pi_dot_sigma_loop_part(r):
    cfg = dict(RAGGED, T=0.07)
    g = cfg["grids"]
    ch = seeded_inputs(cfg, seed=43)
    dot = S.seeded_vertex(g, 0.5, seed=44)
    inc = tuple(c for c in range(3) if c != r)
    sg = O.grid(33)
    sR = S.seeded_sigma(33, seed=45)
    sK = 2j * np.tanh(sg / (2 * cfg["T"])) * sR.imag
    got = gpu_bubble(cfg, ch, r, "mixed", pi_kind=1, left=(dot, inc), sigma=(sR, sK))
    V = oracle_vertex(cfg, c64_as_128(ch))
    Vd = O.Vertex(g, has_R=False, channels=c64_as_128(dot), include=inc)
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], sigR=sR, sigK=sK)
    ref = O.bubble_all(Vd, V, P, r, cfg["nq"], pi_kind=O.PI_GS)
    for k in CLS:
        if np.abs(ref[k]).max() == 0:
            assert np.abs(got[k]).max() == 0
        else:
            assert rel_err(got[k], ref[k]) <= TOL, (k, rel_err(got[k], ref[k]))


def test_mixed_full_size_vs_fp64_gpu_and_oracle_samples():
    """The mixed-precision workload (K1 401, K2 101^2, K3 51^3, 4001 nodes, complex64
    vertex): every class of every channel within 1e-6 of the plain FP64 GPU path, and per
    class 64 random points plus the grid's corner points (first and last index on every
    axis) within 1e-6 (mixed) and 1e-10 (FP64) of the oracle."""
    cfg = CFG1
    ch = seeded_inputs(cfg, seed=1)
    rng = np.random.default_rng(0)
    V = oracle_vertex(cfg, c64_as_128(ch))
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"])
    shapes = {"K1": (401,), "K2": (101, 101), "K2p": (101, 101), "K3": (51, 51, 51)}
    for r in range(3):
        mx = gpu_bubble(cfg, ch, r, "mixed", symmetric=True)
        fp = gpu_bubble(cfg, ch, r, "fp64")
        for k in CLS:
            assert rel_err(mx[k], fp[k]) <= TOL, (r, k, rel_err(mx[k], fp[k]))
            corners = [tuple((n - 1) * ((c >> d) & 1) for d, n in enumerate(shapes[k]))
                       for c in range(1 << len(shapes[k]))]
            idx = corners + [tuple(int(rng.integers(0, n)) for n in shapes[k]) for _ in range(64)]
            ref = O.bubble_class(V, V, P, r, k, cfg["nq"], idx=idx)
            got = np.array([mx[k][i] for i in idx])
            scale = np.abs(fp[k]).max()
            assert np.abs(got - ref).max() <= TOL * scale, (r, k)
            gotf = np.array([fp[k][i] for i in idx])
            assert np.abs(gotf - ref).max() <= 1e-10 * scale, (r, k)


@pytest.mark.parametrize("shape", ["1", "0"], ids=["both-parts", "one-part"])
def test_tensor_core_contraction_matches_simt_reference(shape):
    """K3 through tcgen05 (3xTF32, segmented FP32 accumulation) vs the SIMT FP32
    reference contraction of the same tiles, in each tile shape of the tensor-core kernel
    (both parts of a 128 x 64 complex tile per CTA, or one part of a 128 x 128 tile)."""
    cfg = RAGGED
    ch = seeded_inputs(cfg, seed=47)
    os.environ["KB_TC_SHAPE"] = shape
    try:
        tc = gpu_bubble(cfg, ch, 2, "mixed", mask=8)
    finally:
        os.environ.pop("KB_TC_SHAPE", None)
    os.environ["KB_K3_SIMT"] = "1"
    try:
        simt = gpu_bubble(cfg, ch, 2, "mixed", mask=8)
    finally:
        os.environ.pop("KB_K3_SIMT", None)
    assert rel_err(tc["K3"], simt["K3"]) <= TOL
    assert np.abs(tc["K3"] - simt["K3"]).max() > 0      # the two contractions are distinct code


EVEN = dict(grids=dict(n1=36, n2w=12, n2v=10, n3w=8, n3v=10), nq=161, U=1.2, Delta=1.0, T=0.15)


@pytest.mark.parametrize("cfg", [RAGGED, EVEN], ids=["odd", "even"])
@pytest.mark.parametrize("r", [0, 1, 2])
def test_symmetric_mode_matches_full_and_oracle(cfg, r):
    """Kernel (d): for a conjugation- and crossing-symmetric vertex bubbled with itself only
    the independent part is computed and the rest filled by symmetry; the result equals
    the full computation and the oracle (odd and even grid sizes)."""
    ch = seeded_inputs(cfg, seed=51)
    sym = gpu_bubble(cfg, ch, r, "mixed", symmetric=True)
    full = gpu_bubble(cfg, ch, r, "mixed", symmetric=False)
    V = oracle_vertex(cfg, c64_as_128(ch))
    ref = O.bubble_all(V, V, O.Prop(Delta=cfg["Delta"], T=cfg["T"]), r, cfg["nq"])
    for k in CLS:
        assert rel_err(sym[k], full[k]) <= TOL, (r, k, rel_err(sym[k], full[k]))
        assert rel_err(sym[k], ref[k]) <= TOL, (r, k, rel_err(sym[k], ref[k]))
