"""The largest single-instance workload (K1 801, K2 201^2, K3 101^3, Nq 8001, 16 Keldysh
components, complex64 vertex of all three channels, about 430 MB): the mixed-precision
bubble of every channel and class, symmetric mode, checked against the FP64 oracle at
seeded random output points and at the GPU result's largest point (relative to the class's
max-norm, taken from the oracle's values, <= 1e-6) and, for K1, in
full against the plain FP64 GPU path."""

import numpy as np
import pytest
import torch

import seeded as S
from oracle import oracle as O

pytestmark = pytest.mark.gpu

CFG4 = dict(grids=dict(n1=801, n2w=201, n2v=201, n3w=101, n3v=101), nq=8001, U=3.0, Delta=1.0, T=0.01)
TOL = 1e-6
NSAMPLE = {"K1": 64, "K2": 48, "K2p": 48, "K3": 96}


@pytest.fixture(scope="module")
def large_case():
    from paper_2405_20996_gb300.engine import Engine
    cfg = CFG4
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=400)
    ch64 = {c: tuple(a.astype(np.complex64) for a in v) for c, v in ch.items()}
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    e.set_workspace_limit(8 << 30)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch64, dtype=torch.complex64, symmetric=True)
    e.alloc_out(1, dtype=torch.complex64)
    for r in range(3):
        e.bubble(r, 0, 0, 1, precision="mixed")
    torch.cuda.synchronize()
    out = {r: {k: v.cpu().numpy() for k, v in e.out(1, r).items()} for r in range(3)}
    # plain FP64 GPU K1 of every channel (complex128 output slot)
    e.alloc_out(2, dtype=torch.complex128, classes=(0,))
    for r in range(3):
        e.bubble(r, 0, 0, 2, precision="fp64", class_mask=1)
    torch.cuda.synchronize()
    k1_fp64 = {r: e.out(2, r)["K1"].cpu().numpy() for r in range(3)}
    e.close()
    V = O.Vertex(g, U=cfg["U"], has_R=True,
                 channels={c: tuple(a.astype(np.complex128) for a in v) for c, v in ch64.items()})
    return out, k1_fp64, V


@pytest.mark.parametrize("r", [0, 1, 2])
def test_large_mixed_vs_oracle_sampled(large_case, r):
    out, _, V = large_case
    cfg = CFG4
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"])
    rng = np.random.default_rng(500 + r)
    for cls, n in NSAMPLE.items():
        got = out[r][cls]
        shp = got.shape[:-1]
        idx = [tuple(int(rng.integers(0, m)) for m in shp) for _ in range(n)]
        # plus the point where the GPU result is largest, so that the oracle's own values
        # give the class's max-norm (its value there is within the tolerance of the maximum)
        idx.append(tuple(int(i) for i in np.unravel_index(np.abs(got).max(axis=-1).argmax(), shp)))
        ref = O.bubble_class(V, V, P, r, cls, cfg["nq"], idx=idx)
        scale = max(np.abs(ref[q]).max() for q in range(len(idx)))
        err = max(np.abs(got[i] - ref[q]).max() for q, i in enumerate(idx)) / scale
        assert err <= TOL, (r, cls, err)


@pytest.mark.parametrize("r", [0, 1, 2])
def test_large_k1_mixed_vs_fp64_gpu(large_case, r):
    out, k1, _ = large_case
    ref = k1[r]
    err = np.abs(out[r]["K1"] - ref).max() / np.abs(ref).max()
    assert err <= TOL, (r, err)
