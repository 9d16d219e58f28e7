"""Vertex flow of the multiloop fRG in the interaction flow (Σ held at 0): integrating
dγ/dΛ = Σ_{l ≤ n} γ̇^(l) from Λ ≈ 0 (γ = 0) to Λ = 1 with the Cash–Karp pair reproduces the
parquet solution at Λ = 1 (Sec. III.C: a converged multiloop flow equals the parquet
solution), the six-loop flow much better than the one-loop flow."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

CFG = dict(grids=dict(n1=37, n2w=13, n2v=11, n3w=9, n3v=11), nq=201, U=1.0, Delta=1.0, T=0.2)


def test_multiloop_flow_reproduces_the_parquet_solution():
    from paper_2405_20996_gb300.flow import VertexFlow
    from paper_2405_20996_gb300.parquet import ParquetPA
    c = CFG
    pa = ParquetPA(c["grids"], c["nq"], c["U"], c["Delta"], c["T"])
    g_pa, hist, _ = pa.newton_krylov(tol=1e-12)
    assert hist[-1] <= 1e-12
    ref = g_pa.clone()
    pa.close()
    err = {}
    for n in (1, 6):
        fl = VertexFlow(c["grids"], c["nq"], c["U"], c["Delta"], c["T"], n_loops=n)
        y, acc, rej = fl.integrate(1e-3, 1.0, h0=0.05, rtol=1e-5)
        assert acc > 3, (acc, rej)
        err[n] = float((y - ref).abs().max() / ref.abs().max())
        print("%d-loop flow: %d steps (%d rejected), %d right-hand sides, rel. deviation from parquet %.3e"
              % (n, acc, rej, fl.rhs_calls, err[n]))
        fl.close()
    assert err[6] <= 0.05, err
    assert err[6] < 0.5 * err[1], err
