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


def test_one_loop_flow_of_the_self_energy_is_second_order_at_weak_coupling():
    """The one-loop flow of (γ, Σ) with Σ-dot = loop(Γ, S) and the Katanin substitution is
    exact to second order in U, and at particle-hole symmetry Σ has no third order: Σ/U² at
    U = 0.25 and 0.5 extrapolated in U² equals the second-order self-energy, whose Im Σ^R is
    the textbook double spectral integral; the flowed Σ is causal and obeys the FDR."""
    from paper_2405_20996_gb300.flow import VertexFlow
    from test_oracle_loop import _sigma2_spectral
    grids = dict(n1=201, n2w=9, n2v=9, n3w=5, n3v=5)
    nq, D, T, n_sig = 801, 1.0, 0.1, 41
    per_u2 = {}
    for U in (0.25, 0.5):
        fl = VertexFlow(grids, nq, U, D, T, n_loops=1, n_sig=n_sig)
        y, acc, rej = fl.integrate(1e-3, 1.0, h0=0.05, rtol=1e-7, atol=1e-13)
        sR, sK = (t.cpu().numpy() for t in fl.sigma(y))
        per_u2[U] = (sR / U ** 2, sK / U ** 2)
        nu = fl.sig_grid
        print("U = %.2f: %d steps (%d rejected), %d right-hand sides" % (U, acc, rej, fl.rhs_calls))
        fl.close()
    ext = (4 * per_u2[0.25][0] - per_u2[0.5][0]) / 3
    pick = (np.abs(nu) >= 0.3) & (np.abs(nu) <= 3.0)
    ref = _sigma2_spectral(nu[pick], 1.0, T, D)
    err = np.abs(ext[pick].imag - ref).max() / np.abs(ref).max()
    print("Im Sigma/U^2 extrapolated vs second order: max rel. deviation %.2e" % err)
    assert err <= 0.02, err
    sR, sK = per_u2[0.5]
    assert (sR.imag <= 1e-12).all()
    # the FDR holds where the vertex grids reach (the outermost Sigma points, |v| ~ 67, see the
    # K2 and K3 classes only through their interpolation to zero at x = +-1)
    inside = np.abs(nu) <= 10.0
    fdr = 2j * np.tanh(nu / (2 * T)) * sR.imag
    assert np.abs(sK - fdr)[inside].max() <= 1e-2 * np.abs(sR).max()
    assert np.abs(sR + np.conj(sR[::-1])).max() <= 1e-10 * np.abs(sR).max()     # particle-hole symmetry
