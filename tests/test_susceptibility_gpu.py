"""Susceptibilities on the GPU: the K1 readout kernel (kb_susceptibility_k1) equals the
host formulas of observables.py for the a, p and t (charge) channels, and the leg contraction
built from library bubbles (Engine.susceptibility_legs) equals the oracle's
oracle_susc.chi_legs element by element (FP64 path; the mixed path within 1e-6)."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import RAGGED
from oracle import oracle as O
from oracle import oracle_susc as OS
from paper_2405_20996_gb300.observables import charge_susceptibility_from_K1, susceptibility_from_K1

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_k1_readout_matches_host_formulas(dtype):
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=801)
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch, dtype=dtype)
    U = 1.7
    k1 = {r: e.tensors[0][(r, 0)].to(torch.complex128).cpu().numpy() for r in range(3)}
    for r in (0, 1):
        got = e.susceptibility(r, 0, U).cpu().numpy()
        rR, rK = susceptibility_from_K1(k1[r], r, U)
        assert np.abs(got[:, 0] - rR).max() <= 1e-14 * np.abs(rR).max()
        assert np.abs(got[:, 1] - rK).max() <= 1e-14 * np.abs(rK).max()
    got = e.susceptibility(2, 0, U).cpu().numpy()
    rR, rK = charge_susceptibility_from_K1(k1[2], k1[0], U)
    assert np.abs(got[:, 0] - rR).max() <= 1e-14 * np.abs(rR).max()
    assert np.abs(got[:, 1] - rK).max() <= 1e-14 * np.abs(rK).max()
    e.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("r", [0, 1])
def test_leg_contraction_matches_oracle(precision, r):
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=802)
    dt = torch.complex64 if precision == "mixed" else torch.complex128
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"])
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch, dtype=dt)
    got = e.susceptibility_legs(r, 0, precision=precision).cpu().numpy()
    if precision == "mixed":
        ch = {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}
    V = O.Vertex(g, U=cfg["U"], has_R=True, channels=ch)
    rR, rK = OS.chi_legs(V, O.Prop(Delta=cfg["Delta"], T=cfg["T"]), r, cfg["nq"])
    tol = 1e-10 if precision == "fp64" else 1e-6
    assert np.abs(got[:, 0] - rR).max() <= tol * np.abs(rR).max(), np.abs(got[:, 0] - rR).max() / np.abs(rR).max()
    assert np.abs(got[:, 1] - rK).max() <= tol * np.abs(rK).max(), np.abs(got[:, 1] - rK).max() / np.abs(rK).max()
    e.close()
