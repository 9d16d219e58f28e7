"""Self-energy loop on the GPU (kb_loop): the FP64 kernel equals the oracle's loop element by
element — seeded vertex with every class in the three channels, complex128 and complex64
classes, a channel-subset slot, a Sigma table, the interaction flow's scaled propagator,
the single-scale propagator of each flow scheme (with the Katanin substitution),
frequencies on, between and far beyond the grids — and the bare vertex alone gives the
Hartree shift U (n - 1/2)."""

import numpy as np
import pytest
import torch
from scipy import integrate

import seeded as S
from helpers import RAGGED
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _nus():
    g = O.grid(RAGGED["grids"]["n2v"])
    return np.concatenate([np.linspace(-7.0, 7.0, 29), g[:3], [0.0, 1e-3, 40.0, -250.0, 3e4]])


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("include", [(0, 1, 2), (0, 2)])
def test_loop_matches_oracle(dtype, include):
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=81)
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"], eps=0.25)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch, dtype=dtype, include=include)
    if dtype == torch.complex64:
        ch = {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}
    V = O.Vertex(g, U=cfg["U"], has_R=True, channels=ch, include=include)
    nus = _nus()
    got = e.loop(0, nus).cpu().numpy()
    ref = O.loop(V, O.Prop(Delta=cfg["Delta"], T=cfg["T"], eps=0.25), cfg["nq"], nus)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), np.abs(got - ref).max()
    e.close()


def test_loop_with_sigma_table_and_interaction_flow():
    from paper_2405_20996_gb300 import kb
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=82)
    sR = S.seeded_sigma(23, seed=6)
    sK = 2j * np.tanh(S.grid_freqs(23) / (2 * cfg["T"])) * sR.imag
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"], eps=-0.4)
    e.set_self_energy(sR, sK)
    e.set_regulator(kb.KB_REG_U, 0.6)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch)
    nus = _nus()
    got = e.loop(0, nus).cpu().numpy()
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], eps=-0.4, sigR=sR, sigK=sK, reg=O.REG_U, lam=0.6)
    ref = O.loop(O.Vertex(g, U=cfg["U"], has_R=True, channels=ch), P, cfg["nq"], nus)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), np.abs(got - ref).max()
    e.close()


def test_loop_of_bare_vertex_is_the_hartree_shift():
    from paper_2405_20996_gb300.engine import Engine
    U, D, T, eps = 1.3, 1.0, 0.1, 0.3
    g = RAGGED["grids"]
    e = Engine(g, 1001)
    e.set_model(D, T, eps=eps)
    e.set_vertex(0, U=U, has_R=True)
    got = e.loop(0, [0.0, 1.5, -4.0]).cpu().numpy()
    A = lambda v: (D / np.pi) / ((v - eps) ** 2 + D ** 2)
    n = integrate.quad(lambda v: 0.5 * (1 - np.tanh(v / (2 * T))) * A(v), -np.inf, np.inf,
                       epsabs=1e-14, epsrel=1e-14, limit=400)[0]
    assert np.abs(got[:, 1, 0] - U * (n - 0.5)).max() <= 1e-9 * U
    assert np.abs(got[:, 0, 1] - U * (n - 0.5)).max() <= 1e-9 * U
    assert np.abs(got[:, 0, 0]).max() <= 1e-12 and np.abs(got[:, 1, 1]).max() <= 1e-12
    e.close()


@pytest.mark.parametrize("reg,lam,katanin", [(0, 1.0, False), (1, 0.7, False), (2, 1.0, False), (0, 1.0, True)])
def test_single_scale_loop_matches_oracle(reg, lam, katanin):
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=83)
    sR = S.seeded_sigma(23, seed=6)
    sK = 2j * np.tanh(S.grid_freqs(23) / (2 * cfg["T"])) * sR.imag
    dR = S.seeded_sigma(19, seed=7) if katanin else None
    dK = 2j * np.tanh(S.grid_freqs(19) / (2 * cfg["T"])) * dR.imag if katanin else None
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"], eps=0.15)
    e.set_self_energy(sR, sK)
    e.set_regulator(reg, lam)
    if katanin:
        e.set_self_energy_derivative(dR, dK)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch)
    nus = _nus()
    got = e.loop(0, nus, single_scale=True).cpu().numpy()
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], eps=0.15, sigR=sR, sigK=sK, reg=reg, lam=lam, dsigR=dR, dsigK=dK)
    ref = O.loop(O.Vertex(g, U=cfg["U"], has_R=True, channels=ch), P, cfg["nq"], nus, which=1)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), np.abs(got - ref).max()
    e.close()


def test_loop_with_a_self_energy_insertion_matches_oracle():
    from paper_2405_20996_gb300.engine import Engine
    cfg = RAGGED
    g = cfg["grids"]
    ch = S.seeded_vertex(g, cfg["U"], seed=84)
    sR = S.seeded_sigma(23, seed=6)
    sK = 2j * np.tanh(S.grid_freqs(23) / (2 * cfg["T"])) * sR.imag
    dR = S.seeded_sigma(19, seed=9)
    dK = 2j * np.tanh(S.grid_freqs(19) / (2 * cfg["T"])) * dR.imag
    e = Engine(g, cfg["nq"])
    e.set_model(cfg["Delta"], cfg["T"], eps=0.15)
    e.set_self_energy(sR, sK)
    e.set_self_energy_derivative(dR, dK)
    e.set_vertex(0, U=cfg["U"], has_R=True, channels=ch)
    nus = _nus()
    got = e.loop(0, nus, line=2).cpu().numpy()
    P = O.Prop(Delta=cfg["Delta"], T=cfg["T"], eps=0.15, sigR=sR, sigK=sK, dsigR=dR, dsigK=dK)
    ref = O.loop(O.Vertex(g, U=cfg["U"], has_R=True, channels=ch), P, cfg["nq"], nus, which=2)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), np.abs(got - ref).max()
    e.close()
