"""GPU parity with the oracle of the self-energy parts of the flow and of the parquet solver:

- the multiloop flow's right-hand side (VertexFlow.rhs) at one state (γ, Σ) and one Λ of the
  interaction flow equals the oracle's mfrg_rhs element by element: the vertex derivative of
  every loop order with the Katanin substitution, and Σ-dot with, from three loops on, the
  t̄ and t terms iterated with the vertex step to self-consistency (Sec. III.C);
- the up-down-only line of the self-energy loop (kb_loop with KB_LOOP_UD_ONLY) equals the
  oracle's loop(ud_only=True);
- the Schwinger–Dyson self-energy in its p-channel form, its t-channel form and the means of
  forms (ParquetSDE form "p", "ap", "t", "apt") equals the oracle's composition of bubbles and
  up-down or up-up loops (Sec. III.B)."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CLS
from oracle import oracle as O
from oracle import oracle_flow as OF

pytestmark = pytest.mark.gpu

TOL = 1e-10
G_SMALL = dict(n1=13, n2w=7, n2v=6, n3w=5, n3v=4)


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.mark.parametrize("n_loops", [1, 3, 4])
def test_flow_rhs_matches_oracle(n_loops):
    from paper_2405_20996_gb300.flow import VertexFlow
    g, nq, U, D, T, n_sig, lam = G_SMALL, 41, 1.0, 1.0, 0.2, 9, 0.7
    fl = VertexFlow(g, nq, U, D, T, n_loops=n_loops, n_sig=n_sig, sigma_iters=40, sigma_tol=1e-13)
    ch = S.seeded_vertex(g, 0.5 * U, seed=700 + n_loops)
    sR = S.seeded_sigma(n_sig, seed=710 + n_loops)
    sK = 2j * np.tanh(fl.sig_grid / (2 * T)) * sR.imag
    y = torch.zeros(fl.size(), dtype=torch.complex128, device=fl.dev)
    views = fl.channels(y)
    for c in range(3):
        for k, name in enumerate(CLS):
            views[c][name].copy_(torch.from_numpy(ch[c][k]))
    yr, yk = fl.sigma(y)
    yr.copy_(torch.from_numpy(sR))
    yk.copy_(torch.from_numpy(sK))
    out = fl.rhs(lam, y)
    got = fl.channels(out)
    dR, dK = (t.cpu().numpy() for t in fl.sigma(out))
    gam = {c: [ch[c][k].copy() for k in range(4)] for c in range(3)}
    ref, rR, rK = OF.mfrg_rhs(g, nq, U, D, T, lam, gam, sR, sK, n_loops, OF.sig_grid(n_sig), iters=40,
                              tol=1e-13)
    assert np.allclose(OF.sig_grid(n_sig), fl.sig_grid, rtol=0, atol=1e-13)
    for c in range(3):
        for k, name in enumerate(CLS):
            e = _rel(got[c][name].cpu().numpy(), ref[c][k])
            assert e <= TOL, (n_loops, c, name, e)
    scale = max(np.abs(rR).max(), np.abs(rK).max())
    assert np.abs(dR - rR).max() <= TOL * scale, np.abs(dR - rR).max() / scale
    assert np.abs(dK - rK).max() <= TOL * scale, np.abs(dK - rK).max() / scale
    if n_loops >= 3:
        assert fl.sigma_iterations >= 2          # the multiloop terms were iterated
    fl.close()


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_loop_up_down_only_matches_oracle(dtype):
    from paper_2405_20996_gb300.engine import Engine
    g = dict(n1=37, n2w=13, n2v=11, n3w=9, n3v=11)
    nq, U, D, T = 201, 1.5, 1.0, 0.2
    ch = S.seeded_vertex(g, U, seed=720)
    e = Engine(g, nq)
    e.set_model(D, T, eps=0.3)
    e.set_vertex(0, U=U, has_R=True, channels=ch, dtype=dtype)
    if dtype == torch.complex64:
        ch = {c: tuple(a.astype(np.complex64).astype(np.complex128) for a in v) for c, v in ch.items()}
    V = O.Vertex(g, U=U, has_R=True, channels=ch)
    nus = np.concatenate([np.linspace(-6.0, 6.0, 25), [0.0, 1e-3, 35.0, -300.0, 2e4]])
    P = O.Prop(Delta=D, T=T, eps=0.3)
    got = e.loop(0, nus, ud_only=True).cpu().numpy()
    ref = O.loop(V, P, nq, nus, ud_only=True)
    assert _rel(got, ref) <= 1e-11, _rel(got, ref)
    # and with the single-scale line (the flow's loop(Γ, S))
    got_s = e.loop(0, nus, single_scale=True, ud_only=True).cpu().numpy()
    ref_s = O.loop(V, P, nq, nus, which=1, ud_only=True)
    assert _rel(got_s, ref_s) <= 1e-11, _rel(got_s, ref_s)
    # the full loop differs: the up-up part is not dropped there
    assert _rel(e.loop(0, nus).cpu().numpy(), ref) > 1e-3
    e.close()


@pytest.mark.parametrize("form", ["p", "ap", "t", "apt"])
def test_sde_forms_match_oracle(form):
    from paper_2405_20996_gb300.parquet import ParquetSDE
    g = G_SMALL
    nq, U, D, T, n_sig = 81, 1.2, 1.0, 0.15, 15
    pa = ParquetSDE(g, nq, U, D, T, n_sig=n_sig, form=form)
    ch = S.seeded_vertex(g, U, seed=730)
    sR = S.seeded_sigma(n_sig, seed=731)
    sK = 2j * np.tanh(S.grid_freqs(n_sig) / (2 * T)) * sR.imag
    z = pa._zero_state()
    gam, zr, zk = pa.split(z)
    for c in range(3):
        for k, name in enumerate(CLS):
            pa.classes(gam, c)[name].copy_(torch.from_numpy(ch[c][k]))
    zr.copy_(torch.from_numpy(sR))
    zk.copy_(torch.from_numpy(sK))
    out = pa.bse(z)
    b, oR, oK = pa.split(out)
    P = O.Prop(Delta=D, T=T, sigR=sR, sigK=sK)
    Gam = O.Vertex(g, U=U, has_R=True, channels=ch)
    for r in range(3):
        I_r = O.Vertex(g, U=U, has_R=True, channels=ch, include=[c for c in range(3) if c != r])
        ref = O.bubble_all(I_r, Gam, P, r, nq)
        got = pa.classes(b, r)
        for name in CLS:
            assert _rel(got[name].cpu().numpy(), ref[name]) <= TOL, (r, name)
    Rh = O.Vertex(g, U=1.0, has_R=True)
    if form in ("p", "ap"):
        s = U * O.loop(Rh, P, nq, pa.sig_grid)
        forms = {"p": (1,), "ap": (0, 1)}[form]
        for r in forms:
            X = O.bubble_all(Rh, Gam, P, r, nq)
            VX = O.Vertex(g, channels={r: tuple(X[name] for name in CLS)}, include=(r,))
            s = s + U / len(forms) * O.loop(VX, P, nq, pa.sig_grid, ud_only=True)
    else:
        s = OF.sde_map(g, nq, U, Gam, P, pa.sig_grid, form)
    scale = np.abs(s).max()
    assert np.abs(oR.cpu().numpy() - s[:, 1, 0]).max() <= TOL * scale
    assert np.abs(oK.cpu().numpy() - s[:, 1, 1]).max() <= TOL * scale
    pa.close()


def test_sde_t_form_fixed_point_matches_oracle():
    """The self-consistent parquet solution with the Schwinger–Dyson self-energy in the mean
    of its a, p and t forms: the GPU fixed point (Newton–Krylov on the joint state) equals the
    oracle's damped iteration (oracle_flow.parquet_sde(form="apt")) on small grids."""
    from paper_2405_20996_gb300.parquet import ParquetSDE
    g = G_SMALL
    nq, U, D, T, n_sig = 41, 1.0, 1.0, 0.2, 9
    pa = ParquetSDE(g, nq, U, D, T, n_sig=n_sig, form="apt")
    z, h, _ = pa.newton_krylov(tol=1e-12)
    assert h[-1] <= 1e-12, h
    gam, sR, _ = pa.split(z)
    og, osR, _ = OF.parquet_sde(g, nq, U, D, T, pa.sig_grid, tol=1e-13, maxit=2000, form="apt")
    assert _rel(sR.cpu().numpy(), osR) <= 1e-9
    for c in range(3):
        got = pa.classes(gam, c)
        for k, name in enumerate(CLS):
            assert _rel(got[name].cpu().numpy(), og[c][k]) <= 1e-9, (c, name)
    pa.close()
