"""Parquet approximation with the self-energy from the Schwinger–Dyson equation (ParquetSDE):

- the joint map (Bethe–Salpeter right-hand sides and SDE self-energy at G[Σ]) equals the
  oracle's composition element by element: oracle bubbles with a Σ table, and
  Σ = U [loop(R̂) + ½ loop(X̂)], X̂ = B_a(R̂, Γ) in a channel-a-only vertex;
- weak coupling: the self-consistent Σ has no third order at particle-hole symmetry, so Σ/U²
  at U = 0.25 and 0.5 extrapolated in U² is the second-order self-energy, whose Im Σ^R is the
  textbook double spectral integral; the solution is causal and obeys the FDR;
- the Jacobian product of the joint map (vertex directions and the propagators' change
  along δΣ) equals central differences of the map, for the a, p, ap, t and apt forms and the
  symmetrised Bethe–Salpeter form, and Newton–Krylov on the joint state reaches the
  Anderson-accelerated fixed point."""

import numpy as np
import pytest
import torch

import seeded as S
from helpers import CLS
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def test_sde_map_matches_oracle():
    from paper_2405_20996_gb300.parquet import ParquetSDE
    g = dict(n1=13, n2w=7, n2v=6, n3w=5, n3v=4)
    nq, U, D, T, n_sig = 81, 1.2, 1.0, 0.15, 15
    pa = ParquetSDE(g, nq, U, D, T, n_sig=n_sig)
    ch = S.seeded_vertex(g, U, seed=41)
    sR = S.seeded_sigma(n_sig, seed=42)
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
            x = got[name].cpu().numpy()
            assert np.abs(x - ref[name]).max() <= 1e-10 * max(np.abs(ref[name]).max(), 1e-300), (r, name)
    Rh = O.Vertex(g, U=1.0, has_R=True)
    X = O.bubble_all(Rh, Gam, P, 0, nq)
    VX = O.Vertex(g, channels={0: tuple(X[name] for name in CLS)}, include=(0,))
    s = U * (O.loop(Rh, P, nq, pa.sig_grid) + 0.5 * O.loop(VX, P, nq, pa.sig_grid))
    scale = np.abs(s).max()
    assert np.abs(oR.cpu().numpy() - s[:, 1, 0]).max() <= 1e-10 * scale
    assert np.abs(oK.cpu().numpy() - s[:, 1, 1]).max() <= 1e-10 * scale
    pa.close()


def test_self_consistent_parquet_is_second_order_at_weak_coupling():
    from paper_2405_20996_gb300.parquet import ParquetSDE
    from test_oracle_loop import _sigma2_spectral
    grids = dict(n1=201, n2w=33, n2v=33, n3w=5, n3v=5)
    nq, D, T, n_sig = 801, 1.0, 0.1, 41
    per_u2 = {}
    for U in (0.25, 0.5):
        pa = ParquetSDE(grids, nq, U, D, T, n_sig=n_sig)
        z, hist = pa.anderson(mix=0.7, m=5, tol=1e-11, maxit=200)
        assert hist[-1] <= 1e-11, hist[-5:]
        _, sR, sK = pa.split(z)
        per_u2[U] = (sR.cpu().numpy() / U ** 2, sK.cpu().numpy() / U ** 2)
        nu = pa.sig_grid
        print("U = %.2f: %d iterations, %d bubbles" % (U, len(hist), pa.bubbles))
        pa.close()
    ext = (4 * per_u2[0.25][0] - per_u2[0.5][0]) / 3
    pick = (np.abs(nu) >= 0.3) & (np.abs(nu) <= 3.0)
    ref = _sigma2_spectral(nu[pick], 1.0, T, D)
    err = np.abs(ext[pick].imag - ref).max() / np.abs(ref).max()
    print("Im Sigma/U^2 extrapolated vs second order: max rel. deviation %.2e" % err)
    assert err <= 0.02, err
    sR, sK = per_u2[0.5]
    assert (sR.imag <= 1e-12).all()
    # the FDR holds up to the discretisation of the vertex's K2-type classes (on the oracle at
    # U = 0.5: 7.5 %, 3.9 %, 1.2 % of max |Sigma^R| for K2 grids 9, 17, 33)
    inside = np.abs(nu) <= 10.0
    fdr = 2j * np.tanh(nu / (2 * T)) * sR.imag
    assert np.abs(sK - fdr)[inside].max() <= 3e-2 * np.abs(sR).max()
    assert np.abs(sR + np.conj(sR[::-1])).max() <= 1e-10 * np.abs(sR).max()


def _seeded_state(pa, g, U, T, seed):
    ch = S.seeded_vertex(g, 0.5 * U, seed=seed)
    sR = 0.3 * S.seeded_sigma(pa.n_sig, seed=seed + 1)
    sK = 2j * np.tanh(S.grid_freqs(pa.n_sig) / (2 * T)) * sR.imag
    z = pa._zero_state()
    gam, zr, zk = pa.split(z)
    for c in range(3):
        for k, name in enumerate(CLS):
            pa.classes(gam, c)[name].copy_(torch.from_numpy(ch[c][k]))
    zr.copy_(torch.from_numpy(sR))
    zk.copy_(torch.from_numpy(sK))
    return z


@pytest.mark.parametrize("form,sym", [("a", False), ("p", False), ("ap", False), ("t", False), ("apt", False),
                                      ("a", True)])
def test_sde_jacobian_matches_central_differences(form, sym):
    from paper_2405_20996_gb300.parquet import ParquetSDE
    g = dict(n1=13, n2w=7, n2v=6, n3w=5, n3v=4)
    nq, U, D, T, n_sig = 81, 1.0, 1.0, 0.15, 15
    pa = ParquetSDE(g, nq, U, D, T, n_sig=n_sig, form=form, symmetric_bse=sym)
    z = _seeded_state(pa, g, U, T, 50)
    gen = torch.Generator().manual_seed(51)
    v = torch.randn(z.numel(), dtype=torch.complex128, generator=gen).to(pa.dev)
    v[pa.n:] *= 0.3
    h = 1e-4
    fd = ((z + h * v) - pa.bse(z + h * v) - ((z - h * v) - pa.bse(z - h * v))) / (2 * h)
    jv = pa.jvp(z, v)
    b_fd, r_fd, k_fd = pa.split(fd)
    b_jv, r_jv, k_jv = pa.split(jv)
    for a_, b_ in ((b_jv, b_fd), (r_jv, r_fd), (k_jv, k_fd)):
        err = float((a_ - b_).abs().max()) / float(b_.abs().max())
        assert err <= 1e-6, (form, sym, err)
    # the δΣ part is a genuine contribution (the map depends on Σ through every propagator)
    vs = v.clone()
    vs[:pa.n] = 0
    assert float((vs - pa.jvp(z, vs))[:pa.n].abs().max()) > 1e-3 * float(b_fd.abs().max())
    pa.close()


def test_sde_newton_krylov_reaches_the_fixed_point():
    from paper_2405_20996_gb300.parquet import ParquetSDE
    g = dict(n1=37, n2w=13, n2v=11, n3w=9, n3v=11)
    nq, U, D, T, n_sig = 201, 1.0, 1.0, 0.2, 21
    pa = ParquetSDE(g, nq, U, D, T, n_sig=n_sig)
    z_a, h_a = pa.anderson(mix=0.5, m=5, tol=1e-11, maxit=300)
    assert h_a[-1] <= 1e-11, h_a[-5:]
    n_a = pa.bubbles
    pa.bubbles = 0
    z_nk, h_nk, lin = pa.newton_krylov(tol=1e-11)
    assert h_nk[-1] <= 1e-11 and len(h_nk) <= 10, (h_nk, lin)
    assert pa.rel(z_nk - z_a, z_a) < 1e-9
    print("self-consistent parquet: Anderson %d iterations (%d bubbles); Newton-Krylov %d steps, GMRES %s "
          "(%d bubbles)" % (len(h_a), n_a, len(h_nk), lin, pa.bubbles))
    pa.close()
