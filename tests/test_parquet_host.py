"""Host logic of the parquet solvers, on the CPU with stand-in maps (no library calls):

- restarted GMRES against a dense solve, for a nonsymmetric complex matrix, with restarts;
- the damped fixed point and inexact Newton-Krylov on a small quadratic map
  B(γ) = c + Q(γ, γ) (the bilinear structure of the Bethe-Salpeter right-hand side, with
  J v = v - Q(v, γ) - Q(γ, v)): both reach the same fixed point, Newton-Krylov in a handful
  of steps with its residual falling faster than linearly;
- Anderson acceleration: with no memory it is the damped iteration step for step; on an
  affine map with undamped updates and memory at least the dimension it terminates like
  GMRES (Walker and Ni, Theorem 2.2); on the quadratic map it needs fewer right-hand sides
  than the damped iteration and reaches the same fixed point;
- the Schwinger–Dyson self-energy's a and p forms and their mean issue the right bubbles and
  combine the loops with the right weights (stand-in context)."""

import numpy as np
import torch

from paper_2405_20996_gb300.parquet import ParquetPA


def test_gmres_matches_dense_solve():
    rng = np.random.default_rng(0)
    n = 120
    A = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    At = torch.from_numpy(A)
    x, its, res = ParquetPA._gmres(lambda v: At @ v, torch.from_numpy(b), 1e-12, 15, 400)
    assert res <= 1e-12 and its > 15                      # converged, with at least one restart
    ref = np.linalg.solve(A, b)
    assert np.abs(x.numpy() - ref).max() <= 1e-10 * np.abs(ref).max()


class _Toy(ParquetPA):
    """Stand-in with B(γ) = c + Q(γ, γ) on C^n."""

    def __init__(self, n=12, seed=1, scale=0.15):
        rng = np.random.default_rng(seed)
        self.T = torch.from_numpy((rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))) * scale / n)
        self.c = torch.from_numpy(rng.standard_normal(n) + 1j * rng.standard_normal(n))
        self.gamma = torch.zeros(n, dtype=torch.complex128)
        self.bubbles = 0

    def Q(self, x, y):
        return torch.einsum("ijk,j,k->i", self.T, x, y)

    def bse(self, g):
        self.bubbles += 1
        return self.c + self.Q(g, g)

    def jvp(self, g, v):
        return v - self.Q(v, g) - self.Q(g, v)


def test_fixed_point_and_newton_krylov_on_a_quadratic_map():
    toy = _Toy()
    g_fp, h_fp = toy.fixed_point(mix=0.5, tol=1e-13, maxit=2000)
    assert h_fp[-1] <= 1e-13
    g_nk, h_nk, lin = toy.newton_krylov(tol=1e-13, gmres_m=12)
    assert h_nk[-1] <= 1e-13 and len(h_nk) <= 8, h_nk
    assert torch.abs(g_fp - g_nk).max() <= 1e-11 * torch.abs(g_fp).max()
    # fixed point of the map itself
    assert torch.abs(toy.c + toy.Q(g_nk, g_nk) - g_nk).max() <= 1e-12 * torch.abs(g_nk).max()
    # faster than linear: each late step gains more than the previous one
    r = [x for x in h_nk if x > 0]
    assert r[-2] < r[-3] ** 1.5 or r[-2] < 1e-9, h_nk


class _Affine(ParquetPA):
    """Stand-in with B(γ) = c + A γ (spectral radius 0.9) on C^n."""

    def __init__(self, n=8, seed=2):
        rng = np.random.default_rng(seed)
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        A *= 0.9 / np.abs(np.linalg.eigvals(A)).max()
        self.A = torch.from_numpy(A)
        self.c = torch.from_numpy(rng.standard_normal(n) + 1j * rng.standard_normal(n))
        self.gamma = torch.zeros(n, dtype=torch.complex128)
        self.bubbles = 0
        self.sol = torch.from_numpy(np.linalg.solve(np.eye(n) - A, self.c.numpy()))

    def bse(self, g):
        self.bubbles += 1
        return self.c + self.A @ g


def test_anderson_without_memory_is_the_damped_iteration():
    a, b = _Toy(), _Toy()
    _, h_fp = a.fixed_point(mix=0.4, tol=0.0, maxit=25)
    g_aa, h_aa = b.anderson(mix=0.4, m=0, tol=0.0, maxit=25)
    assert h_aa == h_fp


def test_anderson_terminates_like_gmres_on_an_affine_map():
    aff = _Affine(n=8)
    g, h = aff.anderson(mix=1.0, m=20, tol=1e-12, maxit=40)
    assert h[-1] <= 1e-12 and len(h) <= 8 + 3, h
    assert torch.abs(g - aff.sol).max() <= 1e-10 * torch.abs(aff.sol).max()
    # the damped iteration contracts only by the spectral radius per step
    _, h_fp = _Affine(n=8).fixed_point(mix=1.0, tol=1e-12, maxit=40)
    assert h_fp[-1] > 1e-6


def test_anderson_on_the_quadratic_map():
    toy = _Toy()
    g_fp, h_fp = toy.fixed_point(mix=0.5, tol=1e-13, maxit=2000)
    n_fp = toy.bubbles
    toy.bubbles = 0
    g_aa, h_aa = toy.anderson(mix=0.5, m=5, tol=1e-13, maxit=2000)
    assert h_aa[-1] <= 1e-13 and toy.bubbles <= 0.6 * n_fp, (toy.bubbles, n_fp)
    assert torch.abs(g_aa - g_fp).max() <= 1e-11 * torch.abs(g_fp).max()


class _SDEEngine:
    """Stand-in for the context of ParquetSDE.sde: records bubbles and returns loops that
    depend on the slot and on whether the up-down vertex alone is asked for."""

    def __init__(self, n):
        self.n, self.calls = n, []

    def bubble(self, r, sl, sr, so, precision="fp64"):
        self.calls.append(("bubble", r, sl, sr, so))

    def loop(self, slot, nus, ud_only=False, line=None):
        self.calls.append(("loop", slot, ud_only))
        v = {10: 1.0, 11: 3.0, 12: 5.0, 13: 11.0}[slot] * (7.0 if ud_only else 1.0)
        out = torch.zeros((self.n, 2, 2), dtype=torch.complex128)
        out[:, 1, 0], out[:, 1, 1] = v, 1j * v
        return out


def test_sde_forms_combine_the_loops():
    from paper_2405_20996_gb300.parquet import S_GAMMA, S_RHAT, S_X, S_XP, S_XT, ParquetSDE
    # the t form takes loop - loop_ud of its slot (the up-up loop)
    tt = 11.0 - 7 * 11.0
    for form, expect in (("a", 1.0 + 0.5 * 3.0), ("p", 1.0 + 7 * 5.0), ("ap", 1.0 + 0.5 * (7 * 3.0 + 7 * 5.0)),
                         ("t", 1.0 + tt), ("apt", 1.0 + (7 * 3.0 + 7 * 5.0 + tt) / 3)):
        pa = ParquetSDE.__new__(ParquetSDE)
        pa.form, pa.U, pa.bubbles = form, 2.0, 0
        pa.sig_grid = np.linspace(-1.0, 1.0, 3)
        pa.gamma = torch.zeros(4, dtype=torch.complex128)
        pa.e = _SDEEngine(3)
        sR, sK = pa.sde(torch.ones(4, dtype=torch.complex128))
        assert torch.allclose(sR, torch.full((3,), 2.0 * expect, dtype=torch.complex128)), (form, sR)
        assert torch.allclose(sK, torch.full((3,), 2.0j * expect, dtype=torch.complex128))
        bubbles = [c for c in pa.e.calls if c[0] == "bubble"]
        want = {"a": [(0, S_X)], "p": [(1, S_XP)], "ap": [(0, S_X), (1, S_XP)], "t": [(0, S_X), (2, S_XT)],
                "apt": [(0, S_X), (1, S_XP), (2, S_XT)]}[form]
        assert [(c[1], c[4]) for c in bubbles] == want
        assert all(c[2] == S_RHAT and c[3] == S_GAMMA for c in bubbles)
        assert pa.bubbles == len(want)
