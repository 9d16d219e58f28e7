"""Host logic of the flow's self-energy right-hand side, on the CPU with stand-in engines (no
library calls): from three loops on, Σ-dot = L(Γ, S) + L(γ̇^C_t̄, G) + L(Γ, G Σ-dot_t̄ G) is
iterated with the vertex step (whose central parts depend on the Katanin table) to its
self-consistent value; below three loops a single pass with Σ-dot = L(Γ, S)."""

import numpy as np
import torch

from paper_2405_20996_gb300.flow import VertexFlow
from paper_2405_20996_gb300.multiloop import S_GAMMA, s_central

N_SIG = 5
C_GAIN, D_GAIN = 0.3, 0.5          # central parts = C_GAIN * (Katanin table); t line = D_GAIN * insertion


def _t(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.complex128)


class _Engine:
    def __init__(self, ml):
        self.ml, self.dsig = ml, None

    def set_regulator(self, kind, lam):
        pass

    def set_self_energy(self, sR, sK, A):
        pass

    def set_self_energy_derivative(self, dR=None, dK=None, A=5.0):
        self.dsig = None if dR is None else (np.array(dR), np.array(dK))

    def _table(self):
        out = torch.zeros((N_SIG, 2, 2), dtype=torch.complex128)
        out[:, 1, 0], out[:, 1, 1] = _t(self.dsig[0]), _t(self.dsig[1])
        return out

    def loop(self, slot, nus, single_scale=False, line=None):
        if slot == S_GAMMA and single_scale:
            return self.ml.a.clone()
        if slot == S_GAMMA and line == 2:
            return D_GAIN * self._table()
        assert slot == s_central(self.ml.n_loops) and line is None and not single_scale
        return self.ml.central_val.clone()


class _Step:
    def __init__(self, n_loops):
        self.n_loops, self.keep_central, self.channels = n_loops, n_loops >= 3, (0, 1, 2)
        self.e = {r: _Engine(self) for r in range(3)}
        rng = np.random.default_rng(1)
        a = torch.zeros((N_SIG, 2, 2), dtype=torch.complex128)
        a[:, 1, 0] = _t(rng.standard_normal(N_SIG) - 1j * np.abs(rng.standard_normal(N_SIG)))
        a[:, 1, 1] = _t(1j * rng.standard_normal(N_SIG))
        self.a = a
        self.total = {(c, k): torch.zeros(2, dtype=torch.complex128) for c in range(3) for k in range(4)}
        self.runs = 0

    def zero(self):
        for t in self.total.values():
            t.zero_()

    def run_eager(self):
        # the vertex derivative and central parts follow the Katanin table every context holds
        tabs = [e.dsig for e in self.e.values()]
        assert all(np.array_equal(tabs[0][0], t[0]) for t in tabs)
        tab = self.e[0]._table()
        self.central_val = C_GAIN * tab
        for t in self.total.values():
            t += tab[:2, 1, 0]
        self.runs += 1


def _flow(n_loops):
    fl = VertexFlow.__new__(VertexFlow)
    fl.ml = _Step(n_loops)
    fl.gamma_t = [torch.zeros(2, dtype=torch.complex128) for _ in range(12)]
    fl.sizes = [2] * 12
    fl.n_gamma, fl.n_sig, fl.A = 24, N_SIG, 5.0
    fl.sig_grid = np.linspace(-2.0, 2.0, N_SIG)
    fl.dtype, fl.dev = torch.complex128, "cpu"
    fl.sigma_iters, fl.sigma_tol, fl.sigma_iterations, fl.rhs_calls = 200, 1e-14, 0, 0
    return fl


def test_multiloop_self_energy_is_iterated_to_self_consistency():
    fl = _flow(4)
    y = torch.zeros(fl.size(), dtype=torch.complex128)
    out = fl.rhs(0.5, y)
    a = fl.ml.a
    star = a / (1.0 - C_GAIN * (1.0 + D_GAIN))          # ds = a + c ds + d c ds
    dR, dK = fl.sigma(out)
    assert torch.abs(dR - star[:, 1, 0]).max() <= 1e-12 * torch.abs(star).max()
    assert torch.abs(dK - star[:, 1, 1]).max() <= 1e-12 * torch.abs(star).max()
    assert fl.ml.runs == fl.sigma_iterations and fl.ml.runs > 10
    # the vertex part comes from the last vertex step (Katanin table within tolerance of Σ-dot)
    assert torch.abs(out[:2] - star[:2, 1, 0]).max() <= 1e-12 * torch.abs(star).max()


def test_one_and_two_loops_take_the_one_loop_self_energy():
    for n in (1, 2):
        fl = _flow(n)
        out = fl.rhs(0.5, torch.zeros(fl.size(), dtype=torch.complex128))
        dR, dK = fl.sigma(out)
        assert fl.ml.runs == 1 and fl.sigma_iterations == 0
        assert torch.equal(dR, fl.ml.a[:, 1, 0]) and torch.equal(dK, fl.ml.a[:, 1, 1])
