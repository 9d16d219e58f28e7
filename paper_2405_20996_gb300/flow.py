"""Vertex flow of the multiloop fRG (Sec. III.C) in the interaction-flow scheme, with the
self-energy held fixed or flowing at one loop.

The interaction flow scales the propagator, G_Λ = Λ G at Σ = 0 (Sec. III.C.2), from Λ ≈ 0
(where γ = 0) to Λ = 1.  The vertex's reducible parts obey dγ_r/dΛ = Σ_{l ≤ n} γ̇_r^(l), the
right-hand side of the n-loop flow built by `MultiloopStep` (one-loop part with
Π-dot = G S + S G, S = dG/dΛ, then the left, central and right parts); with all loop orders
the flow reproduces the parquet solution at the final Λ (the parquet approximation's R = Γ0
does not depend on Λ).  The integrator is the embedded Runge–Kutta pair of Cash and Karp
(orders 5 and 4, six stages) with step-size control on the maximum norm, the scheme the
paper uses for its flows (Sec. III.C.1); the step advances with the fifth-order solution and
the difference of the two solutions is the error estimate.

With n_sig > 0 the self-energy flows too, Σ stored on an n_sig-point tan grid (the
library's Σ tables, linear in x, zero at v = ±inf), and the vertex's Π-dot takes the
Katanin substitution S -> S + G Σ-dot G.  Σ-dot = L(Γ, S) at one and two loops, with L the
`loop` function (the single-scale propagator at fixed Σ); from three loops on it adds the
multiloop terms,
    Σ-dot = L(Γ, S) + Σ-dot_t̄ + Σ-dot_t,   Σ-dot_t̄ = L(γ̇^C_t̄, G),   Σ-dot_t = L(Γ, G Σ-dot_t̄ G),
γ̇^C_t̄ the central parts (orders l >= 3) of the a and p channels, and since the vertex's
central parts depend on Σ-dot through the Katanin line, Σ-dot and the vertex step are
iterated to self-consistency (at most sigma_iters times, relative change sigma_tol).
"""

import numpy as np
import torch

from . import kb
from .engine import CLASS_NAMES
from .multiloop import S_GAMMA, MultiloopStep, s_central

# Cash-Karp Butcher tableau (published coefficients of the embedded 5(4) pair)
_C = (0.0, 1 / 5, 3 / 10, 3 / 5, 1.0, 7 / 8)
_A = ((),
      (1 / 5,),
      (3 / 40, 9 / 40),
      (3 / 10, -9 / 10, 6 / 5),
      (-11 / 54, 5 / 2, -70 / 27, 35 / 27),
      (1631 / 55296, 175 / 512, 575 / 13824, 44275 / 110592, 253 / 4096))
_B5 = (37 / 378, 0.0, 250 / 621, 125 / 594, 0.0, 512 / 1771)
_B4 = (2825 / 27648, 0.0, 18575 / 48384, 13525 / 55296, 277 / 14336, 1 / 4)


class VertexFlow:
    """n-loop vertex flow of one parameter point (grids, Nq, U, Δ, T) in the interaction flow."""

    def __init__(self, grids, nq, U, Delta, T, n_loops=6, precision="fp64", A=5.0, device=0, n_sig=0,
                 sigma_iters=10, sigma_tol=1e-8):
        g = grids
        shapes = {"K1": (g["n1"], 16), "K2": (g["n2w"], g["n2v"], 16), "K2p": (g["n2w"], g["n2v"], 16),
                  "K3": (g["n3w"], g["n3v"], g["n3v"], 16)}
        zero = {c: tuple(np.zeros(shapes[k], dtype=np.complex128) for k in CLASS_NAMES) for c in range(3)}
        # Γ along the flow is not kept exactly symmetric by the central parts' discretisation,
        # so no symmetry reduction is used
        self.ml = MultiloopStep(grids, nq, U, Delta, T, zero, n_loops=n_loops, precision=precision, A=A,
                                device=device, symmetric=False, cache=False,
                                keep_central=(n_sig > 0 and n_loops >= 3))
        self.sigma_iters, self.sigma_tol = int(sigma_iters), float(sigma_tol)
        self.sigma_iterations = 0
        e0 = self.ml.e[self.ml.channels[0]]
        self.gamma_t = [e0.tensors[S_GAMMA][(c, k)] for c in range(3) for k in range(4)]
        self.sizes = [t.numel() for t in self.gamma_t]
        self.dtype = self.gamma_t[0].dtype
        self.dev = e0.device
        self.rhs_calls = 0
        self.n_sig, self.A = int(n_sig), A
        self.n_gamma = sum(self.sizes)
        if self.n_sig:
            x = -1.0 + 2.0 * (np.arange(self.n_sig) + 1) / (self.n_sig + 1)
            self.sig_grid = A * np.tan(np.pi * x / 2)           # the Σ table's frequencies

    def close(self):
        self.ml.close()

    # flat state <-> the Γ slot's class tensors
    def _store(self, y):
        off = 0
        for t, n in zip(self.gamma_t, self.sizes):
            t.view(-1).copy_(y[off:off + n])
            off += n

    def _total(self):
        return torch.cat([self.ml.total[(c, k)].reshape(-1) for c in range(3) for k in range(4)])

    def size(self):
        """Length of the flat state: the 12 class arrays, then Σ^R and Σ^K on the Σ grid."""
        return self.n_gamma + 2 * self.n_sig

    def sigma(self, y):
        """(Σ^R, Σ^K) views of a flat state on the Σ grid (empty without a flowing Σ)."""
        return y[self.n_gamma:self.n_gamma + self.n_sig], y[self.n_gamma + self.n_sig:]

    def channels(self, y):
        """{channel: {class: tensor}} views of a flat state."""
        out, off = {}, 0
        for c in range(3):
            out[c] = {}
            for k in range(4):
                n = self.sizes[4 * c + k]
                out[c][CLASS_NAMES[k]] = y[off:off + n].view(self.gamma_t[4 * c + k].shape)
                off += n
        return out

    def rhs(self, lam, y):
        """dy/dΛ at Λ = lam: the multiloop right-hand side of the vertex with the
        interaction-flow propagator; with a flowing Σ, Σ-dot (one-loop term, and from three
        loops on its t̄ and t terms, iterated with the vertex step) and the vertex's Katanin
        substitution."""
        engines = list(self.ml.e.values())
        for e in engines:
            e.set_regulator(kb.KB_REG_U, lam)
        self._store(y[:self.n_gamma])
        if self.n_sig:
            sR, sK = (t.detach().cpu().numpy() for t in self.sigma(y))
            for e in engines:
                e.set_self_energy(sR, sK, self.A)
                e.set_self_energy_derivative(None)
            e0 = self.ml.e[self.ml.channels[0]]
            d1 = e0.loop(S_GAMMA, self.sig_grid, single_scale=True)          # L(Γ, S)
            ds = d1
            for _ in range(self.sigma_iters if self.ml.keep_central else 1):
                dRh, dKh = ds[:, 1, 0].cpu().numpy(), ds[:, 1, 1].cpu().numpy()
                for e in engines:
                    e.set_self_energy_derivative(dRh, dKh, self.A)
                self.ml.zero()
                self.ml.run_eager()
                if not self.ml.keep_central:
                    break
                tb = e0.loop(s_central(self.ml.n_loops), self.sig_grid)           # L(γ̇^C_t̄, G)
                e0.set_self_energy_derivative(tb[:, 1, 0].cpu().numpy(), tb[:, 1, 1].cpu().numpy(), self.A)
                tt = e0.loop(S_GAMMA, self.sig_grid, line=2)                         # L(Γ, G Σ̇_t̄ G)
                new = d1 + tb + tt
                change = float((new - ds).abs().max()) / max(float(new.abs().max()), 1e-300)
                ds = new
                self.sigma_iterations += 1
                if change <= self.sigma_tol:
                    break
            dR, dK = ds[:, 1, 0], ds[:, 1, 1]
        else:
            self.ml.zero()
            self.ml.run_eager()
        self.rhs_calls += 1
        out = self._total()
        if self.n_sig:
            out = torch.cat([out, dR.to(out.dtype), dK.to(out.dtype)])
        return out.clone()

    def integrate(self, lam0, lam1, y0=None, h0=0.05, rtol=1e-6, atol=1e-10, max_steps=500, callback=None):
        """Cash–Karp integration from Λ = lam0 (state y0, default 0) to lam1; returns
        (y, accepted steps, rejected steps).  callback(Λ, y) after every accepted step (e.g.
        a checkpoint layer); a run resumes from a saved (Λ, y)."""
        y = torch.zeros(self.size(), dtype=self.dtype, device=self.dev) if y0 is None else y0.clone()
        lam, h = float(lam0), float(h0)
        acc = rej = 0
        while lam < lam1 - 1e-14 and acc + rej < max_steps:
            h = min(h, lam1 - lam)
            k = []
            for s in range(6):
                ys = y.clone()
                for j, a in enumerate(_A[s]):
                    if a != 0.0:
                        ys += (h * a) * k[j]
                k.append(self.rhs(lam + _C[s] * h, ys))
            y5 = y.clone()
            y4 = y.clone()
            for s in range(6):
                if _B5[s] != 0.0:
                    y5 += (h * _B5[s]) * k[s]
                if _B4[s] != 0.0:
                    y4 += (h * _B4[s]) * k[s]
            scale = atol + rtol * max(float(y.abs().max()), float(y5.abs().max()))
            err = float((y5 - y4).abs().max()) / scale
            if err <= 1.0:
                y, lam = y5, lam + h
                acc += 1
                if callback is not None:
                    callback(lam, y)
            else:
                rej += 1
            h *= min(5.0, max(0.2, 0.9 * (err if err > 0 else 1e-10) ** -0.2))
        return y, acc, rej
