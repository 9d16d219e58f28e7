"""Parquet approximation solved with the library's bubble (Sec. III.B).

The parquet approximation takes the totally irreducible vertex as the bare one, R = Γ0
(strength U; Sec. I.B).  With the self-energy held fixed (the context's Σ table, or Σ = 0),
the reducible vertices of the three channels solve the Bethe–Salpeter equations

    γ_r = B_r(I_r, Γ),   I_r = Γ − γ_r,   Γ = R + γ_a + γ_p + γ_t,   r ∈ {a, p, t},

where B_r carries the channel prefactor c_r (1, 1/2, −1) and γ_r is stored as its
asymptotic classes K1, K2, K2', K3 (Sec. II.C.1).  I_r is the vertex slot of Γ with
channel r left out of the slot's channel mask; the library still reads channel r's data
as the crossing partner of the up-up component, as the vertex requires.

Three solvers; the residual bubbles go through the library's plain FP64 path:

- the damped fixed point γ ← (1 − m) γ + m B(γ) with mixing m, the scheme the paper
  describes for its parquet solver, stopped on the relative maximum-norm change;
- Anderson acceleration of that iteration over the last few iterates (`anderson`), the
  paper's other mixing scheme;
- Newton–Krylov on F(γ) = γ − B(γ): each Newton step solves J δ = −F by restarted
  GMRES.  B_r is bilinear in its two vertices, so the Jacobian product is
      J v = v − Σ_r [B_r(V_I_r, Γ) + B_r(I_r, V)],   V = Σ_r v_r (no bare part),
  two bubbles per channel; J^H comes from kb_bubble_vjp (`adjoint`), and with it the
  adjoint sensitivity of an observable of the converged vertex to the coupling U
  (`sensitivity_U`: one GMRES solve with J^H instead of one Newton solve per parameter).
  The Jacobian products may use the mixed-precision bubble (`jvp_precision`).

symmetric_bse=True takes the symmetrised form the paper recommends for stability,
    γ_r = ½ [B_r(I_r, Γ) + B_r(Γ, I_r)],
the right-hand side as is and with I_r and Γ interchanged, averaged (Sec. III.B); it has the
same fixed point (the two orders agree at the solution), and its Jacobian and adjoint are
the averages of the two orders' (four bubbles per channel in J v, two adjoint calls).

The state is one flat complex128 device vector holding the 12 class arrays; the vertex
slots are views of it, so no data moves between a solver update and the next bubble.  The
solvers' vector algebra (updates, norms, inner products) are PyTorch device operations;
the GMRES Hessenberg least-squares problem (at most a few dozen unknowns) is solved on the
host.
"""

import numpy as np
import torch

from . import kb
from .engine import CLASS_NAMES, Engine

# vertex slots of the engine context
S_GAMMA = 0                 # Γ = R + γ_a + γ_p + γ_t
S_I = (1, 2, 3)             # I_r = Γ − γ_r
S_DELTA = 4                 # V = v_a + v_p + v_t (a tangent or adjoint direction, no R)
S_DELTA_I = (5, 6, 7)       # V − v_r
S_OUT = 8                   # bubble outputs, all channels
S_GRAD = 9                  # adjoint accumulation, all channels
S_RHAT = 10                 # the bare vertex of unit strength, no classes (∂/∂U, the SDE)
S_X = 11                    # X̂ = B_a(R̂, Γ) of the Schwinger–Dyson equation: channel a only
S_XP = 12                   # B_p(R̂, Γ), the SDE's p-channel form: channel p only
S_XT = 13                   # the SDE's t-channel form: channel a = B_a(R̂, Γ) (the S_X arrays),
                            # channel t = B_t(R̂, Γ) as crossing-partner data, mask {a}
SDE_FORMS = ("a", "p", "ap", "t", "apt")


class ParquetPA:
    """Parquet-approximation solver of one parameter point (grids, Nq, U, Δ, T).

    jvp_precision="mixed" evaluates the Jacobian products of Newton–Krylov with the
    mixed-precision bubble (complex64 copies of the state in a second context, FP32 gather,
    3xTF32 contraction, ~1e-6 relative error) while the residual F(γ) stays FP64: the Newton
    iteration is then inexact only in its linear model, and converges to the FP64 fixed
    point."""

    def __init__(self, grids, nq, U, Delta, T, A=5.0, eps=0.0, device=0, jvp_precision="fp64",
                 symmetric_bse=False):
        self.e = Engine(grids, nq, A=A, device=device)
        self.symmetric_bse = bool(symmetric_bse)
        self.e.set_model(Delta, T, eps)
        self.jvp_precision = jvp_precision
        self.U = float(U)
        self.dev = self.e.device
        sh = self.e.class_shapes()
        self.layout, off = [], 0
        for ch in range(3):
            for k, name in enumerate(CLASS_NAMES):
                n = int(np.prod(sh[name]))
                self.layout.append((ch, k, sh[name], off, n))
                off += n
        self.n = off
        z = lambda: torch.zeros(self.n, dtype=torch.complex128, device=self.dev)
        self.gamma, self.delta, self.out, self.grad = z(), z(), z(), z()
        self._attach(S_GAMMA, self.gamma, True, 7)
        self._attach(S_DELTA, self.delta, False, 7)
        for r in range(3):
            self._attach(S_I[r], self.gamma, True, 7 & ~(1 << r))
            self._attach(S_DELTA_I[r], self.delta, False, 7 & ~(1 << r))
        self._attach(S_OUT, self.out, False, 7)
        self._attach(S_GRAD, self.grad, False, 7)
        self.bubbles = 0
        self.mixed_bubbles = 0
        if jvp_precision == "mixed":
            self.m = Engine(grids, nq, A=A, device=device)
            self.m.set_model(Delta, T, eps)
            z32 = lambda: torch.zeros(self.n, dtype=torch.complex64, device=self.dev)
            self.gamma32, self.delta32 = z32(), z32()
            self._attach(S_GAMMA, self.gamma32, True, 7, e=self.m)
            self._attach(S_DELTA, self.delta32, False, 7, e=self.m)
            for r in range(3):
                self._attach(S_I[r], self.gamma32, True, 7 & ~(1 << r), e=self.m)
                self._attach(S_DELTA_I[r], self.delta32, False, 7 & ~(1 << r), e=self.m)
            self._attach(S_OUT, self.out, False, 7, e=self.m)
            self._gamma32_of = None

    def close(self):
        self.e.close()
        if self.jvp_precision == "mixed":
            self.m.close()

    def _attach(self, slot, buf, has_R, mask, e=None):
        e = e or self.e
        kb.kb_set_vertex(e.ctx, slot, has_R, self.U)
        kb.kb_set_vertex_channels(e.ctx, slot, mask)
        kb.kb_set_vertex_symmetric(e.ctx, slot, False)
        e.tensors[slot] = {}
        for ch, k, shape, off, n in self.layout:
            e.attach(slot, ch, k, buf[off:off + n].view(shape))

    def classes(self, buf, ch):
        """{"K1", "K2", "K2p", "K3"} views of channel ch of a flat state vector."""
        return {CLASS_NAMES[k]: buf[off:off + n].view(shape) for c, k, shape, off, n in self.layout if c == ch}

    def channels(self, buf):
        """{channel: (K1, K2, K2p, K3)} of a flat state vector (views)."""
        return {ch: tuple(self.classes(buf, ch)[k] for k in CLASS_NAMES) for ch in range(3)}

    # ---- the map and its derivatives ----------------------------------------------------
    def bse(self, gamma):
        """Right-hand sides B_r(I_r, Γ) of the three Bethe–Salpeter equations at γ (or their
        symmetrised form ½ [B_r(I_r, Γ) + B_r(Γ, I_r)])."""
        self.gamma.copy_(gamma)
        for r in range(3):
            if self.symmetric_bse:
                self.e.bubble(r, S_I[r], S_GAMMA, S_OUT, alpha=0.5, precision="fp64")
                self.e.bubble(r, S_GAMMA, S_I[r], S_OUT, alpha=0.5, beta=1.0, precision="fp64")
            else:
                self.e.bubble(r, S_I[r], S_GAMMA, S_OUT, precision="fp64")
        self.bubbles += 6 if self.symmetric_bse else 3
        return self.out.clone()

    def _jvp_bubbles(self, e, prec):
        """Σ_r dB_r into S_OUT of engine e: B_r(V_I_r, Γ) + B_r(I_r, V), symmetrised with the
        interchanged order when the symmetric form is used."""
        a = 0.5 if self.symmetric_bse else 1.0
        for r in range(3):
            e.bubble(r, S_DELTA_I[r], S_GAMMA, S_OUT, alpha=a, precision=prec)
            e.bubble(r, S_I[r], S_DELTA, S_OUT, alpha=a, beta=1.0, precision=prec)
            if self.symmetric_bse:
                e.bubble(r, S_DELTA, S_I[r], S_OUT, alpha=a, beta=1.0, precision=prec)
                e.bubble(r, S_GAMMA, S_DELTA_I[r], S_OUT, alpha=a, beta=1.0, precision=prec)
        return 12 if self.symmetric_bse else 6

    def residual(self, gamma):
        return gamma - self.bse(gamma)

    def jvp(self, gamma, v):
        """J v at γ for F(γ) = γ − B(γ) (in the precision chosen for the Jacobian products)."""
        if self.jvp_precision == "mixed":
            if self._gamma32_of is not gamma:              # one conversion per Newton step
                self.gamma32.copy_(gamma)
                self._gamma32_of = gamma
            self.delta32.copy_(v)
            self.mixed_bubbles += self._jvp_bubbles(self.m, "mixed")
            return v - self.out
        self.gamma.copy_(gamma)
        self.delta.copy_(v)
        self.bubbles += self._jvp_bubbles(self.e, "fp64")
        return v - self.out

    def adjoint(self, gamma, u):
        """J^H u at γ: u − Σ_r (dB_r/dγ)^H u_r through the adjoint kernels (complex-linear
        map, so J^H is the conjugate transpose; gradients in PyTorch's convention)."""
        self.gamma.copy_(gamma)
        self.out.copy_(u)
        self.grad.zero_()
        a = 0.5 if self.symmetric_bse else 1.0
        for r in range(3):
            self.e.bubble_vjp(r, S_I[r], S_GAMMA, S_OUT, alpha=a, grad_left=S_GRAD, grad_right=S_GRAD)
            if self.symmetric_bse:
                self.e.bubble_vjp(r, S_GAMMA, S_I[r], S_OUT, alpha=a, grad_left=S_GRAD, grad_right=S_GRAD)
        return u - self.grad

    def _zero_state(self):
        return torch.zeros_like(self.gamma)

    @staticmethod
    def rel(diff, ref):
        return float(diff.abs().max()) / max(float(ref.abs().max()), 1e-300)

    # ---- solvers ------------------------------------------------------------------------
    def fixed_point(self, mix=0.5, tol=1e-10, maxit=500, gamma0=None, callback=None):
        """Damped iteration; returns (γ, history of relative residuals).  callback(it, γ, r)
        after every iteration (e.g. a checkpoint); gamma0 resumes from a saved state."""
        g = self._zero_state() if gamma0 is None else gamma0.clone()
        hist = []
        for it in range(maxit):
            b = self.bse(g)
            hist.append(self.rel(g - b, b))
            if hist[-1] <= tol:
                return b, hist
            g = (1.0 - mix) * g + mix * b
            if callback is not None:
                callback(it, g, hist[-1])
        return g, hist

    def anderson(self, mix=0.5, m=5, tol=1e-10, maxit=500, gamma0=None, callback=None, cond_max=1e10):
        """Anderson acceleration of the damped iteration (the paper's alternative to plain
        mixing in the parquet solver, Sec. III.B), in the form of Walker and Ni (SIAM J.
        Numer. Anal. 49, 1715 (2011)): with g_k = BSE(γ_k), f_k = g_k − γ_k and the last m
        differences ΔG, ΔF of g and f, the coefficients c minimise ||f_k − ΔF c||_2 and
        γ_{k+1} = (g_k − ΔG c) − (1 − mix)(f_k − ΔF c).  The least-squares problem is solved by
        QR; the oldest differences are dropped while R's diagonal spans more than cond_max.
        m = 0 is the damped iteration.  Returns (γ, history of relative residuals)."""
        g = self._zero_state() if gamma0 is None else gamma0.clone()
        hist = []
        dF, dG = [], []
        f_prev = b_prev = None
        for it in range(maxit):
            b = self.bse(g)
            f = b - g
            hist.append(self.rel(f, b))
            if hist[-1] <= tol:
                return b, hist
            if f_prev is not None and m > 0:
                dF.append(f - f_prev)
                dG.append(b - b_prev)
                if len(dF) > m:
                    dF.pop(0)
                    dG.pop(0)
            f_prev, b_prev = f, b
            g_next = None
            while dF:
                Q, R = torch.linalg.qr(torch.stack(dF, dim=1))
                d = R.diagonal().abs()
                if float(d.min()) * cond_max < float(d.max()) or float(d.max()) == 0.0:
                    dF.pop(0)
                    dG.pop(0)
                    continue
                c = torch.linalg.solve_triangular(R, (Q.conj().T @ f).unsqueeze(1), upper=True).squeeze(1)
                fa = f - torch.stack(dF, dim=1) @ c
                ba = b - torch.stack(dG, dim=1) @ c
                g_next = ba - (1.0 - mix) * fa
                break
            g = (1.0 - mix) * g + mix * b if g_next is None else g_next
            if callback is not None:
                callback(it, g, hist[-1])
        return g, hist

    def gmres(self, gamma, rhs, rtol, m=30, maxit=300):
        """Restarted GMRES(m) for J x = rhs at γ.  Returns (x, Jacobian products, relative
        residual)."""
        return self._gmres(lambda v: self.jvp(gamma, v), rhs, rtol, m, maxit)

    @staticmethod
    def _gmres(apply, rhs, rtol, m, maxit):
        """Restarted GMRES(m) for A x = rhs, A given by apply(v) (Arnoldi with modified
        Gram–Schmidt; the small least-squares problem min ||β e1 − H y|| solved on the host
        each step)."""
        x = torch.zeros_like(rhs)
        bnorm = float(torch.linalg.vector_norm(rhs))
        if bnorm == 0.0:
            return x, 0, 0.0
        its, res = 0, 1.0
        r = rhs.clone()
        while its < maxit:
            beta = float(torch.linalg.vector_norm(r))
            res = beta / bnorm
            if res <= rtol:
                break
            V = [r / beta]
            H = np.zeros((m + 1, m), dtype=np.complex128)
            y = None
            for k in range(m):
                w = apply(V[k])
                its += 1
                for i in range(k + 1):
                    h = torch.vdot(V[i], w)
                    H[i, k] = complex(h)
                    w = w - h * V[i]
                hn = float(torch.linalg.vector_norm(w))
                H[k + 1, k] = hn
                e1 = np.zeros(k + 2, dtype=np.complex128)
                e1[0] = beta
                y = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)[0]
                res = float(np.linalg.norm(e1 - H[:k + 2, :k + 1] @ y)) / bnorm
                if res <= rtol or hn == 0.0 or its >= maxit:
                    break
                V.append(w / hn)
            for i in range(len(y)):
                x = x + complex(y[i]) * V[i]
            if res <= rtol or its >= maxit:
                break
            r = rhs - apply(x)
        return x, its, res

    # ---- adjoint sensitivities ------------------------------------------------------------
    def dF_dU(self, gamma):
        """∂F/∂U at fixed γ: F = γ − B(γ) with R = U R̂ in both I_r and Γ, and B bilinear, so
        ∂F/∂U = −Σ_r [B_r(R̂, Γ) + B_r(I_r, R̂)] (R̂ the bare vertex of unit strength)."""
        kb.kb_set_vertex(self.e.ctx, S_RHAT, True, 1.0)
        self.gamma.copy_(gamma)
        a = 0.5 if self.symmetric_bse else 1.0
        for r in range(3):
            self.e.bubble(r, S_RHAT, S_GAMMA, S_OUT, alpha=a, precision="fp64")
            self.e.bubble(r, S_I[r], S_RHAT, S_OUT, alpha=a, beta=1.0, precision="fp64")
            if self.symmetric_bse:
                self.e.bubble(r, S_RHAT, S_I[r], S_OUT, alpha=a, beta=1.0, precision="fp64")
                self.e.bubble(r, S_GAMMA, S_RHAT, S_OUT, alpha=a, beta=1.0, precision="fp64")
        self.bubbles += 12 if self.symmetric_bse else 6
        return -self.out.clone()

    def sensitivity_U(self, gamma, c, rtol=1e-10, m=30, maxit=300):
        """d/dU of the observable L = Re<c, γ*> at a converged γ* = gamma, by the adjoint
        method: solve J^H λ = c with GMRES on the adjoint kernels' products, then
        dL/dU = −Re<λ, ∂F/∂U>.  Returns (dL/dU, adjoint products, relative residual)."""
        lam, its, res = self._gmres(lambda u: self.adjoint(gamma, u), c, rtol, m, maxit)
        return -float(torch.vdot(lam, self.dF_dU(gamma)).real), its, res

    def newton_krylov(self, tol=1e-10, maxit=30, gmres_m=30, gmres_maxit=300, gamma0=None, callback=None):
        """Inexact Newton; returns (γ, history of relative residuals, GMRES products per step).
        callback(step, γ, r) after every Newton step; gamma0 resumes from a saved state."""
        g = self._zero_state() if gamma0 is None else gamma0.clone()
        hist, lin = [], []
        for step in range(maxit):
            b = self.bse(g)
            F = g - b
            hist.append(self.rel(F, b))
            if hist[-1] <= tol:
                return b, hist, lin
            eta = min(1e-2, max(1e-4 * hist[-1], 1e-12))    # forcing term of the inexact Newton step
            d, its, _ = self.gmres(g, -F, eta, gmres_m, gmres_maxit)
            lin.append(its)
            g = g + d
            if callback is not None:
                callback(step, g, hist[-1])
        return g, hist, lin


class ParquetSDE(ParquetPA):
    """Parquet approximation with a self-consistent self-energy from the Schwinger–Dyson
    equation (Sec. III.B), the self-energy on an n_sig-point tan grid (the library's Σ
    tables: linear in x, zero at v = ±inf).

    The state is z = [γ (the 12 class arrays), Σ^R, Σ^K]; the map sets G[Σ] and returns the
    Bethe–Salpeter right-hand sides B_r(I_r, Γ) and the Schwinger–Dyson self-energy, both
    with that G.  SDE in its a-channel form: the bare vertex, an a-channel bubble to the full
    vertex and the line that closes it,
        Σ = U loop(R̂) + loop_ud(B_a(R, Γ)) = U [loop(R̂) + ½ loop(X̂)],   X̂ = B_a(R̂, Γ),
    where loop is kb_loop (Σ = −∫dv'/(2πi) Γ_s G with Γ_s = Γ_ud + Γ_uu) and the closed line
    joins legs 2' (on Γ) and 2 (on R), so only X̂'s up-down part enters: X̂ sits in a slot
    with channel a alone and no crossing-partner data, where Γ_s = 2 X̂_ud.  loop(R̂) is the
    Hartree shift per unit U (zero at particle-hole symmetry).  At second order this is the
    sunset self-energy exactly (pinned against the textbook spectral integral).  form "p"
    takes the p-channel form U [loop(R̂) + loop_ud(B_p(R̂, Γ))], both through kb_loop's
    up-down-only line.  form "t" draws the bubble in the t channel: R̂ then holds legs 1', 1
    and Γ legs 2', 2, the closing line joins 1 and 2' and carries the external spin, and
    with SU(2) and crossing the up-up t bubble is B_t(R̂, Γ) − X[B_a(R̂, Γ)] (X: legs 1 and 2
    exchanged), so Σ = U [loop(R̂) + loop_uu(S_XT)] with loop_uu = loop − loop_ud of a slot
    holding B_a(R̂, Γ) in channel a and B_t(R̂, Γ) as its crossing-partner data.  "ap" and
    "apt" average the forms (the paper combines them).  Solved with the damped iteration,
    Anderson acceleration or Newton–Krylov on z.

    The Jacobian product J v of F(z) = z − M(z) in a direction v = [v_γ, δΣ^R, δΣ^K] adds to
    the vertex terms of the base class the change of every propagator along δΣ: the Dyson
    propagator changes by G δΣ G, which the library provides as the Katanin line of the
    no-flow scheme (KB_REG_NONE: S = 0, the δΣ tables as the dΣ tables), so each bubble gains
    B_r(·, ·; Π̇) with Π̇ = G (G δΣ G) + (G δΣ G) G, and each self-energy loop its G δΣ G line
    (kb_loop line 2); the Schwinger–Dyson bubble X̂ changes by B(R̂, V) + B(R̂, Γ; Π̇).  The
    adjoint of this map is not built (sensitivities need the Σ-free base class)."""

    def __init__(self, grids, nq, U, Delta, T, n_sig=41, A=5.0, eps=0.0, device=0, form="a", symmetric_bse=False):
        super().__init__(grids, nq, U, Delta, T, A=A, eps=eps, device=device, symmetric_bse=symmetric_bse)
        if form not in SDE_FORMS:
            raise ValueError("form: one of %s" % (SDE_FORMS,))
        self.form = form
        self.n_sig, self.A_sig = int(n_sig), A
        x = -1.0 + 2.0 * (np.arange(self.n_sig) + 1) / (self.n_sig + 1)
        self.sig_grid = A * np.tan(np.pi * x / 2)
        sh = self.e.class_shapes()
        self.xa = [torch.zeros(sh[name], dtype=torch.complex128, device=self.dev) for name in CLASS_NAMES]
        kb.kb_set_vertex(self.e.ctx, S_X, False, 0.0)
        kb.kb_set_vertex_channels(self.e.ctx, S_X, 1 << 0)
        kb.kb_set_vertex_symmetric(self.e.ctx, S_X, False)
        self.e.tensors[S_X] = {}
        for k in range(4):
            self.e.attach(S_X, 0, k, self.xa[k])
        if "t" in form:
            self.xt = [torch.zeros(sh[name], dtype=torch.complex128, device=self.dev) for name in CLASS_NAMES]
            kb.kb_set_vertex(self.e.ctx, S_XT, False, 0.0)
            kb.kb_set_vertex_channels(self.e.ctx, S_XT, 1 << 0)
            kb.kb_set_vertex_symmetric(self.e.ctx, S_XT, False)
            self.e.tensors[S_XT] = {}
            for k in range(4):
                self.e.attach(S_XT, 0, k, self.xa[k])
                self.e.attach(S_XT, 2, k, self.xt[k])
        if "p" in form:
            self.xp = [torch.zeros(sh[name], dtype=torch.complex128, device=self.dev) for name in CLASS_NAMES]
            kb.kb_set_vertex(self.e.ctx, S_XP, False, 0.0)
            kb.kb_set_vertex_channels(self.e.ctx, S_XP, 1 << 1)
            kb.kb_set_vertex_symmetric(self.e.ctx, S_XP, False)
            self.e.tensors[S_XP] = {}
            for k in range(4):
                self.e.attach(S_XP, 1, k, self.xp[k])
        kb.kb_set_vertex(self.e.ctx, S_RHAT, True, 1.0)
        # S = 0, so that the Katanin line of Π-dot and of the loop is G δΣ G alone
        self.e.set_regulator(kb.KB_REG_NONE)

    def _zero_state(self):
        return torch.zeros(self.n + 2 * self.n_sig, dtype=torch.complex128, device=self.dev)

    def split(self, z):
        """(γ, Σ^R, Σ^K) views of a state."""
        return z[:self.n], z[self.n:self.n + self.n_sig], z[self.n + self.n_sig:]

    def set_sigma(self, sR, sK):
        self.e.set_self_energy(sR.detach().cpu().numpy(), sK.detach().cpu().numpy(), self.A_sig)

    def _sde_terms(self):
        """Terms of the form: (slot, bubbles (channel, output slot) that fill it, loop, weight);
        loop "half": ½ loop (channel a alone, no partner data: the up-down loop), "ud":
        loop_ud, "uu": loop − loop_ud."""
        a_half = (S_X, ((0, S_X),), "half")
        a = (S_X, ((0, S_X),), "ud")
        p = (S_XP, ((1, S_XP),), "ud")
        t = (S_XT, ((0, S_X), (2, S_XT)), "uu")
        terms = {"a": (a_half,), "p": (p,), "ap": (a, p), "t": (t,), "apt": (a, p, t)}[self.form]
        return [(slot, bub, mode, 1.0 / len(terms)) for slot, bub, mode in terms]

    def _sde_bubbles(self):
        out = []
        for _, bub, _, _ in self._sde_terms():
            out += [b for b in bub if b not in out]
        return out

    def _sde_loop(self, slot, mode, line=None):
        if mode == "half":
            return 0.5 * self.e.loop(slot, self.sig_grid, line=line)
        ud = self.e.loop(slot, self.sig_grid, line=line, ud_only=True)
        return ud if mode == "ud" else self.e.loop(slot, self.sig_grid, line=line) - ud

    def sde(self, gamma):
        """(Σ^R, Σ^K) on the Σ grid from the SDE for γ, with the context's current G."""
        self.gamma.copy_(gamma)
        s = self.e.loop(S_RHAT, self.sig_grid)
        for r, slot in self._sde_bubbles():
            self.e.bubble(r, S_RHAT, S_GAMMA, slot, precision="fp64")
            self.bubbles += 1
        for slot, _, mode, w in self._sde_terms():
            s = s + w * self._sde_loop(slot, mode)
        s = self.U * s
        return s[:, 1, 0], s[:, 1, 1]

    def bse(self, z):
        """The joint map: [B_r(I_r, Γ), Σ_SDE] at G[Σ]."""
        g, sR, sK = self.split(z)
        self.set_sigma(sR, sK)
        b = ParquetPA.bse(self, g)
        sR2, sK2 = self.sde(g)
        return torch.cat([b, sR2, sK2])

    def jvp(self, z, v):
        """J v at z = [γ, Σ^R, Σ^K] for F(z) = z − M(z), M the joint map of `bse`."""
        g, sR, sK = self.split(z)
        vg, vR, vK = self.split(v)
        self.set_sigma(sR, sK)
        self.e.set_self_energy_derivative(vR.detach().cpu().numpy(), vK.detach().cpu().numpy(), self.A_sig)
        self.gamma.copy_(g)
        self.delta.copy_(vg)
        # Bethe–Salpeter right-hand sides: the vertex directions, then the propagators' change
        self.bubbles += self._jvp_bubbles(self.e, "fp64")
        a = 0.5 if self.symmetric_bse else 1.0
        for r in range(3):
            self.e.bubble(r, S_I[r], S_GAMMA, S_OUT, pi_kind=kb.KB_PI_GS_SG, alpha=a, beta=1.0, precision="fp64")
            self.bubbles += 1
            if self.symmetric_bse:
                self.e.bubble(r, S_GAMMA, S_I[r], S_OUT, pi_kind=kb.KB_PI_GS_SG, alpha=a, beta=1.0, precision="fp64")
                self.bubbles += 1
        dB = self.out.clone()
        # Schwinger–Dyson self-energy: the loops' G δΣ G lines and the change of X̂
        ds = self.e.loop(S_RHAT, self.sig_grid, line=2)
        bubbles, terms = self._sde_bubbles(), self._sde_terms()
        for r, slot in bubbles:
            self.e.bubble(r, S_RHAT, S_GAMMA, slot, precision="fp64")
        for slot, _, mode, w in terms:
            ds = ds + w * self._sde_loop(slot, mode, line=2)
        for r, slot in bubbles:
            self.e.bubble(r, S_RHAT, S_DELTA, slot, precision="fp64")
            self.e.bubble(r, S_RHAT, S_GAMMA, slot, pi_kind=kb.KB_PI_GS_SG, beta=1.0, precision="fp64")
            self.bubbles += 3
        for slot, _, mode, w in terms:
            ds = ds + w * self._sde_loop(slot, mode)
        ds = self.U * ds
        self.e.set_self_energy_derivative(None)
        return v - torch.cat([dB, ds[:, 1, 0], ds[:, 1, 1]])

    def adjoint(self, z, u):
        raise NotImplementedError("the adjoint of the self-energy-coupled map is not built")
