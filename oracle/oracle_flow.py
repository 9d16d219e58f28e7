"""Plain multiloop fRG flow and self-consistent parquet solution on the oracle's bubbles and
loops (TEST INFRASTRUCTURE: only tests use this module; it shares no code with the CUDA
library or its Python package).

Interaction flow (Sec. III.C.2): G_L = L / (v - eps + i Delta - L Sigma), from L = lam0 to 1.

Vertex (Sec. III.C), per channel r, at fixed Γ = R + Σ_r γ_r and Σ:
    γ̇_r^(1) = B_r(Γ, Γ; Π̇),  Π̇ = G Ġ + Ġ G,  Ġ = S + G Σ̇ G (Katanin),
    γ̇_r^(l) = B_r(γ̇_r̄^(l-1), Γ) + [l >= 3] B_r(Γ, B_r(γ̇_r̄^(l-2), Γ)) + B_r(Γ, γ̇_r̄^(l-1))  (Π = G G).
Self-energy: Σ̇ = L(Γ, S) + L(γ̇^C_t̄, G) + L(Γ, G Σ̇_t̄ G), Σ̇_t̄ = L(γ̇^C_t̄, G), with L the loop
(oracle.loop, which 1, 0, 2), γ̇^C_t̄ the central parts B_r(Γ, B_r(γ̇_r̄^(l-2), Γ)), l >= 3, of the
channels a and p (the t data entering only as the crossing partner); Σ̇ and the vertex
derivative are iterated together because Ġ contains Σ̇.  Integrated by the classical
fourth-order Runge-Kutta rule with fixed steps.

Parquet approximation with the Schwinger-Dyson equation (Sec. III.B): γ_r = B_r(I_r, Γ),
Σ = U L(R̂, G) + U L_ud(B_r(R̂, Γ), G) in its a- or p-channel form (L_ud the loop of the up-down
vertex alone), or its t-channel form U L(R̂, G) + U L_uu of B_a(R̂, Γ) with B_t(R̂, Γ) as
crossing-partner data (sde_map), or the mean of forms, at G = G[Σ] (L = 1), by the damped
iteration.
"""

import numpy as np

from . import oracle as O

CLS = ("K1", "K2", "K2p", "K3")


def sig_grid(n, A=5.0):
    return A * np.tan(np.pi * (-1.0 + 2.0 * (np.arange(n) + 1) / (n + 1)) / 2)


def _zero(grids):
    return {c: [np.zeros(O.class_shape(grids, k), dtype=np.complex128) for k in CLS] for c in range(3)}


def _add(a, b, f=1.0):
    return {c: [a[c][k] + f * b[c][k] for k in range(4)] for c in a}


def _classes(d):
    return [d[k] for k in CLS]


def _vertex(grids, U, has_R, gam, include=(0, 1, 2)):
    return O.Vertex(grids, U=U, has_R=has_R, channels=gam, include=include)


def mfrg_rhs(grids, nq, U, D, T, lam, gam, sR, sK, n_loops, nus, A=5.0, multiloop_sigma=True, iters=30,
             tol=1e-12):
    """(γ̇, Σ̇^R, Σ̇^K) at L = lam."""
    Gam = _vertex(grids, U, True, gam)
    P0 = O.Prop(Delta=D, T=T, sigR=sR, sigK=sK, reg=O.REG_U, lam=lam)
    d1 = O.loop(Gam, P0, nq, nus, which=1)                         # L(Γ, S), plain S
    ds = d1
    for _ in range(iters if (multiloop_sigma and n_loops >= 3) else 1):
        P = O.Prop(Delta=D, T=T, sigR=sR, sigK=sK, reg=O.REG_U, lam=lam, dsigR=ds[:, 1, 0], dsigK=ds[:, 1, 1])
        orders, central = [], _zero(grids)
        o1 = {r: _classes(O.bubble_all(Gam, Gam, P, r, nq, pi_kind=O.PI_GS)) for r in range(3)}
        orders.append(o1)
        left_prev = None
        for l in range(2, n_loops + 1):
            prev = orders[-1]
            new, left = {}, {}
            for r in range(3):
                bar = _vertex(grids, 0.0, False, prev, include=[c for c in range(3) if c != r])
                Lr = _classes(O.bubble_all(bar, Gam, P0, r, nq))
                Rr = _classes(O.bubble_all(Gam, bar, P0, r, nq))
                tot = [Lr[k] + Rr[k] for k in range(4)]
                if l >= 3:
                    lv = _vertex(grids, 0.0, False, {r: left_prev[r]}, include=(r,))
                    Cr = _classes(O.bubble_all(Gam, lv, P0, r, nq))
                    tot = [tot[k] + Cr[k] for k in range(4)]
                    central[r] = [central[r][k] + Cr[k] for k in range(4)]
                new[r], left[r] = tot, Lr
            orders.append(new)
            left_prev = left
        if not (multiloop_sigma and n_loops >= 3):
            break
        tb = O.loop(_vertex(grids, 0.0, False, central, include=(0, 1)), P0, nq, nus)
        Pt = O.Prop(Delta=D, T=T, sigR=sR, sigK=sK, reg=O.REG_U, lam=lam, dsigR=tb[:, 1, 0], dsigK=tb[:, 1, 1])
        tt = O.loop(Gam, Pt, nq, nus, which=2)
        new_ds = d1 + tb + tt
        change = np.abs(new_ds - ds).max() / max(np.abs(new_ds).max(), 1e-300)
        ds = new_ds
        if change <= tol:
            break
    dgam = _zero(grids)
    for o in orders:
        dgam = _add(dgam, o)
    return dgam, ds[:, 1, 0], ds[:, 1, 1]


def mfrg_flow(grids, nq, U, D, T, n_loops, nus, lam0=1e-3, steps=20, A=5.0, multiloop_sigma=True):
    """(γ, Σ^R, Σ^K) at L = 1 by fixed-step RK4 from L = lam0 (γ = 0, Σ = 0)."""
    n = len(nus)
    gam, sR, sK = _zero(grids), np.zeros(n, complex), np.zeros(n, complex)
    lams = np.linspace(lam0, 1.0, steps + 1)
    f = lambda lam, g, r, k: mfrg_rhs(grids, nq, U, D, T, lam, g, r, k, n_loops, nus, A, multiloop_sigma)
    for lam, lam_next in zip(lams[:-1], lams[1:]):
        h = lam_next - lam
        k1 = f(lam, gam, sR, sK)
        k2 = f(lam + h / 2, _add(gam, k1[0], h / 2), sR + h / 2 * k1[1], sK + h / 2 * k1[2])
        k3 = f(lam + h / 2, _add(gam, k2[0], h / 2), sR + h / 2 * k2[1], sK + h / 2 * k2[2])
        k4 = f(lam + h, _add(gam, k3[0], h), sR + h * k3[1], sK + h * k3[2])
        for kk, w in ((k1, 1.0), (k2, 2.0), (k3, 2.0), (k4, 1.0)):
            gam = _add(gam, kk[0], h * w / 6)
            sR = sR + h * w / 6 * kk[1]
            sK = sK + h * w / 6 * kk[2]
    return gam, sR, sK


SDE_FORMS = ("a", "p", "ap", "t", "apt")


def sde_map(grids, nq, U, Gam, P, nus, form="a"):
    """The Schwinger-Dyson self-energy (Sec. III.B) at the frequencies nus for the full vertex
    Gam and the propagators P, [n][2][2] as oracle.loop returns it:
        Σ = U L(R̂) + U Σ_f L_f / (number of forms),   X̂_r = B_r(R̂, Γ),
    with R̂ the bare vertex of unit strength and L the loop (Hartree part U L(R̂)).  The bare
    vertex, a bubble to Γ and the closing line can be drawn in each channel:
      a: L_ud of X̂_a (a slot with channel a alone, no crossing-partner data): the line joins
         legs 2' (on Γ) and 2 (on R̂) and carries the spin opposite to the external one;
      p: L_ud of X̂_p likewise;
      t: the t bubble holds legs 1', 1 on R̂ and 2', 2 on Γ, so the line must join 1 and 2',
         and it carries the external spin: with SU(2) (the magnetic combination of the
         up-up and up-down vertices is minus the up-down vertex with legs 1 and 2 exchanged)
         and crossing, the up-up t bubble of R̂ with Γ is X̂_t − X[X̂_a], X the exchange of
         legs 1 and 2; closed on 1 and 2' this is the up-up loop L_uu = L − L_ud of a vertex
         holding X̂_a in channel a and X̂_t as its crossing-partner data (the exchanged term
         reads X̂_t at the exchanged legs).
    form "ap" and "apt" average the forms (the paper combines them)."""
    Rh = O.Vertex(grids, U=1.0, has_R=True)
    s = U * O.loop(Rh, P, nq, nus)
    if form not in SDE_FORMS:
        raise ValueError("form: one of %s" % (SDE_FORMS,))
    terms = form
    X = {}
    for r in ((0,) if "a" in terms or "t" in terms else ()) + ((1,) if "p" in terms else ()) + \
            ((2,) if "t" in terms else ()):
        X[r] = _classes(O.bubble_all(Rh, Gam, P, r, nq))
    for f in terms:
        if f in "ap":
            r = 0 if f == "a" else 1
            Vx = O.Vertex(grids, channels={r: tuple(X[r])}, include=(r,))
            s = s + U / len(terms) * O.loop(Vx, P, nq, nus, ud_only=True)
        else:
            Vx = O.Vertex(grids, channels={0: tuple(X[0]), 2: tuple(X[2])}, include=(0,))
            s = s + U / len(terms) * (O.loop(Vx, P, nq, nus) - O.loop(Vx, P, nq, nus, ud_only=True))
    return s


def parquet_sde(grids, nq, U, D, T, nus, mix=0.5, tol=1e-12, maxit=400, A=5.0, form="a"):
    """(γ, Σ^R, Σ^K) of the parquet approximation with the Schwinger-Dyson self-energy in
    the form `form` of sde_map ("a", "p", "ap", "t", "apt")."""
    n = len(nus)
    gam, sR, sK = _zero(grids), np.zeros(n, complex), np.zeros(n, complex)
    for _ in range(maxit):
        P = O.Prop(Delta=D, T=T, sigR=sR, sigK=sK)
        Gam = _vertex(grids, U, True, gam)
        new = {}
        for r in range(3):
            I_r = _vertex(grids, U, True, gam, include=[c for c in range(3) if c != r])
            new[r] = _classes(O.bubble_all(I_r, Gam, P, r, nq))
        s = sde_map(grids, nq, U, Gam, P, nus, form)
        scale = max(max(np.abs(new[c][k]).max() for c in range(3) for k in range(4)), np.abs(s).max())
        change = max(max(np.abs(new[c][k] - gam[c][k]).max() for c in range(3) for k in range(4)),
                     np.abs(s[:, 1, 0] - sR).max(), np.abs(s[:, 1, 1] - sK).max()) / scale
        gam = {c: [(1 - mix) * gam[c][k] + mix * new[c][k] for k in range(4)] for c in range(3)}
        sR = (1 - mix) * sR + mix * s[:, 1, 0]
        sK = (1 - mix) * sK + mix * s[:, 1, 1]
        if change <= tol:
            break
    return gam, sR, sK
