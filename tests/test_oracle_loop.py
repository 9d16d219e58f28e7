"""Pins of the oracle's self-energy loop (Sec. II.D.2), independent of its code:

- the limits the rule uses at x = +-1 equal the integrand's values as x -> +-1, evaluated
  through the general vertex and propagator routines (numerical limit, O(1 - |x|));
- bare vertex: the loop is the Hartree shift U (n - 1/2) (Sec. III.A.1) with n from the
  Lorentzian spectral function by QUADPACK (T > 0) or in closed form (T = 0); its (c|c) and
  Keldysh components vanish;
- the principal value at v' = +-inf: a constant K1_t on the Keldysh component that picks
  G^R alone gives int dv' G^R/(2 pi i) = -1/2 (equal-time average);
- second order: with the interaction flow's homogeneity (G_L = L G, S = G, Sigma2 of degree 3
  in G), the loop of the second-order vertex is 3 Sigma2; Im Sigma2^R against the textbook
  double spectral integral of the symmetric Anderson model, converging at second order in
  the grid spacing; causality, FDR and particle-hole symmetry of the result;
- linearity in the vertex;
- the line with one self-energy insertion, G dSigma G: it is the derivative of the Dyson
  propagator along dSigma, and the loop with it is the derivative of the loop along dSigma;
- brute force: the fixed rule converges to an adaptive integration of the defining
  integrand (vertex and propagator through the general routines, x paired with -x for the
  principal value) for a seeded vertex with every class."""

import numpy as np
import pytest
from scipy import integrate

import seeded
from oracle import oracle as O

G = dict(n1=21, n2w=9, n2v=11, n3w=7, n3v=9)
K = lambda a1p, a2p, a1, a2: 8 * a1p + 4 * a2p + 2 * a1 + a2


def _seeded(U=1.0, seed=3, include=(0, 1, 2)):
    return O.Vertex(G, U=U, has_R=True, channels=seeded.seeded_vertex(G, U=U, seed=seed), include=include)


def _sigma_tables(n=17, seed=5, T=0.1):
    sR = seeded.seeded_sigma(n, seed=seed)
    sK = 2j * np.tanh(seeded.grid_freqs(n) / (2 * T)) * sR.imag         # equilibrium Keldysh part
    return sR, sK


# (propagator: 0 G, 1 S; flow scheme; lambda; Katanin tables) and lim v' P(v') for each
CASES = [(0, O.REG_DELTA, 1.0, False, 1.0), (0, O.REG_U, 0.7, False, 0.7), (1, O.REG_DELTA, 1.0, False, 0.0),
         (1, O.REG_U, 0.7, False, 1.0), (1, O.REG_T, 1.0, False, 0.0), (1, O.REG_DELTA, 1.0, True, 0.0),
         (2, O.REG_DELTA, 1.0, True, 0.0)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("nu", [0.0, 0.7, -2.3])
def test_loop_endpoint_limits(nu, case):
    which, reg, lam, katanin, m = case
    V = _seeded()
    sR, sK = _sigma_tables()
    dR, dK = _sigma_tables(13, seed=8) if katanin else (None, None)
    P = O.Prop(Delta=1.0, T=0.1, eps=0.3, sigR=sR, sigK=sK, reg=reg, lam=lam, dsigR=dR, dsigK=dK)
    M = m * np.array([[0, 1], [1, 0]])
    for side in (1, -1):
        N, E = O.loop_limits(V, P, nu, side, which=which)
        errs = []
        for d in (1e-4, 1e-5):
            a, b, c = O.loop_pieces(V, P, nu, side * (1 - d), which=which)
            errs.append((np.abs(a - N).max(), np.abs(b - side * E).max() / np.abs(E).max(), np.abs(c - M).max()))
        for k in range(3):
            assert errs[1][k] <= 0.2 * errs[0][k] + 1e-12, (side, k, errs)    # O(1 - |x|)
        assert errs[1][0] <= 1e-4 and errs[1][1] <= 1e-5 and errs[1][2] <= 1e-4, errs


@pytest.mark.parametrize("reg,lam,katanin", [(O.REG_DELTA, 1.0, False), (O.REG_U, 0.7, False),
                                             (O.REG_T, 1.0, False), (O.REG_DELTA, 1.0, True)])
def test_loop_with_single_scale_propagator_is_the_derivative(reg, lam, katanin):
    """loop(Gamma, S) = d/dLambda loop(Gamma, G_Lambda) at fixed Sigma (the self-energy flow's
    one-loop term), by central differences in the flow parameter (Delta, lambda or T); with
    the Katanin tables the derivative is taken along Sigma + Lambda dSigma."""
    V = _seeded()
    sR, sK = _sigma_tables()
    dR, dK = _sigma_tables(17, seed=8) if katanin else (None, None)     # on Sigma's grid
    D, T, eps, h = 1.0, 0.1, 0.3, 1e-4
    nus = np.array([0.0, 0.8, -2.5, 9.0])

    def G_at(t):
        par = dict(Delta=D, T=T, eps=eps, reg=reg, lam=lam)
        key = {O.REG_DELTA: "Delta", O.REG_U: "lam", O.REG_T: "T"}[reg]
        par[key] = par[key] + t
        sr, sk = (sR + t * dR, sK + t * dK) if katanin else (sR, sK)
        return O.Prop(sigR=sr, sigK=sk, **par)

    fd = (O.loop(V, G_at(h), 401, nus) - O.loop(V, G_at(-h), 401, nus)) / (2 * h)
    P = O.Prop(Delta=D, T=T, eps=eps, sigR=sR, sigK=sK, reg=reg, lam=lam, dsigR=dR, dsigK=dK)
    S = O.loop(V, P, 401, nus, which=1)
    assert np.abs(S - fd).max() <= 1e-6 * np.abs(S).max(), np.abs(S - fd).max() / np.abs(S).max()


@pytest.mark.parametrize("T", [0.1, 0.0])
def test_loop_of_bare_vertex_is_the_hartree_shift(T):
    U, D = 1.3, 1.0
    V = O.Vertex(G, U=U, has_R=True)
    for eps in (0.0, 0.3, -0.8):
        P = O.Prop(Delta=D, T=T, eps=eps)
        S = O.loop(V, P, 1001, np.array([0.0, 1.5, -4.0]))
        if T > 0:
            A = lambda v: (D / np.pi) / ((v - eps) ** 2 + D ** 2)
            n = integrate.quad(lambda v: 0.5 * (1 - np.tanh(v / (2 * T))) * A(v), -np.inf, np.inf,
                               epsabs=1e-14, epsrel=1e-14, limit=400)[0]
        else:
            n = 0.5 - np.arctan(eps / D) / np.pi
        ref = U * (n - 0.5)
        assert np.abs(S[:, 1, 0] - ref).max() <= 1e-9 * U, (eps, S[:, 1, 0], ref)   # Sigma^R
        assert np.abs(S[:, 0, 1] - ref).max() <= 1e-9 * U                           # Sigma^A
        assert np.abs(S[:, 0, 0]).max() <= 1e-12 and np.abs(S[:, 1, 1]).max() <= 1e-12


def test_loop_principal_value_at_infinity():
    """Only K1_t, constant in w, on component (c q|c c): Gamma_s = 2 K1_t (the up-up vertex's
    own-channel part, no crossing partner), and Sigma^{c|c} = -2c int dv' G^R/(2 pi i) = c."""
    c = 0.37 - 0.21j
    K1 = np.zeros((G["n1"], 16), dtype=np.complex128)
    K1[:, K(0, 1, 0, 0)] = c
    V = O.Vertex(G, channels={2: (K1, None, None, None)}, include=(2,))
    for eps in (0.0, 0.4):
        S = O.loop(V, O.Prop(Delta=0.8, T=0.05, eps=eps), 4001, np.array([0.0, 2.0]))
        assert np.abs(S[:, 0, 0] - c).max() <= 1e-9
        assert np.abs(S[:, 1, 0]).max() + np.abs(S[:, 0, 1]).max() + np.abs(S[:, 1, 1]).max() <= 1e-12


def _sigma2_spectral(nus, U, T, D, n=800):
    """Im Sigma2^R(w) = -pi U^2 int de1 de2 A1 A2 A3 [n3 (1-n1)(1-n2) + (1-n3) n1 n2],
    e3 = e1 + e2 - w, A Lorentzian (e = D tan(theta) makes A de = dtheta / pi)."""
    x, wx = np.polynomial.legendre.leggauss(n)
    th, wth = x * np.pi / 2, wx * np.pi / 2
    e = D * np.tan(th)
    nf = lambda v: 0.5 * (1 - np.tanh(v / (2 * T)))
    A = lambda v: (D / np.pi) / (v ** 2 + D ** 2)
    E1, E2 = np.meshgrid(e, e, indexing="ij")
    W = np.outer(wth, wth) / np.pi ** 2
    out = []
    for w in nus:
        E3 = E1 + E2 - w
        n1, n2, n3 = nf(E1), nf(E2), nf(E3)
        out.append(-np.pi * U ** 2 * np.sum(W * A(E3) * (n3 * (1 - n1) * (1 - n2) + (1 - n3) * n1 * n2)))
    return np.array(out)


def _loop_of_second_order_vertex(n1, nq, U, T, D, nus):
    g = dict(n1=n1, n2w=3, n2v=3, n3w=3, n3v=3)
    P = O.Prop(Delta=D, T=T)
    V0 = O.Vertex(g, U=U, has_R=True)
    ch = {r: (O.bubble_all(V0, V0, P, r, nq, classes=("K1",))["K1"], None, None, None) for r in range(3)}
    return O.loop(O.Vertex(g, channels=ch), P, nq, nus)


def test_loop_of_second_order_vertex_is_three_sigma2():
    U, T, D = 1.0, 0.1, 1.0
    nus = np.array([0.0, 0.5, 1.0, -0.5, -1.0])
    ref = _sigma2_spectral(nus[:3], U, T, D)
    errs = []
    for n1, nq in ((201, 801), (401, 1601)):
        S = _loop_of_second_order_vertex(n1, nq, U, T, D, nus) / 3
        SR = S[:, 1, 0]
        errs.append(np.abs(SR[:3].imag - ref).max())
    assert errs[1] <= 5e-4 * np.abs(ref).max() and errs[1] <= 0.35 * errs[0], errs   # O(h^2)
    # causality, FDR, conjugation and particle-hole symmetry of the finer result
    assert (SR.imag < 0).all()
    assert np.abs(S[:, 0, 1] - np.conj(SR)).max() <= 1e-14
    fdr = 2j * np.tanh(nus / (2 * T)) * SR.imag
    assert np.abs(S[:, 1, 1] - fdr).max() <= 1e-3 * np.abs(SR).max()
    assert np.abs(S[:, 0, 0]).max() <= 1e-3 * np.abs(SR).max()
    assert np.abs(SR[3:] + np.conj(SR[1:3])).max() <= 1e-12 * np.abs(SR).max()   # Re odd, Im even
    assert (SR[1:3].real < 0).all()                                               # Re Sigma2' < 0


def test_loop_is_linear_in_the_vertex():
    a, b = 0.7 - 0.2j, -1.3
    ch1 = seeded.seeded_vertex(G, U=1.0, seed=3)
    ch2 = seeded.seeded_vertex(G, U=0.4, seed=9)
    chs = {c: tuple(a * x + b * y for x, y in zip(ch1[c], ch2[c])) for c in range(3)}
    Vs = O.Vertex(G, channels=chs)
    P = O.Prop(Delta=1.0, T=0.1, eps=0.2)
    nus = np.array([0.0, 0.9, -3.1])
    V1c, V2c = O.Vertex(G, channels=ch1), O.Vertex(G, channels=ch2)
    S = O.loop(Vs, P, 401, nus)
    ref = a * O.loop(V1c, P, 401, nus) + b * O.loop(V2c, P, 401, nus)
    assert np.abs(S - ref).max() <= 1e-13 * np.abs(ref).max()


def _loop_brute(V, P, nu, A=5.0):
    """-int dv'/(2 pi i) Gamma_s . G by adaptive quadrature in x, the integrand at x and -x
    summed (symmetric principal value), each point through vertex_eval and prop_eval."""
    def f(x):
        xs = np.array([x, -x])
        nup = A * np.tan(np.pi * xs / 2)
        J = A * np.pi / 2 * (1 + np.tan(np.pi * xs / 2) ** 2)
        pts = np.stack([np.zeros(2), np.full(2, nu), nup], axis=1)
        Gs = O.vertex_eval(V, 2, 0, 1, O.SEL_FULL, pts) + O.vertex_eval(V, 2, 1, 1, O.SEL_FULL, pts)
        Gs = Gs.reshape(2, 2, 2, 2, 2)                          # [point][a1'][a2'][a1][a2]
        S = np.einsum("npqrs,nsq->npr", Gs, O.prop_eval(P, 0, nup))
        S = -(J[:, None, None] * S).sum(0) / (2j * np.pi)
        return np.concatenate([S.real.ravel(), S.imag.ravel()])
    res, _ = integrate.quad_vec(f, 0.0, 1.0, epsabs=1e-12, epsrel=1e-12, limit=20000)
    return (res[:4] + 1j * res[4:]).reshape(2, 2)


def _flat_vertex(seed=11):
    """Classes that stay finite out to the grid edges and differ between the two ends (K1
    ramps from -1 to 1 across the w grid, K2' and K3 across the v' grid), so that the rule's
    end-node limits carry weight and do not cancel between x = -1 and x = +1."""
    rng = np.random.default_rng(seed)
    rnd = lambda *sh: rng.standard_normal(sh) + 1j * rng.standard_normal(sh)
    ramp = lambda n: np.linspace(-1.0, 1.0, n)
    ch = {}
    for c in range(3):
        K1 = ramp(G["n1"])[:, None] * rnd(16)[None, :]
        K2p = ramp(G["n2v"])[None, :, None] * rnd(G["n2w"], 1, 16)
        K3 = ramp(G["n3v"])[None, None, :, None] * rnd(G["n3w"], G["n3v"], 1, 16)
        ch[c] = (0.1 * K1, None, 0.1 * K2p, 0.1 * K3)
    return O.Vertex(G, U=1.0, has_R=True, channels=ch)


@pytest.mark.parametrize("flat", [False, True])
def test_loop_fixed_rule_converges_to_adaptive_brute_force(flat):
    V = _flat_vertex() if flat else _seeded()
    P = O.Prop(Delta=1.0, T=0.1, eps=0.3)
    for nu in (0.0, 1.3):
        ref = _loop_brute(V, P, nu)
        errs = [np.abs(O.loop(V, P, nq, np.array([nu]))[0] - ref).max() / np.abs(ref).max() for nq in (1001, 4001)]
        assert errs[1] <= 0.2 * errs[0] and errs[1] <= 5e-6, (nu, errs)


def test_line_with_a_self_energy_insertion_is_the_derivative_along_dsigma():
    """G dSigma G (which 2) = d/dt G[Sigma + t dSigma] (the contour product, all four Keldysh
    entries), and loop(Gamma, G dSigma G) = d/dt loop(Gamma, G[Sigma + t dSigma]) at t = 0."""
    sR, sK = _sigma_tables()
    dR, dK = _sigma_tables(17, seed=8)
    D, T, eps, h = 1.0, 0.1, 0.3, 1e-4
    at = lambda t: O.Prop(Delta=D, T=T, eps=eps, sigR=sR + t * dR, sigK=sK + t * dK)
    P = O.Prop(Delta=D, T=T, eps=eps, sigR=sR, sigK=sK, dsigR=dR, dsigK=dK)
    v = np.array([-30.0, -2.2, -0.4, 0.0, 0.1, 0.9, 4.0, 77.0])
    line = O.prop_eval(P, 2, v)
    fd = (O.prop_eval(at(h), 0, v) - O.prop_eval(at(-h), 0, v)) / (2 * h)
    assert np.abs(line - fd).max() <= 1e-7 * np.abs(line).max()
    V = _seeded()
    nus = np.array([0.0, 0.8, -2.5, 9.0])
    S = O.loop(V, P, 401, nus, which=2)
    fdl = (O.loop(V, at(h), 401, nus) - O.loop(V, at(-h), 401, nus)) / (2 * h)
    assert np.abs(S - fdl).max() <= 1e-6 * np.abs(S).max(), np.abs(S - fdl).max() / np.abs(S).max()


def test_up_down_loop_and_the_sde_forms_at_second_order():
    """The loop of the up-down vertex alone: for a vertex holding channel a only (no crossing
    partner data) it is half the spin-summed loop (the identity the a-channel SDE form uses);
    at second order both the a- and the p-channel bubble closed this way are Σ2, against the
    textbook spectral integral (the SDE's a and p forms, with the same coefficient)."""
    U, T, D = 1.0, 0.1, 1.0
    g = dict(n1=201, n2w=3, n2v=3, n3w=3, n3v=3)
    P = O.Prop(Delta=D, T=T)
    V0 = O.Vertex(g, U=U, has_R=True)
    nus = np.array([0.5, 1.0])
    ref = _sigma2_spectral(nus, U, T, D)
    for r, coef in ((0, 1.0), (1, 1.0)):
        K1 = O.bubble_all(V0, V0, P, r, 801, classes=("K1",))["K1"]
        X = O.Vertex(g, channels={r: (K1, None, None, None)}, include=(r,))
        ud = O.loop(X, P, 801, nus, ud_only=True)
        if r == 0:
            assert np.abs(ud - O.loop(X, P, 801, nus) / 2).max() <= 1e-14 * np.abs(ud).max()
        assert np.abs(coef * ud[:, 1, 0].imag - ref).max() <= 3e-3 * np.abs(ref).max(), (r, coef * ud[:, 1, 0].imag, ref)


def test_sde_t_form_pins():
    """The Schwinger-Dyson equation's t-channel form (oracle_flow.sde_map), whose line joins
    legs 1 and 2' of the t bubble and carries the external spin (the up-up loop of B_a(R̂, Γ)
    with B_t(R̂, Γ) as crossing-partner data):
    - second order (Γ = R): the up-down t bubble of R̂ with R vanishes (Γ0's up-up part is
      zero), so the t form is the a form, i.e. the sunset the a form is pinned to;
    - third order (Γ = R + Σ_r B_r(R, R), the exact second-order vertex): on the same grids
      the t form lies exactly at the mean of the a and p forms — which differ by
      discretisation at this order — while the t term taken with the opposite sign, or twice,
      does not;
    - for a seeded vertex the t form is not that mean (it is an independent form)."""
    from oracle import oracle_flow as F
    g = dict(n1=41, n2w=13, n2v=13, n3w=9, n3v=9)
    nq, U = 401, 0.3
    nus = F.sig_grid(21)
    P = O.Prop(Delta=1.0, T=0.2)
    R = O.Vertex(g, U=U, has_R=True)
    m2 = {f: F.sde_map(g, nq, U, R, P, nus, f) for f in ("a", "t")}
    assert np.abs(m2["t"] - m2["a"]).max() <= 1e-14 * np.abs(m2["a"]).max()
    g2 = {r: F._classes(O.bubble_all(R, R, P, r, nq)) for r in range(3)}
    Gam = F._vertex(g, U, True, g2)
    m3 = {f: F.sde_map(g, nq, U, Gam, P, nus, f) for f in F.SDE_FORMS}
    s = np.abs(m3["a"]).max()
    mid = 0.5 * (m3["a"] + m3["p"])
    assert np.abs(m3["t"] - mid).max() <= 1e-13 * s
    assert np.abs(m3["apt"] - (m3["a"] + m3["p"] + m3["t"]) / 3).max() <= 1e-14 * s
    dt = m3["t"] - m3["a"]                       # the t form's own term, U (L_uu - L_ud(X̂_a))
    assert np.abs(dt).max() >= 3e-3 * s
    for wrong in (m3["a"] - dt, m3["a"] + 2 * dt):
        assert np.abs(wrong - mid).max() >= 0.5 * np.abs(dt).max()
    Vs = _seeded(U=1.0, seed=3)
    ms = {f: F.sde_map(G, 201, 1.0, Vs, P, nus, f) for f in ("a", "p", "t")}
    assert np.abs(ms["t"] - 0.5 * (ms["a"] + ms["p"])).max() >= 1e-2 * np.abs(ms["a"]).max()
