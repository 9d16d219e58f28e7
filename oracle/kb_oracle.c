/*
 * Plain FP64 CPU oracle for the Keldysh loop bubble of the single-impurity Anderson
 * model (KeldyshQFT paper, arXiv:2405.20996).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load this code.  It shares no source with the CUDA library.
 *
 * What it computes (one output point at a time, no blocking or reordering):
 *
 *   B_r(w, v, v')^{alpha} = c_r * sum_j  w_j/(2 pi i) * J(x_j)
 *        * sum_{beta} Gamma1^{...}(w, v, v''_j) Pi_r^{beta}(w, v''_j) Gamma2^{...}(w, v''_j, v')
 *
 *   - the bubble Gamma1 o Pi_r o Gamma2 of two vertices in channel r (Sec. II.D.1,
 *     "bubble_function"), with the propagator pair Pi = G G or Pi-dot = G S + S G
 *     (Sec. II.C.5, "Bubble");
 *   - the v'' integral taken by a fixed composite 5-point Gauss-Lobatto rule in the
 *     auxiliary variable x of the frequency grid v = A tan(pi x / 2)
 *     (Sec. II.G.4 and II.G.5; x covers [-1, 1] including v = +-inf, where the
 *     integrand times the Jacobian is replaced by its limit);
 *   - vertices stored as asymptotic classes K1, K2, K2', K3 per channel and read out
 *     by multilinear interpolation in x ("linear_on_aux", Sec. II.G.7) with zero
 *     values at x = +-1;
 *   - the output split into classes by which parts of the two vertices are used
 *     (Sec. II.C.1: parts whose external legs do / do not meet at one bare vertex).
 *
 * Conventions (readings of the paper where it defers to its companion paper):
 *   Keldysh: 1 = classical, 2 = quantum; G^{1|1} = G^K, G^{1|2} = G^R, G^{2|1} = G^A,
 *   G^{2|2} = 0.  Bare vertex (parquet approximation R = Gamma_0, Sec. I.B):
 *   Gamma_0^{up,down} = -U/2 on components with an odd number of quantum indices (the
 *   sign that, with the bubble's measure below and the loop's sign of the Schwinger-Dyson
 *   equation of Sec. III.B, gives the Hartree shift U (n - 1/2) of a repulsive U and a
 *   causal second-order self-energy; see og_loop).
 *   Channel variables: a: w = v1'-v2, v = (v1'+v2)/2, v' = (v1+v2')/2;
 *   p: w = v1'+v2', v = (v1'-v2')/2, v' = (v1-v2)/2; t: w = v2'-v2, v = (v1'+v1)/2,
 *   v' = (v2'+v2)/2.  Spin: only the up-down component is stored; the up-up component
 *   is Gamma(1'2'|12) - Gamma(1'2'|21) (SU(2) + crossing, Sec. II.G.3).
 *   Bubbles (antisymmetric diagram rules, Eq. (1a-c) of Sec. III.B with c_a = 1,
 *   c_p = 1/2 x 2 equal spin terms = 1, c_t = -1):
 *     a: sum G1^{a1' b4'|b3 a2} G^{b3|b3'}(v''+w/2) G^{b4|b4'}(v''-w/2) G2^{b3' a2'|a1 b4}
 *     p: sum G1^{a1' a2'|b3 b4} G^{b3|b3'}(w/2+v'') G^{b4|b4'}(w/2-v'') G2^{b3' b4'|a1 a2}
 *     t: -sum [G1uu G2ud + G1ud G2uu], G1^{a1' b3'|a1 b4}(w,v,v'') G^{b3|b3'}(v''+w/2)
 *         G^{b4|b4'}(v''-w/2) G2^{b4' a2'|b3 a2}(w,v'',v')
 *   Measure dv''/(2 pi i).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------
 * Frequency grid (Sec. II.G.4): N points x_i = -1 + 2(i+1)/(N+1), v_i = A tan(pi x_i/2).
 * The extended node list X_k = -1 + 2(k+1)/(N+1), k = -1..N adds x = -1 and x = +1,
 * where every vertex class takes the value 0.
 * ------------------------------------------------------------------------------------ */
static double nu_to_x(double nu, double A) {
    if (isinf(nu)) return nu > 0 ? 1.0 : -1.0;
    return (2.0 / PI) * atan(nu / A);
}

/* Linear interpolation stencil in x: up to two real nodes with weights. Returns the
 * number of contributing real nodes (0, 1 or 2). */
static int stencil(double nu, int n, double A, int idx[2], double wt[2]) {
    if (!isfinite(nu)) return 0;               /* value at x = +-1 is zero */
    double x = nu_to_x(nu, A);
    double d = 2.0 / (n + 1);
    int k = (int)floor((x + 1.0) / d) - 1;     /* X_k <= x < X_{k+1} */
    if (k < -1) k = -1;
    if (k > n - 1) k = n - 1;
    double Xk = -1.0 + 2.0 * (k + 1) / (n + 1);
    double t = (x - Xk) / d;
    int m = 0;
    if (k >= 0 && k <= n - 1) { idx[m] = k; wt[m] = 1.0 - t; ++m; }
    if (k + 1 >= 0 && k + 1 <= n - 1) { idx[m] = k + 1; wt[m] = t; ++m; }
    return m;
}

/* ------------------------------------------------------------------------------------
 * Vertex object: bare part plus, per channel, the four asymptotic classes (Sec. II.C.1).
 * ------------------------------------------------------------------------------------ */
typedef struct {
    int n1, n2w, n2v, n3w, n3v;   /* class grids (shared by the three channels) */
    double A;                      /* grid scale */
    double U;                      /* bare vertex strength; used only if has_R */
    int has_R;
    int mask;                      /* channels included in the vertex (bit c); see parts_uu */
    const cplx *K1[3], *K2[3], *K2p[3], *K3[3];   /* NULL = class absent (reads 0) */
} ovtx;

/* Component index of (a1', a2' | a1, a2), each given as 0 (classical) / 1 (quantum). */
static inline int kidx(int b1p, int b2p, int b1, int b2) { return 8 * b1p + 4 * b2p + 2 * b1 + b2; }

static int popc4(int c) { return (c & 1) + ((c >> 1) & 1) + ((c >> 2) & 1) + ((c >> 3) & 1); }

/* Bare vertex, up-down component, 16 Keldysh components (Sec. I.B, PA R = Gamma_0). */
static void bare_vertex(const ovtx *V, cplx out[16]) {
    for (int c = 0; c < 16; ++c) out[c] = (V->has_R && (popc4(c) & 1)) ? -0.5 * V->U : 0.0;
}

/* Add f * class(w, v, v') of channel ch into out (16 comps). k: 0 K1, 1 K2, 2 K2', 3 K3. */
static void add_class(const ovtx *V, int ch, int k, double w, double v, double vp, double f, cplx out[16]) {
    int iw[2], iv[2], ip[2];
    double ww[2], wv[2], wp[2];
    if (k == 0) {
        const cplx *D = V->K1[ch];
        if (!D) return;
        int mw = stencil(w, V->n1, V->A, iw, ww);
        for (int a = 0; a < mw; ++a)
            for (int c = 0; c < 16; ++c) out[c] += f * ww[a] * D[(size_t)iw[a] * 16 + c];
    } else if (k == 1 || k == 2) {
        const cplx *D = (k == 1) ? V->K2[ch] : V->K2p[ch];
        if (!D) return;
        double u = (k == 1) ? v : vp;
        int mw = stencil(w, V->n2w, V->A, iw, ww);
        int mv = stencil(u, V->n2v, V->A, iv, wv);
        for (int a = 0; a < mw; ++a)
            for (int b = 0; b < mv; ++b) {
                const cplx *p = D + ((size_t)iw[a] * V->n2v + iv[b]) * 16;
                double g = f * ww[a] * wv[b];
                for (int c = 0; c < 16; ++c) out[c] += g * p[c];
            }
    } else {
        const cplx *D = V->K3[ch];
        if (!D) return;
        int mw = stencil(w, V->n3w, V->A, iw, ww);
        int mv = stencil(v, V->n3v, V->A, iv, wv);
        int mp = stencil(vp, V->n3v, V->A, ip, wp);
        for (int a = 0; a < mw; ++a)
            for (int b = 0; b < mv; ++b)
                for (int e = 0; e < mp; ++e) {
                    const cplx *p = D + (((size_t)iw[a] * V->n3v + iv[b]) * V->n3v + ip[e]) * 16;
                    double g = f * ww[a] * wv[b] * wp[e];
                    for (int c = 0; c < 16; ++c) out[c] += g * p[c];
                }
    }
}

/* Leg frequencies (v1', v2', v1, v2) from channel variables, and back. */
static void legs_from(int r, double w, double v, double vp, double L[4]) {
    if (r == 0) { L[0] = v + w / 2; L[3] = v - w / 2; L[2] = vp + w / 2; L[1] = vp - w / 2; }
    else if (r == 1) { L[0] = w / 2 + v; L[1] = w / 2 - v; L[2] = w / 2 + vp; L[3] = w / 2 - vp; }
    else { L[1] = vp + w / 2; L[3] = vp - w / 2; L[0] = v - w / 2; L[2] = v + w / 2; }
}
static void chan_from(int r, const double L[4], double *w, double *v, double *vp) {
    if (r == 0) { *w = L[0] - L[3]; *v = (L[0] + L[3]) / 2; *vp = (L[2] + L[1]) / 2; }
    else if (r == 1) { *w = L[0] + L[1]; *v = (L[0] - L[1]) / 2; *vp = (L[2] - L[3]) / 2; }
    else { *w = L[1] - L[3]; *v = (L[0] + L[2]) / 2; *vp = (L[1] + L[3]) / 2; }
}

/* Parts of the up-down vertex relative to channel r, evaluated at r-variables
 * (w, v, vp) (v or vp may be +-inf): R, own classes k = 0..3 (if r is included), and the
 * sum of the other included channels (evaluated at the converted frequencies). */
typedef struct { cplx R[16]; cplx own[4][16]; cplx other[16]; } vparts;

static void parts_ud(const ovtx *V, int r, double w, double v, double vp, int want_other, vparts *P) {
    memset(P, 0, sizeof(*P));
    bare_vertex(V, P->R);
    if ((V->mask >> r) & 1)
        for (int k = 0; k < 4; ++k) add_class(V, r, k, w, v, vp, 1.0, P->own[k]);
    if (want_other) {
        double L[4];
        legs_from(r, w, v, vp, L);
        for (int c = 0; c < 3; ++c) {
            if (c == r || !((V->mask >> c) & 1)) continue;
            double wc, vc, pc;
            chan_from(c, L, &wc, &vc, &pc);
            for (int k = 0; k < 4; ++k) add_class(V, c, k, wc, vc, pc, 1.0, P->other);
        }
    }
}

/* Parts of the up-up vertex split relative to channel r (used by the t-channel bubble).
 * For the full vertex Gamma_uu(1'2'|12) = Gamma_ud(1'2'|12) - Gamma_ud(1'2'|21).  Channel by
 * channel, exchanging legs 1 and 2 turns a-reducible diagrams into t-reducible ones and
 * keeps p-reducible ones, so the r-reducible up-up part is
 *     gamma_c^uu(1'2'|12) = gamma_c^ud(1'2'|12) - gamma_{sigma(c)}^ud(1'2'|21),
 * sigma: a <-> t, p -> p.  A vertex that includes only some channels (e.g. the sum over
 * the channels other than r in a multiloop correction) takes the exchanged term from the
 * partner channel's data, whether or not the partner itself is included. */
static void parts_uu(const ovtx *V, int r, double w, double v, double vp, int want_other, vparts *P) {
    parts_ud(V, r, w, v, vp, want_other, P);
    double L[4], S[4];
    legs_from(r, w, v, vp, L);
    S[0] = L[0]; S[1] = L[1]; S[2] = L[3]; S[3] = L[2];         /* legs 1 <-> 2 */
    cplx R[16], own[4][16], oth[16];
    memset(own, 0, sizeof(own));
    memset(oth, 0, sizeof(oth));
    bare_vertex(V, R);
    for (int c = 0; c < 3; ++c) {
        if (!((V->mask >> c) & 1)) continue;
        int sc = (c == 0) ? 2 : (c == 2) ? 0 : 1;
        double wc, vc, pc;
        if (c == r) {
            /* sigma(r)-variables of the exchanged legs, written out exactly so that an
             * infinite v or v' needs no cancellation: a <-> t: (w, v, v') -> (-w, v, v');
             * p: (w, v, v') -> (w, v, -v') */
            if (r == 1) { wc = w; vc = v; pc = -vp; }
            else { wc = -w; vc = v; pc = vp; }
            for (int k = 0; k < 4; ++k) add_class(V, sc, k, wc, vc, pc, 1.0, own[k]);
        } else {
            if (!want_other) continue;
            chan_from(sc, S, &wc, &vc, &pc);
            for (int k = 0; k < 4; ++k) add_class(V, sc, k, wc, vc, pc, 1.0, oth);
        }
    }
    /* component of the exchanged term: (a1' a2' | a2 a1) */
    for (int cc = 0; cc < 16; ++cc) {
        int b1p = (cc >> 3) & 1, b2p = (cc >> 2) & 1, b1 = (cc >> 1) & 1, b2 = cc & 1;
        int sw = kidx(b1p, b2p, b2, b1);
        P->R[cc] -= R[sw];
        for (int k = 0; k < 4; ++k) P->own[k][cc] -= own[k][sw];
        P->other[cc] -= oth[sw];
    }
}

/* Selection of vertex parts (Sec. II.C.1).  For the left vertex Gamma1(w, v, v''):
 *   SEL_ZERO = R + K1_r + K2'_r   (independent of the external v)
 *   SEL_NU   = K2_r + K3_r + other channels
 * for the right vertex Gamma2(w, v'', v'):
 *   SEL_ZERO = R + K1_r + K2_r    (independent of the external v')
 *   SEL_NU   = K2'_r + K3_r + other channels
 * SEL_FULL = everything. */
enum { SEL_ZERO = 0, SEL_NU = 1, SEL_FULL = 2 };

static void vertex_select(const ovtx *V, int r, int spin_uu, int side_right, int sel, double w, double v,
                          double vp, cplx out[16]) {
    vparts P;
    int want_other = (sel != SEL_ZERO);
    if (spin_uu) parts_uu(V, r, w, v, vp, want_other, &P);
    else parts_ud(V, r, w, v, vp, want_other, &P);
    /* class that does not depend on the external argument of this side */
    int k_ext_free = side_right ? 1 : 2;   /* right: K2_r(w, v''); left: K2'_r(w, v'') */
    int k_ext_dep = side_right ? 2 : 1;
    for (int c = 0; c < 16; ++c) {
        cplx zero = P.R[c] + P.own[0][c] + P.own[k_ext_free][c];
        cplx nu = P.own[k_ext_dep][c] + P.own[3][c] + P.other[c];
        out[c] = (sel == SEL_ZERO) ? zero : (sel == SEL_NU) ? nu : zero + nu;
    }
}

/* ------------------------------------------------------------------------------------
 * Propagators (Sec. II.C.4, III.C.2): G^R = 1 / (v - eps + i Delta - Sigma^R(v)),
 * G^A = (G^R)*, G^K = G^R [Sigma^K - 2 i Delta tanh(v/2T)] G^A.  Sigma tables (optional)
 * are interpolated linearly in x with zero at x = +-1.
 * Single-scale propagator S = d/dLambda G at fixed Sigma of the flow scheme (Sec. III.C.2):
 *   reg 0, hybridisation flow: Lambda = Delta;
 *   reg 1, interaction flow: G^R = lam / (v - eps + i Delta - lam Sigma^R), i.e. the bare
 *          inverse propagator divided by lam, and G^K = G^R [Sigma^K - 2 i Delta th / lam] G^A
 *          (the equilibrium Keldysh part of the scaled bare propagator); Lambda = lam;
 *   reg 2, temperature flow: Lambda = T (only the Keldysh component depends on it).
 * ------------------------------------------------------------------------------------ */
typedef struct {
    double Delta, T, eps, A_sig;
    int n_sig;                    /* 0: Sigma = 0 */
    const cplx *sigR, *sigK;
    int reg;                      /* 0 hybridisation, 1 interaction, 2 temperature flow */
    double lam;                   /* the interaction-flow parameter (reg 1) */
    int n_dsig;                   /* > 0: Katanin substitution with the table dSigma/dLambda */
    double A_dsig;
    const cplx *dsigR, *dsigK;
    int n_gt;                     /* > 0: G^R, G^K given as tables (the G-table propagator input) */
    double A_gt;
    const cplx *gtR, *gtK;
    int n_st;                     /* > 0: S^R, S^K given as tables */
    double A_st;
    const cplx *stR, *stK;
} oprop;

/* retarded and Keldysh parts of a self-energy table at v (linear in x, zero at x = +-1) */
static void sigma_at(int n, double A, const cplx *tR, const cplx *tK, double v, cplx *sR, cplx *sK) {
    *sR = 0;
    *sK = 0;
    if (n <= 0) return;
    int id[2];
    double wt[2];
    int m = stencil(v, n, A, id, wt);
    for (int a = 0; a < m; ++a) { *sR += wt[a] * tR[id[a]]; if (tK) *sK += wt[a] * tK[id[a]]; }
}

static double tanh_ft(double v, double T) {
    if (T <= 0.0) return v > 0 ? 1.0 : (v < 0 ? -1.0 : 0.0);
    return tanh(v / (2.0 * T));
}

/* 2x2 Keldysh matrices M[a][a'] (a, a' = 0 classical, 1 quantum). which: 0 = G, 1 = S,
 * 2 = G dSigma G alone (the line with one insertion of the dSigma tables, the multiloop
 * self-energy flow's t term) */
static void prop_matrix(const oprop *P, int which, double v, cplx M[2][2]) {
    /* Tabulated lines (Sec. II.C.2-II.C.5 with the propagators given instead of computed):
     * retarded and Keldysh parts read from the tables like a self-energy (linear in x, zero at
     * x = +-1), the advanced part their conjugate; a tabulated S uses the tabulated G (or the
     * model's) only in the Katanin term. */
    if ((P->n_gt > 0 && which != 1) || (which == 1 && P->n_st > 0)) {
        cplx GR, GK, GA, XR, XK;
        if (P->n_gt > 0) {
            sigma_at(P->n_gt, P->A_gt, P->gtR, P->gtK, v, &GR, &GK);
        } else {
            cplx Gm[2][2];
            oprop Q = *P;
            Q.n_st = 0;
            prop_matrix(&Q, 0, v, Gm);
            GR = Gm[0][1];
            GK = Gm[0][0];
        }
        GA = conj(GR);
        M[1][1] = 0;
        if (which == 0) {
            M[0][0] = GK;
            M[0][1] = GR;
            M[1][0] = GA;
            return;
        }
        cplx dR = 0, dK = 0;
        if (P->n_dsig > 0) sigma_at(P->n_dsig, P->A_dsig, P->dsigR, P->dsigK, v, &dR, &dK);
        cplx dA = conj(dR);
        if (which == 2) {
            M[0][1] = GR * dR * GR;
            M[1][0] = GA * dA * GA;
            M[0][0] = GR * dR * GK + GK * dA * GA + GR * dK * GA;
            return;
        }
        sigma_at(P->n_st, P->A_st, P->stR, P->stK, v, &XR, &XK);
        M[0][0] = XK + GR * dR * GK + GK * dA * GA + GR * dK * GA;
        M[0][1] = XR + GR * dR * GR;
        M[1][0] = conj(XR) + GA * dA * GA;
        return;
    }
    cplx sR, sK;
    sigma_at(P->n_sig, P->A_sig, P->sigR, P->sigK, v, &sR, &sK);
    const double lam = (P->reg == 1) ? P->lam : 1.0;
    const cplx g0inv = v - P->eps + I * P->Delta;          /* lam times the bare inverse */
    cplx GR = 1.0 / (g0inv / lam - sR);
    cplx GA = conj(GR);
    double th = tanh_ft(v, P->T);
    cplx mid = sK - 2.0 * I * P->Delta * th / lam;
    if (which == 0) {
        M[0][0] = GR * mid * GA;
        M[0][1] = GR;
        M[1][0] = GA;
        M[1][1] = 0;
    } else if (which == 2) {
        /* the contour product G dSigma G with dSigma = [[0, dS^A], [dS^R, dS^K]] */
        cplx dR = 0, dK = 0;
        if (P->n_dsig > 0) sigma_at(P->n_dsig, P->A_dsig, P->dsigR, P->dsigK, v, &dR, &dK);
        cplx dA = conj(dR), GK = GR * mid * GA;
        M[0][1] = GR * dR * GR;
        M[1][0] = GA * dA * GA;
        M[0][0] = GR * dR * GK + GK * dA * GA + GR * dK * GA;
        M[1][1] = 0;
    } else {
        /* S^R = -(G^R)^2 d[(G^R)^-1]/dLambda: hybridisation -i (G^R)^2; interaction
         * (G^R)^2 g0inv / lam^2; temperature 0.  dmid = d(mid)/dLambda: -2i th;
         * +2i Delta th / lam^2; -2i Delta d(th)/dT.  reg 3: no flow parameter, S = 0, so
         * that with the dSigma tables S + G dSigma G is the change of G along dSigma. */
        cplx SR, dmid;
        if (P->reg == 3) {
            SR = 0;
            dmid = 0;
        } else if (P->reg == 1) {
            SR = GR * GR * g0inv / (lam * lam);
            dmid = 2.0 * I * P->Delta * th / (lam * lam);
        } else if (P->reg == 2) {
            double c = cosh(v / (2.0 * P->T));
            double dth = -v / (2.0 * P->T * P->T) / (c * c);   /* d tanh(v/2T) / dT */
            SR = 0;
            dmid = -2.0 * I * P->Delta * dth;
        } else {
            SR = -I * GR * GR;
            dmid = -2.0 * I * th;
        }
        cplx SA = conj(SR);
        M[0][0] = SR * mid * GA + GR * dmid * GA + GR * mid * SA;
        M[0][1] = SR;
        M[1][0] = SA;
        M[1][1] = 0;
        if (P->n_dsig > 0) {
            /* Katanin substitution: S -> S + G dSigma G, the contour matrix product with
             * dSigma = [[0, dS^A], [dS^R, dS^K]] in the [[K, R], [A, 0]] layout of G */
            cplx dR, dK;
            sigma_at(P->n_dsig, P->A_dsig, P->dsigR, P->dsigK, v, &dR, &dK);
            cplx dA = conj(dR), GK = GR * mid * GA;
            M[0][1] += GR * dR * GR;
            M[1][0] += GA * dA * GA;
            M[0][0] += GR * dR * GK + GK * dA * GA + GR * dK * GA;
        }
    }
}

/* lim_{v->+-inf} v * P(v): G -> lam [[0,1],[1,0]] (lam = 1 but in the interaction flow);
 * S -> [[0,1],[1,0]] in the interaction flow (S^R -> 1/v), else 0 */
static void prop_asym(const oprop *P, int which, cplx M[2][2]) {
    double g = (which == 0) ? ((P->reg == 1) ? P->lam : 1.0) : (which == 1 && P->reg == 1) ? 1.0 : 0.0;
    M[0][0] = 0; M[1][1] = 0;
    M[0][1] = M[1][0] = g;
}

/* ------------------------------------------------------------------------------------
 * Bubble integrand: 16 output components at one node.
 * x_node in [-1, 1]; returns J(x) * F(v(x)) (or its limit at x = +-1), without the
 * 1/(2 pi i), the weight and the channel prefactor.
 * pi_kind: 0 = G G, 1 = G S + S G.
 * ------------------------------------------------------------------------------------ */
typedef struct {
    const ovtx *V1, *V2;
    const oprop *P;
    int pi_kind, r, lsel, rsel;
    double w, v, vp;
} bctx;

/* Arguments of the two propagators of the bubble in channel r (Sec. II.C.5):
 * a, t: v'' + w/2 and v'' - w/2; p: w/2 + v'' and w/2 - v''. */
static void prop_args(int r, double w, double nupp, double *a3, double *a4) {
    if (r == 1) { *a3 = w / 2 + nupp; *a4 = w / 2 - nupp; }
    else { *a3 = nupp + w / 2; *a4 = nupp - w / 2; }
}

/* Pi^{b3 b3' b4 b4'} = P1^{b3|b3'}(arg3) P2^{b4|b4'}(arg4) summed over the pair kinds. */
static void pi_matrix(const bctx *B, double nupp, int at_inf, double sgn_inf, cplx Pi[2][2][2][2]) {
    double w = B->w;
    double a3, a4, s3, s4;
    prop_args(B->r, w, nupp, &a3, &a4);
    s3 = 1;
    s4 = (B->r == 1) ? -1 : 1;
    cplx G3[2][2], G4[2][2], S3[2][2], S4[2][2];
    if (at_inf) {
        /* lim v''^2 P(a3) P(a4) = s3 s4 * asym * asym (independent of the sign of v'') */
        (void)sgn_inf;
        prop_asym(B->P, 0, G3); prop_asym(B->P, 0, G4); prop_asym(B->P, 1, S3); prop_asym(B->P, 1, S4);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                G3[i][j] *= s3; S3[i][j] *= s3; G4[i][j] *= s4; S4[i][j] *= s4;
            }
    } else {
        prop_matrix(B->P, 0, a3, G3);
        prop_matrix(B->P, 0, a4, G4);
        if (B->pi_kind == 1) { prop_matrix(B->P, 1, a3, S3); prop_matrix(B->P, 1, a4, S4); }
    }
    for (int b3 = 0; b3 < 2; ++b3)
        for (int b3p = 0; b3p < 2; ++b3p)
            for (int b4 = 0; b4 < 2; ++b4)
                for (int b4p = 0; b4p < 2; ++b4p) {
                    cplx val = G3[b3][b3p] * G4[b4][b4p];
                    if (B->pi_kind == 1) val = G3[b3][b3p] * S4[b4][b4p] + S3[b3][b3p] * G4[b4][b4p];
                    Pi[b3][b3p][b4][b4p] = val;
                }
}

/* Components of the left and right vertex that meet output component o and internal
 * indices (b3, b3', b4, b4') in channel r (leg routing of the bubble, see the header). */
static void contract_idx(int r, int o, int b3, int b3p, int b4, int b4p, int *li, int *ri) {
    int a1p = (o >> 3) & 1, a2p = (o >> 2) & 1, a1 = (o >> 1) & 1, a2 = o & 1;
    if (r == 0) { *li = kidx(a1p, b4p, b3, a2); *ri = kidx(b3p, a2p, a1, b4); }
    else if (r == 1) { *li = kidx(a1p, a2p, b3, b4); *ri = kidx(b3p, b4p, a1, a2); }
    else { *li = kidx(a1p, b3p, a1, b4); *ri = kidx(b4p, a2p, b3, a2); }
}

static void contract(int r, const cplx L[16], const cplx Pi[2][2][2][2], const cplx R[16], cplx F[16]) {
    for (int o = 0; o < 16; ++o) {
        cplx s = 0;
        for (int b3 = 0; b3 < 2; ++b3)
            for (int b3p = 0; b3p < 2; ++b3p)
                for (int b4 = 0; b4 < 2; ++b4)
                    for (int b4p = 0; b4p < 2; ++b4p) {
                        int li, ri;
                        contract_idx(r, o, b3, b3p, b4, b4p, &li, &ri);
                        s += L[li] * Pi[b3][b3p][b4][b4p] * R[ri];
                    }
        F[o] += s;
    }
}

static void integrand_x(const bctx *B, double x, cplx F[16]) {
    const ovtx *V1 = B->V1, *V2 = B->V2;
    double A = V1->A;
    int at_inf = (x <= -1.0 || x >= 1.0);
    double nupp, jac;
    if (at_inf) {
        nupp = (x > 0) ? INFINITY : -INFINITY;
        jac = PI / (2.0 * A);     /* J(x) / v''^2 at x = +-1 */
    } else {
        double tn = tan(PI * x / 2);
        nupp = A * tn;
        jac = A * PI / 2 * (1.0 + tn * tn);
    }
    cplx Pi[2][2][2][2];
    pi_matrix(B, nupp, at_inf, x, Pi);
    for (int c = 0; c < 16; ++c) F[c] = 0;
    cplx L[16], R[16];
    if (B->r != 2) {
        vertex_select(V1, B->r, 0, 0, B->lsel, B->w, B->v, nupp, L);
        vertex_select(V2, B->r, 0, 1, B->rsel, B->w, nupp, B->vp, R);
        contract(B->r, L, Pi, R, F);
    } else {
        cplx Lu[16], Ru[16];
        vertex_select(V1, 2, 1, 0, B->lsel, B->w, B->v, nupp, Lu);
        vertex_select(V2, 2, 0, 1, B->rsel, B->w, nupp, B->vp, R);
        contract(2, Lu, Pi, R, F);
        vertex_select(V1, 2, 0, 0, B->lsel, B->w, B->v, nupp, L);
        vertex_select(V2, 2, 1, 1, B->rsel, B->w, nupp, B->vp, Ru);
        contract(2, L, Pi, Ru, F);
    }
    for (int c = 0; c < 16; ++c) F[c] *= jac;
}

static double chan_prefactor(int r) { return r == 2 ? -1.0 : 1.0; }

/* ------------------------------------------------------------------------------------
 * Composite 5-point Gauss-Lobatto rule on [-1, 1] with P = (Nq-1)/4 panels
 * (nodes 0, +-sqrt(3/7), +-1 of each panel; weights 32/45, 49/90, 1/10).
 * ------------------------------------------------------------------------------------ */
int og_gl5_rule(int Nq, double *x, double *wt) {
    if (Nq < 5 || (Nq - 1) % 4 != 0) return -1;
    int P = (Nq - 1) / 4;
    double h = 2.0 / P;
    double t[5] = {-1.0, -sqrt(3.0 / 7.0), 0.0, sqrt(3.0 / 7.0), 1.0};
    double u[5] = {1.0 / 10, 49.0 / 90, 32.0 / 45, 49.0 / 90, 1.0 / 10};
    for (int j = 0; j < Nq; ++j) wt[j] = 0.0;
    for (int p = 0; p < P; ++p) {
        double xl = -1.0 + p * h;
        for (int q = 0; q < 5; ++q) {
            int j = 4 * p + q;
            x[j] = (q == 4 && p == P - 1) ? 1.0 : (q == 0 && p == 0) ? -1.0 : xl + (t[q] + 1.0) * h / 2;
            wt[j] += u[q] * h / 2;
        }
    }
    return 0;
}

/* One output point with the fixed rule. */
static void bubble_point_fixed(const bctx *B, int Nq, const double *xq, const double *wq, cplx out[16]) {
    cplx acc[16], F[16];
    for (int c = 0; c < 16; ++c) acc[c] = 0;
    for (int j = 0; j < Nq; ++j) {
        integrand_x(B, xq[j], F);
        for (int c = 0; c < 16; ++c) acc[c] += wq[j] * F[c];
    }
    double cr = chan_prefactor(B->r);
    for (int c = 0; c < 16; ++c) out[c] = cr * acc[c] / (2.0 * PI * I);
}

/* Public: bubble at npts points (w, v, vp) = freqs[3i..3i+2]; out[16 i + c]. */
int og_bubble_points(const ovtx *V1, const ovtx *V2, const oprop *P, int pi_kind, int r, int lsel, int rsel,
                     int Nq, int npts, const double *freqs, cplx *out, int nthreads) {
    if (r < 0 || r > 2 || Nq < 5 || (Nq - 1) % 4) return -1;
    double *xq = malloc(sizeof(double) * Nq), *wq = malloc(sizeof(double) * Nq);
    if (!xq || !wq) { free(xq); free(wq); return -2; }
    og_gl5_rule(Nq, xq, wq);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < npts; ++i) {
        bctx B = {V1, V2, P, pi_kind, r, lsel, rsel, freqs[3 * i], freqs[3 * i + 1], freqs[3 * i + 2]};
        bubble_point_fixed(&B, Nq, xq, wq, out + (size_t)16 * i);
    }
    free(xq);
    free(wq);
    return 0;
}

/* Raw integrand J(x) F(v(x)) at given x nodes for one point (for quadrature tests). */
int og_integrand(const ovtx *V1, const ovtx *V2, const oprop *P, int pi_kind, int r, int lsel, int rsel,
                 double w, double v, double vp, int nx, const double *xs, cplx *out) {
    bctx B = {V1, V2, P, pi_kind, r, lsel, rsel, w, v, vp};
    for (int i = 0; i < nx; ++i) integrand_x(&B, xs[i], out + (size_t)16 * i);
    return 0;
}

/* Full vertex (up-down or up-up) at channel-r variables, for tests. */
int og_vertex_eval(const ovtx *V, int r, int spin_uu, int side_right, int sel, int npts, const double *freqs,
                   cplx *out) {
    for (int i = 0; i < npts; ++i)
        vertex_select(V, r, spin_uu, side_right, sel, freqs[3 * i], freqs[3 * i + 1], freqs[3 * i + 2],
                      out + (size_t)16 * i);
    return 0;
}

/* Propagator matrices at frequencies (for tests): out[4 i + 2 a + a'] */
int og_prop_eval(const oprop *P, int which, int n, const double *v, cplx *out) {
    for (int i = 0; i < n; ++i) {
        cplx M[2][2];
        prop_matrix(P, which, v[i], M);
        out[4 * i + 0] = M[0][0]; out[4 * i + 1] = M[0][1];
        out[4 * i + 2] = M[1][0]; out[4 * i + 3] = M[1][1];
    }
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Adaptive Gauss-Lobatto integrator (Sec. II.G.5): GL4 and its 7-point Kronrod
 * extension on each interval; the 13-point extension gives the error scale I_s once
 * for the whole interval; an interval is accepted when |I7 - I4| < eps |I_s|, else it
 * is split at the 7 nodes.  Vector integrand (16 comps), max-norm.
 * Nodes/weights on [-1, 1] are passed in (derived by the caller from the paper's
 * printed nodes).
 * ------------------------------------------------------------------------------------ */
typedef struct {
    const bctx *B;
    double x7[7], w4[7], w7[7];   /* 7 nodes on [-1,1]; GL4 weights (0 at the Kronrod nodes) */
    double eps, Is;
    int depth_max, evals, fail;
} adapt_t;

static double vnorm(const cplx *a) {
    double m = 0;
    for (int c = 0; c < 16; ++c) { double q = cabs(a[c]); if (q > m) m = q; }
    return m;
}

static void adapt_rec(adapt_t *S, double a, double b, const cplx fa[16], const cplx fb[16], int depth,
                      cplx out[16]) {
    double m = 0.5 * (a + b), h = 0.5 * (b - a);
    cplx f[7][16];
    memcpy(f[0], fa, sizeof(cplx) * 16);
    memcpy(f[6], fb, sizeof(cplx) * 16);
    for (int q = 1; q < 6; ++q) { integrand_x(S->B, m + h * S->x7[q], f[q]); S->evals++; }
    cplx I4[16], I7[16], d[16];
    for (int c = 0; c < 16; ++c) {
        I4[c] = 0; I7[c] = 0;
        for (int q = 0; q < 7; ++q) { I4[c] += S->w4[q] * f[q][c]; I7[c] += S->w7[q] * f[q][c]; }
        I4[c] *= h; I7[c] *= h;
        d[c] = I7[c] - I4[c];
    }
    if (vnorm(d) <= S->eps * S->Is || depth >= S->depth_max || b - a < 1e-14) {
        if (depth >= S->depth_max && vnorm(d) > S->eps * S->Is) S->fail = 1;
        memcpy(out, I7, sizeof(cplx) * 16);
        return;
    }
    for (int c = 0; c < 16; ++c) out[c] = 0;
    for (int q = 0; q < 6; ++q) {
        cplx part[16];
        adapt_rec(S, m + h * S->x7[q], m + h * S->x7[q + 1], f[q], f[q + 1], depth + 1, part);
        for (int c = 0; c < 16; ++c) out[c] += part[c];
    }
}

/* x7: the 7 GLK7 nodes, w4/w7: GL4 (zeros at Kronrod nodes) and GLK7 weights,
 * x13/w13: the 13-point rule used once for I_s.  Returns number of integrand calls,
 * negative if some interval hit the depth limit. */
int og_bubble_points_adaptive(const ovtx *V1, const ovtx *V2, const oprop *P, int pi_kind, int r, int lsel,
                              int rsel, int npts, const double *freqs, const double *x7, const double *w4,
                              const double *w7, const double *x13, const double *w13, double eps,
                              int depth_max, cplx *out, int nthreads) {
    long total = 0;
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total) reduction(| : failed)
#endif
    for (int i = 0; i < npts; ++i) {
        bctx B = {V1, V2, P, pi_kind, r, lsel, rsel, freqs[3 * i], freqs[3 * i + 1], freqs[3 * i + 2]};
        adapt_t S;
        S.B = &B;
        memcpy(S.x7, x7, sizeof(S.x7));
        memcpy(S.w4, w4, sizeof(S.w4));
        memcpy(S.w7, w7, sizeof(S.w7));
        S.eps = eps; S.depth_max = depth_max; S.evals = 0; S.fail = 0;
        cplx f13[13][16], I13[16];
        for (int q = 0; q < 13; ++q) { integrand_x(&B, x13[q], f13[q]); S.evals++; }
        for (int c = 0; c < 16; ++c) {
            I13[c] = 0;
            for (int q = 0; q < 13; ++q) I13[c] += w13[q] * f13[q][c];
        }
        S.Is = vnorm(I13);
        if (S.Is == 0) S.Is = 1e-300;
        cplx res[16];
        adapt_rec(&S, -1.0, 1.0, f13[0], f13[12], 0, res);
        double cr = chan_prefactor(r);
        for (int c = 0; c < 16; ++c) out[(size_t)16 * i + c] = cr * res[c] / (2.0 * PI * I);
        total += S.evals;
        failed |= S.fail;
    }
    return failed ? -(int)(total > 0x7fffffff ? 0x7fffffff : total) : (int)(total > 0x7fffffff ? 0x7fffffff : total);
}

/* ------------------------------------------------------------------------------------
 * Adjoint of the bubble (vector-Jacobian product).
 *
 * Convention: gradients of a real loss L on the real embedding (real and imaginary parts
 * as independent reals), bar(z) = dL/dRe z + i dL/dIm z.  B depends linearly
 * (holomorphically) on the stored class values of either vertex, so the gradient with
 * respect to a stored value e is sum over outputs o of conj(dB_o/de) bar(B_o).
 * With respect to the retarded propagator at one sample frequency, the advanced and
 * Keldysh components are functions of it in equilibrium without a self-energy table:
 * G^A = (G^R)*, G^K = tanh(v/2T) (G^R - G^A) (the FDR, Sec. II.C.4), so
 *     bar(G^R) = bar(G^{1|2}) + conj(bar(G^{2|1})) + th (bar(G^{1|1}) - conj(bar(G^{1|1}))).
 * The bare part R = Gamma_0 is a fixed parameter and gets no gradient.
 * ------------------------------------------------------------------------------------ */
typedef struct { cplx *K1[3], *K2[3], *K2p[3], *K3[3]; } ograd;   /* vertex shapes; NULL = not wanted */

static size_t cls_elems(const ovtx *V, int k) {
    if (k == 0) return (size_t)V->n1 * 16;
    if (k < 3) return (size_t)V->n2w * V->n2v * 16;
    return (size_t)V->n3w * V->n3v * V->n3v * 16;
}

static cplx **grad_slot(ograd *G, int c, int k) {
    return k == 0 ? &G->K1[c] : k == 1 ? &G->K2[c] : k == 2 ? &G->K2p[c] : &G->K3[c];
}

/* Transpose of add_class: grad(class)[corner] += f * weight * bar. */
static void add_class_adj(const ovtx *V, ograd *Gd, int ch, int k, double w, double v, double vp, double f,
                          const cplx bar[16]) {
    cplx *D = *grad_slot(Gd, ch, k);
    if (!D) return;
    int iw[2], iv[2], ip[2];
    double ww[2], wv[2], wp[2];
    if (k == 0) {
        int mw = stencil(w, V->n1, V->A, iw, ww);
        for (int a = 0; a < mw; ++a)
            for (int c = 0; c < 16; ++c) D[(size_t)iw[a] * 16 + c] += f * ww[a] * bar[c];
    } else if (k == 1 || k == 2) {
        double u = (k == 1) ? v : vp;
        int mw = stencil(w, V->n2w, V->A, iw, ww);
        int mv = stencil(u, V->n2v, V->A, iv, wv);
        for (int a = 0; a < mw; ++a)
            for (int b = 0; b < mv; ++b) {
                cplx *p = D + ((size_t)iw[a] * V->n2v + iv[b]) * 16;
                double g = f * ww[a] * wv[b];
                for (int c = 0; c < 16; ++c) p[c] += g * bar[c];
            }
    } else {
        int mw = stencil(w, V->n3w, V->A, iw, ww);
        int mv = stencil(v, V->n3v, V->A, iv, wv);
        int mp = stencil(vp, V->n3v, V->A, ip, wp);
        for (int a = 0; a < mw; ++a)
            for (int b = 0; b < mv; ++b)
                for (int e = 0; e < mp; ++e) {
                    cplx *p = D + (((size_t)iw[a] * V->n3v + iv[b]) * V->n3v + ip[e]) * 16;
                    double g = f * ww[a] * wv[b] * wp[e];
                    for (int c = 0; c < 16; ++c) p[c] += g * bar[c];
                }
    }
}

/* Transpose of vertex_select: bar holds the gradient of the 16 selected components. */
static void vertex_select_adj(const ovtx *V, ograd *Gd, int r, int spin_uu, int side_right, int sel, double w,
                              double v, double vp, const cplx bar[16]) {
    int k_ext_free = side_right ? 1 : 2;
    int k_ext_dep = side_right ? 2 : 1;
    int want_other = (sel != SEL_ZERO);
    cplx bown[4][16], both[16];
    memset(bown, 0, sizeof(bown));
    memset(both, 0, sizeof(both));
    for (int c = 0; c < 16; ++c) {
        if (sel != SEL_NU) { bown[0][c] += bar[c]; bown[k_ext_free][c] += bar[c]; }
        if (sel != SEL_ZERO) { bown[k_ext_dep][c] += bar[c]; bown[3][c] += bar[c]; both[c] += bar[c]; }
    }
    /* direct (up-down) term of parts_ud */
    if ((V->mask >> r) & 1)
        for (int k = 0; k < 4; ++k) add_class_adj(V, Gd, r, k, w, v, vp, 1.0, bown[k]);
    double L[4];
    legs_from(r, w, v, vp, L);
    if (want_other)
        for (int c = 0; c < 3; ++c) {
            if (c == r || !((V->mask >> c) & 1)) continue;
            double wc, vc, pc;
            chan_from(c, L, &wc, &vc, &pc);
            for (int k = 0; k < 4; ++k) add_class_adj(V, Gd, c, k, wc, vc, pc, 1.0, both);
        }
    if (!spin_uu) return;
    /* exchanged term of parts_uu: X[cc] -= X'[sw(cc)], so bar(X')[sw(cc)] = -bar(X)[cc] */
    cplx sown[4][16], soth[16];
    for (int cc = 0; cc < 16; ++cc) {
        int b1p = (cc >> 3) & 1, b2p = (cc >> 2) & 1, b1 = (cc >> 1) & 1, b2 = cc & 1;
        int sw = kidx(b1p, b2p, b2, b1);
        for (int k = 0; k < 4; ++k) sown[k][sw] = -bown[k][cc];
        soth[sw] = -both[cc];
    }
    double S[4];
    S[0] = L[0]; S[1] = L[1]; S[2] = L[3]; S[3] = L[2];
    for (int c = 0; c < 3; ++c) {
        if (!((V->mask >> c) & 1)) continue;
        int sc = (c == 0) ? 2 : (c == 2) ? 0 : 1;
        double wc, vc, pc;
        if (c == r) {
            if (r == 1) { wc = w; vc = v; pc = -vp; }
            else { wc = -w; vc = v; pc = vp; }
            for (int k = 0; k < 4; ++k) add_class_adj(V, Gd, sc, k, wc, vc, pc, 1.0, sown[k]);
        } else {
            if (!want_other) continue;
            chan_from(sc, S, &wc, &vc, &pc);
            for (int k = 0; k < 4; ++k) add_class_adj(V, Gd, sc, k, wc, vc, pc, 1.0, soth);
        }
    }
}

/* Adjoint of one output point: bar holds bar(B_o) for its 16 components. gGR (or NULL)
 * is this point's bosonic row of the propagator-gradient table, [j][side] with side 0 the
 * propagator at arg3 and side 1 the one at arg4 (prop_args). */
static void bubble_point_vjp(const bctx *B, int Nq, const double *xq, const double *wq, const cplx gbar[16],
                             ograd *G1, ograd *G2, cplx *gGR) {
    const ovtx *V1 = B->V1, *V2 = B->V2;
    double A = V1->A, cr = chan_prefactor(B->r);
    int nterm = (B->r == 2) ? 2 : 1;
    for (int j = 0; j < Nq; ++j) {
        double x = xq[j];
        int at_inf = (x <= -1.0 || x >= 1.0);
        double nupp, jac;
        if (at_inf) {
            nupp = (x > 0) ? INFINITY : -INFINITY;
            jac = PI / (2.0 * A);
        } else {
            double tn = tan(PI * x / 2);
            nupp = A * tn;
            jac = A * PI / 2 * (1.0 + tn * tn);
        }
        cplx sj = cr * wq[j] * jac / (2.0 * PI * I);
        cplx Pi[2][2][2][2];
        pi_matrix(B, nupp, at_inf, x, Pi);
        cplx bPi[2][2][2][2];
        memset(bPi, 0, sizeof(bPi));
        for (int term = 0; term < nterm; ++term) {
            /* a, p: (ud, ud); t: term 0 = (uu, ud), term 1 = (ud, uu) */
            int uuL = (B->r == 2) && term == 0, uuR = (B->r == 2) && term == 1;
            cplx L[16], R[16], bL[16], bR[16];
            vertex_select(V1, B->r, uuL, 0, B->lsel, B->w, B->v, nupp, L);
            vertex_select(V2, B->r, uuR, 1, B->rsel, B->w, nupp, B->vp, R);
            memset(bL, 0, sizeof(bL));
            memset(bR, 0, sizeof(bR));
            for (int o = 0; o < 16; ++o)
                for (int b3 = 0; b3 < 2; ++b3)
                    for (int b3p = 0; b3p < 2; ++b3p)
                        for (int b4 = 0; b4 < 2; ++b4)
                            for (int b4p = 0; b4p < 2; ++b4p) {
                                int li, ri;
                                contract_idx(B->r, o, b3, b3p, b4, b4p, &li, &ri);
                                cplx p = Pi[b3][b3p][b4][b4p];
                                bL[li] += conj(sj * p * R[ri]) * gbar[o];
                                bR[ri] += conj(sj * L[li] * p) * gbar[o];
                                bPi[b3][b3p][b4][b4p] += conj(sj * L[li] * R[ri]) * gbar[o];
                            }
            if (G1) vertex_select_adj(V1, G1, B->r, uuL, 0, B->lsel, B->w, B->v, nupp, bL);
            if (G2) vertex_select_adj(V2, G2, B->r, uuR, 1, B->rsel, B->w, nupp, B->vp, bR);
        }
        if (!gGR || at_inf || B->pi_kind != 0) continue;
        /* Pi = G(a3) (x) G(a4); then G^A = (G^R)*, G^K = th (G^R - G^A) */
        double a3, a4;
        prop_args(B->r, B->w, nupp, &a3, &a4);
        cplx G3[2][2], G4[2][2], bG3[2][2], bG4[2][2];
        prop_matrix(B->P, 0, a3, G3);
        prop_matrix(B->P, 0, a4, G4);
        memset(bG3, 0, sizeof(bG3));
        memset(bG4, 0, sizeof(bG4));
        for (int b3 = 0; b3 < 2; ++b3)
            for (int b3p = 0; b3p < 2; ++b3p)
                for (int b4 = 0; b4 < 2; ++b4)
                    for (int b4p = 0; b4p < 2; ++b4p) {
                        bG3[b3][b3p] += conj(G4[b4][b4p]) * bPi[b3][b3p][b4][b4p];
                        bG4[b4][b4p] += conj(G3[b3][b3p]) * bPi[b3][b3p][b4][b4p];
                    }
        double th3 = tanh_ft(a3, B->P->T), th4 = tanh_ft(a4, B->P->T);
        gGR[2 * j + 0] += bG3[0][1] + conj(bG3[1][0]) + th3 * (bG3[0][0] - conj(bG3[0][0]));
        gGR[2 * j + 1] += bG4[0][1] + conj(bG4[1][0]) + th4 * (bG4[0][0] - conj(bG4[0][0]));
    }
}

/* Private copy of the wanted gradient arrays (zeroed); returns the buffer or NULL. */
static cplx *grad_private(const ovtx *V, const ograd *src, ograd *dst) {
    size_t tot = 0;
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 4; ++k)
            if (*grad_slot((ograd *)src, c, k)) tot += cls_elems(V, k);
    cplx *buf = calloc(tot > 0 ? tot : 1, sizeof(cplx));
    if (!buf) return NULL;
    size_t off = 0;
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 4; ++k) {
            if (*grad_slot((ograd *)src, c, k)) { *grad_slot(dst, c, k) = buf + off; off += cls_elems(V, k); }
            else *grad_slot(dst, c, k) = NULL;
        }
    return buf;
}

static void grad_accumulate(const ovtx *V, const ograd *priv, ograd *dst) {
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 4; ++k) {
            cplx *d = *grad_slot(dst, c, k), *p = *grad_slot((ograd *)priv, c, k);
            if (!d || !p) continue;
            size_t n = cls_elems(V, k);
            for (size_t i = 0; i < n; ++i) d[i] += p[i];
        }
}

/* Public: VJP at npts output points (w, v, vp) = freqs[3i..3i+2] with gradients
 * gbar[16 i + c].  G1, G2 (either may be NULL) receive += the gradients with respect to
 * the stored classes of V1 and V2; gGR (or NULL; n_gr entries) receives += the gradient
 * with respect to G^R at the samples [iw[i]][j][side].  pi_kind must be 0 (G G) and P
 * must have no self-energy table when gGR is given. */
int og_bubble_vjp_points(const ovtx *V1, const ovtx *V2, const oprop *P, int pi_kind, int r, int lsel, int rsel,
                         int Nq, int npts, const double *freqs, const cplx *gbar, const int *iw, ograd *G1,
                         ograd *G2, cplx *gGR, int n_gr, int nthreads) {
    if (r < 0 || r > 2 || Nq < 5 || (Nq - 1) % 4) return -1;
    if (gGR && (pi_kind != 0 || P->n_sig > 0 || P->n_dsig > 0 || !iw)) return -3;
    double *xq = malloc(sizeof(double) * Nq), *wq = malloc(sizeof(double) * Nq);
    if (!xq || !wq) { free(xq); free(wq); return -2; }
    og_gl5_rule(Nq, xq, wq);
    int fail = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        ograd p1, p2;
        cplx *b1 = G1 ? grad_private(V1, G1, &p1) : NULL;
        cplx *b2 = G2 ? grad_private(V2, G2, &p2) : NULL;
        cplx *pg = gGR ? calloc((size_t)n_gr, sizeof(cplx)) : NULL;
        int ok = (!G1 || b1) && (!G2 || b2) && (!gGR || pg);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int i = 0; i < npts; ++i) {
            if (!ok) continue;
            if (gGR && ((size_t)iw[i] + 1) * Nq * 2 > (size_t)n_gr) { ok = 0; continue; }
            bctx B = {V1, V2, P, pi_kind, r, lsel, rsel, freqs[3 * i], freqs[3 * i + 1], freqs[3 * i + 2]};
            bubble_point_vjp(&B, Nq, xq, wq, gbar + (size_t)16 * i, G1 ? &p1 : NULL, G2 ? &p2 : NULL,
                             gGR ? pg + (size_t)iw[i] * Nq * 2 : NULL);
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            if (!ok) fail = 1;
            else {
                if (G1) grad_accumulate(V1, &p1, G1);
                if (G2) grad_accumulate(V2, &p2, G2);
                if (gGR) for (int i = 0; i < n_gr; ++i) gGR[i] += pg[i];
            }
        }
        free(b1);
        free(b2);
        free(pg);
    }
    free(xq);
    free(wq);
    return fail ? -2 : 0;
}

/* ------------------------------------------------------------------------------------
 * Self-energy loop (Sec. II.D.2, the `loop` function): the vertex closed by one
 * propagator line,
 *   Sigma^{a1'|a1}(v) = - int dv'/(2 pi i) sum_{a2', a2} Gamma_s^{a1' a2'|a1 a2}(v, v'|v, v')
 *                          P^{a2|a2'}(v'),
 *   Gamma_s = Gamma_ud + Gamma_uu   (the internal line's spin summed, SU(2)),
 * the vertex read in t-channel variables (w_t = 0, v_t = v, v'_t = v').  Sigma is a 2x2
 * Keldysh matrix: (q|c) = Sigma^R, (c|q) = Sigma^A, (q|q) = Sigma^K, (c|c) = 0 for a causal
 * result.  Readings (the loop's equation is in the companion paper): the measure is the
 * bubble's dv'/(2 pi i) and the sign is the minus of the first term of the Schwinger-Dyson
 * equation (Sec. III.B):
 *   Sigma = - int dv'/(2 pi i) Gamma_s . P,
 * so that the bare vertex (-U/2) gives the Hartree shift U (n - 1/2) of Sec. III.A.1 and the
 * second-order vertex gives a causal self-energy obeying the FDR; the v' integral is the
 * symmetric principal value at v' = +-inf (equal-time average of the retarded and advanced
 * lines).
 *
 * Discretisation (the bubble's composite GL5 rule in x = (2/pi) atan(v'/A)): the vertex
 * splits into its v'-independent part C(v) (R, K1_t(0), K2_t(0, v) and the crossed
 * K1_a(0), K2_a(0, v)) and the rest D(v, v'), which vanishes at x = +-1.  Then
 *   Sigma = C(v) . I_P + int D P,   I_P = int dv' [P(v') - M v'/(v'^2 + A^2)]
 * with M = lim v' P(v'): the subtracted term is odd and integrates to zero.  At x = +-1 the
 * rule takes the limits of the integrands times J(x) = dv'/dx:
 *   J [P - M v'/(v'^2+A^2)] -> (pi / 2A) N_+-,   N_+- = lim_{v' -> +-inf} v' (v' P - M);
 *   J D P -> +-M . D_+-,   D_+- = sum over the classes that decay through one argument
 *   y ~ +-v' of (their value at the last grid node along that argument) (N + 1)/2,
 * since a class interpolated to zero at x = +-1 falls like (1 -+ x_y) (N + 1)/2 and
 * (1 -+ x_y) v' -> 2A/pi, while J P -> (pi/2A) M v'.  Classes with two diverging
 * arguments fall like 1/v'^2 and drop out.  P = G, or P = S of the flow scheme (with the
 * Katanin substitution when its tables are set) for the self-energy flow's loop(Gamma, S).
 * ------------------------------------------------------------------------------------ */

/* N_+- = lim_{v' -> +-inf} v' (v' P - M) (side = +1 or -1), with Sigma (and dSigma) tables
 * vanishing at x = +-1 and th = tanh(+-inf) = +-1:
 *   G: v' G^R = lam v' / (v' - eps + i Delta - lam Sigma^R) gives N^R = lam (eps - i Delta),
 *      and v'^2 G^K -> lam^2 (-2 i Delta th / lam);
 *   S, hybridisation flow: S^R = -i (G^R)^2 gives N^R = -i; S^K -> G^R (-2 i th) G^A;
 *   S, interaction flow: S = G / lam at Sigma = 0 to this order: N^R = eps - i Delta,
 *      N^K = -2 i Delta th;
 *   S, temperature flow: S^R = 0 and S^K falls exponentially: N = 0.
 * The Katanin term G dSigma G falls like 1/v'^3 and adds nothing, and the line G dSigma G
 * alone (which 2) has N = 0.  N^A = (N^R)*. */
static void prop_tail2(const oprop *P, int which, int side, cplx N[2][2]) {
    const double lam = (P->reg == 1) ? P->lam : 1.0;
    const double th = (double)side;
    if (which == 2) {
        N[0][1] = 0;
        N[0][0] = 0;
    } else if (which == 0) {
        N[0][1] = lam * (P->eps - I * P->Delta);
        N[0][0] = -2.0 * I * P->Delta * th * lam;
    } else if (P->reg == 1) {
        N[0][1] = P->eps - I * P->Delta;
        N[0][0] = -2.0 * I * P->Delta * th;
    } else if (P->reg == 2 || P->reg == 3) {
        N[0][1] = 0;
        N[0][0] = 0;
    } else {
        N[0][1] = -I;
        N[0][0] = -2.0 * I * th;
    }
    N[1][0] = conj(N[0][1]);
    N[1][1] = 0;
}

/* f * (value of class k of channel ch at its edge node along `axis` (0 w, 1 v, 2 v'),
 * side +1 = last node, -1 = first node, interpolated in the other arguments), times
 * (N + 1)/2 = 1 / (1 - X_last). */
static void class_edge(const ovtx *V, int ch, int k, int axis, int side, double w, double v, double vp, double f,
                       cplx out[16]) {
    int nw, nv = 1, np = 1;
    const cplx *D;
    if (k == 0) { D = V->K1[ch]; nw = V->n1; }
    else if (k == 1) { D = V->K2[ch]; nw = V->n2w; nv = V->n2v; }
    else if (k == 2) { D = V->K2p[ch]; nw = V->n2w; np = V->n2v; }
    else { D = V->K3[ch]; nw = V->n3w; nv = V->n3v; np = V->n3v; }
    if (!D) return;
    int iw[2], iv[2], ip[2], mw, mv, mp;
    double ww[2], wv[2], wp[2];
    int nax = (axis == 0) ? nw : (axis == 1) ? nv : np;
    double g = f * 0.5 * (nax + 1);
    if (axis == 0) { mw = 1; iw[0] = side > 0 ? nw - 1 : 0; ww[0] = g; }
    else mw = stencil(w, nw, V->A, iw, ww);
    if (k == 1 || k == 3) {
        if (axis == 1) { mv = 1; iv[0] = side > 0 ? nv - 1 : 0; wv[0] = g; }
        else mv = stencil(v, nv, V->A, iv, wv);
    } else { mv = 1; iv[0] = 0; wv[0] = 1.0; }
    if (k == 2 || k == 3) {
        if (axis == 2) { mp = 1; ip[0] = side > 0 ? np - 1 : 0; wp[0] = g; }
        else mp = stencil(vp, np, V->A, ip, wp);
    } else { mp = 1; ip[0] = 0; wp[0] = 1.0; }
    for (int a = 0; a < mw; ++a)
        for (int b = 0; b < mv; ++b)
            for (int e = 0; e < mp; ++e) {
                size_t row = ((size_t)iw[a] * nv + iv[b]) * np + ip[e];
                double c = ww[a] * wv[b] * wp[e];
                for (int q = 0; q < 16; ++q) out[q] += c * D[row * 16 + q];
            }
}

/* D_+- of Gamma_s = 2 Gamma_ud(v, v'|v, v') - Gamma_ud(v, v'|v', v) at v' -> side * inf
 * (the exchanged term with Keldysh indices (a1' a2'|a2 a1); each channel's exchanged term
 * comes from its crossing partner's data, a <-> t, p -> p, as for the up-up vertex). */
static void loop_edge(const ovtx *V, double nu, int side, int ud_only, cplx E[16]) {
    cplx ud[16], ex[16];
    memset(ud, 0, sizeof(ud));
    memset(ex, 0, sizeof(ex));
    /* direct legs (v, v'|v, v'): t (0, v, v'), a (v - v', ., .), p (v + v', ., .) */
    if ((V->mask >> 2) & 1) {
        class_edge(V, 2, 2, 2, side, 0.0, nu, 0.0, 1.0, ud);   /* K2'_t(0, v') */
        class_edge(V, 2, 3, 2, side, 0.0, nu, 0.0, 1.0, ud);   /* K3_t(0, v, v') */
    }
    if ((V->mask >> 0) & 1) class_edge(V, 0, 0, 0, -side, 0.0, 0.0, 0.0, 1.0, ud);   /* K1_a(v - v') */
    if ((V->mask >> 1) & 1) class_edge(V, 1, 0, 0, side, 0.0, 0.0, 0.0, 1.0, ud);    /* K1_p(v + v') */
    /* exchanged legs (v, v'|v', v): t (v' - v, ., .), a (0, v, v'), p (v + v', ., .) */
    if ((V->mask >> 0) & 1) class_edge(V, 2, 0, 0, side, 0.0, 0.0, 0.0, 1.0, ex);    /* K1_t(v' - v) */
    if ((V->mask >> 2) & 1) {
        class_edge(V, 0, 2, 2, side, 0.0, nu, 0.0, 1.0, ex);   /* K2'_a(0, v') */
        class_edge(V, 0, 3, 2, side, 0.0, nu, 0.0, 1.0, ex);   /* K3_a(0, v, v') */
    }
    if ((V->mask >> 1) & 1) class_edge(V, 1, 0, 0, side, 0.0, 0.0, 0.0, 1.0, ex);    /* K1_p(v + v') */
    for (int c = 0; c < 16; ++c) {
        int b1p = (c >> 3) & 1, b2p = (c >> 2) & 1, b1 = (c >> 1) & 1, b2 = c & 1;
        E[c] = ud_only ? ud[c] : 2.0 * ud[c] - ex[kidx(b1p, b2p, b2, b1)];
    }
}

/* Gamma_s . P contracted over the internal line: S[a1'][a1] += f sum G[a1' a2'|a1 a2] P[a2][a2'] */
static void loop_contract(const cplx G[16], cplx P[2][2], cplx f, cplx S[2][2]) {
    for (int a1p = 0; a1p < 2; ++a1p)
        for (int a1 = 0; a1 < 2; ++a1) {
            cplx s = 0;
            for (int a2p = 0; a2p < 2; ++a2p)
                for (int a2 = 0; a2 < 2; ++a2) s += G[kidx(a1p, a2p, a1, a2)] * P[a2][a2p];
            S[a1p][a1] += f * s;
        }
}

/* Gamma_s = Gamma_ud + Gamma_uu (or Gamma_ud alone) of the right-vertex selection sel at
 * t-variables (0, v, v') */
static void loop_vertex(const ovtx *V, int sel, double nu, double nup, int ud_only, cplx G[16]) {
    cplx a[16], b[16];
    vertex_select(V, 2, 0, 1, sel, 0.0, nu, nup, a);
    if (ud_only) { for (int c = 0; c < 16; ++c) G[c] = a[c]; return; }
    vertex_select(V, 2, 1, 1, sel, 0.0, nu, nup, b);
    for (int c = 0; c < 16; ++c) G[c] = a[c] + b[c];
}

/* Public: Sigma at npts frequencies nus with P = G (which 0), S (which 1) or G dSigma G (which 2);
 * out[4 i + 2 a1' + a1] (0 classical, 1 quantum). */
int og_loop_spin(const ovtx *V, const oprop *P, int which, int ud_only, int Nq, int npts, const double *nus,
                 cplx *out, int nthreads);
int og_loop(const ovtx *V, const oprop *P, int which, int Nq, int npts, const double *nus, cplx *out,
            int nthreads) {
    return og_loop_spin(V, P, which, 0, Nq, npts, nus, out, nthreads);
}

/* The loop with the up-down vertex alone when ud_only (the closed line carrying the spin
 * opposite to the external one, as in the Schwinger-Dyson equation's bubble forms). */
int og_loop_spin(const ovtx *V, const oprop *P, int which, int ud_only, int Nq, int npts, const double *nus,
                 cplx *out, int nthreads) {
    if (Nq < 5 || (Nq - 1) % 4 || which < 0 || which > 2) return -1;
    double *xq = malloc(sizeof(double) * Nq), *wq = malloc(sizeof(double) * Nq);
    if (!xq || !wq) { free(xq); free(wq); return -2; }
    og_gl5_rule(Nq, xq, wq);
    const double A = V->A;
    cplx M[2][2], Np[2][2], Nm[2][2], IP[2][2];
    prop_asym(P, which, M);
    prop_tail2(P, which, +1, Np);
    prop_tail2(P, which, -1, Nm);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            IP[a][b] = (wq[0] * Nm[a][b] + wq[Nq - 1] * Np[a][b]) * (PI / (2.0 * A));
    for (int j = 1; j < Nq - 1; ++j) {
        double tn = tan(PI * xq[j] / 2), nup = A * tn, jac = A * PI / 2 * (1.0 + tn * tn);
        cplx G[2][2];
        prop_matrix(P, which, nup, G);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) IP[a][b] += wq[j] * jac * (G[a][b] - M[a][b] * nup / (nup * nup + A * A));
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < npts; ++i) {
        const double nu = nus[i];
        cplx S[2][2] = {{0, 0}, {0, 0}}, Cv[16], E[16];
        loop_vertex(V, SEL_ZERO, nu, 0.0, ud_only, Cv);
        loop_contract(Cv, IP, 1.0, S);
        for (int j = 1; j < Nq - 1; ++j) {
            double tn = tan(PI * xq[j] / 2), nup = A * tn, jac = A * PI / 2 * (1.0 + tn * tn);
            cplx G[2][2], D[16];
            prop_matrix(P, which, nup, G);
            loop_vertex(V, SEL_NU, nu, nup, ud_only, D);
            loop_contract(D, G, wq[j] * jac, S);
        }
        loop_edge(V, nu, +1, ud_only, E);
        loop_contract(E, M, wq[Nq - 1], S);
        loop_edge(V, nu, -1, ud_only, E);
        loop_contract(E, M, -wq[0], S);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) out[(size_t)4 * i + 2 * a + b] = -S[a][b] / (2.0 * PI * I);
    }
    free(xq);
    free(wq);
    return 0;
}

/* Integrand pieces of the loop at one x in (-1, 1), for limit tests:
 * out[0..3] = J (P - M v'/(v'^2 + A^2))  -> (pi/2A) N_+- at x -> +-1,
 * out[4..19] = (pi/2A) v' D(v, v')       -> +-D_+-  (D: the v'-dependent part of Gamma_s),
 * out[20..23] = v' P(v')                 -> M  (P = G for which 0, S for which 1). */
int og_loop_pieces(const ovtx *V, const oprop *P, int which, double nu, double x, cplx *out) {
    const double A = V->A;
    double tn = tan(PI * x / 2), nup = A * tn, jac = A * PI / 2 * (1.0 + tn * tn);
    cplx G[2][2], M[2][2], D[16];
    prop_matrix(P, which, nup, G);
    prop_asym(P, which, M);
    loop_vertex(V, SEL_NU, nu, nup, 0, D);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            out[2 * a + b] = jac * (G[a][b] - M[a][b] * nup / (nup * nup + A * A));
            out[20 + 2 * a + b] = nup * G[a][b];
        }
    for (int c = 0; c < 16; ++c) out[4 + c] = (PI / (2.0 * A)) * nup * D[c];
    return 0;
}

/* The limits the rule uses at x = +-1 (side): out[0..3] = (pi/2A) N_+-, out[4..19] = D_+-. */
int og_loop_limits(const ovtx *V, const oprop *P, int which, double nu, int side, cplx *out) {
    cplx N[2][2], E[16];
    prop_tail2(P, which, side, N);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) out[2 * a + b] = N[a][b] * (PI / (2.0 * V->A));
    memset(E, 0, sizeof(E));
    loop_edge(V, nu, side, 0, E);
    for (int c = 0; c < 16; ++c) out[4 + c] = E[c];
    return 0;
}
