// Device helpers shared by the FP64 and mixed-precision kernels: complex FP64 arithmetic,
// propagators (Sec. II.C.4, III.C.2), the x-grid stencil (Sec. II.G.4, II.G.7), channel
// frequency maps (Sec. II.C.1) and the Pi table (Sec. II.C.5).
#pragma once
#include <cuda_runtime.h>

#include "kb_internal.h"

namespace kb {

// Bounds-checked builds (compiled with -DKB_CHECKED): every vertex record index that comes
// from a frequency lookup (the stencil corners of a gather, of an adjoint scatter) is checked
// against the record count of its class before the access; an index outside it is counted,
// the first one kept (site << 48 | index), and the access skipped.  kb_check_device reports
// them.  In the normal build the check is the constant true and costs nothing.
enum { KB_SITE_MIXED_REC = 1, KB_SITE_K2_GATHER = 2, KB_SITE_FP64_REC = 3, KB_SITE_FP64_ADJ = 4,
       KB_SITE_MIXED_ADJ = 5 };
#ifdef KB_CHECKED
namespace {
__device__ unsigned int kb_oob_count;
__device__ unsigned long long kb_oob_first;
unsigned kb_oob_take_here(unsigned long long* first) {
    unsigned n = 0;
    if (cudaMemcpyFromSymbol(&n, kb_oob_count, sizeof n) != cudaSuccess) return 0;
    if (n) {
        cudaMemcpyFromSymbol(first, kb_oob_first, sizeof *first);
        const unsigned z = 0;
        cudaMemcpyToSymbol(kb_oob_count, &z, sizeof z);
    }
    return n;
}
const bool kb_oob_registered = kb_oob_register(&kb_oob_take_here);
}  // namespace
__device__ __forceinline__ bool kb_rec_ok(long long idx, long long n, int site) {
    if (idx >= 0 && idx < n) return true;
    if (atomicAdd(&kb_oob_count, 1u) == 0u)
        kb_oob_first = ((unsigned long long)site << 48) | ((unsigned long long)idx & 0xffffffffffffull);
    return false;
}
#else
__device__ __forceinline__ bool kb_rec_ok(long long, long long, int) { return true; }
#endif

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cinv(double2 a) {
    const double id = 1.0 / (a.x * a.x + a.y * a.y);
    return make_double2(a.x * id, -a.y * id);
}
// z += a * b
__device__ __forceinline__ void cfma(double2& z, double2 a, double2 b) {
    z.x = fma(a.x, b.x, fma(-a.y, b.y, z.x));
    z.y = fma(a.x, b.y, fma(a.y, b.x, z.y));
}

constexpr double KB_PI = 3.14159265358979323846;

// Linear stencil in x on an n-point grid with zero-valued virtual nodes at x = -1 and x = 1.
// Returns the lower node k in [-1, n-1] and the weight t of node k+1; non-finite v gives
// k = -2 (the class contributes nothing).
__device__ __forceinline__ int xstencil(double v, int n, double A, double& t) {
    if (!isfinite(v)) return -2;
    double x = (2.0 / KB_PI) * atan(v / A);
    double s = (x + 1.0) * (0.5 * (n + 1));   // position in units of the spacing, X_k at s = k + 1
    double fk = floor(s);
    int k = (int)fk - 1;
    if (k < -1) k = -1;
    if (k > n - 1) k = n - 1;
    double Xk = -1.0 + 2.0 * (k + 1) / (n + 1);
    t = (x - Xk) * (0.5 * (n + 1));
    return k;
}

// legs (v1', v2', v1, v2) from channel variables (w, v, vp) and back (Sec. II.C.1)
__device__ __forceinline__ void legs_of(int r, double w, double v, double vp, double L[4]) {
    if (r == KB_CH_A) { L[0] = v + 0.5 * w; L[3] = v - 0.5 * w; L[2] = vp + 0.5 * w; L[1] = vp - 0.5 * w; }
    else if (r == KB_CH_P) { L[0] = 0.5 * w + v; L[1] = 0.5 * w - v; L[2] = 0.5 * w + vp; L[3] = 0.5 * w - vp; }
    else { L[1] = vp + 0.5 * w; L[3] = vp - 0.5 * w; L[0] = v - 0.5 * w; L[2] = v + 0.5 * w; }
}
__device__ __forceinline__ void vars_of(int c, const double L[4], double& w, double& v, double& vp) {
    if (c == KB_CH_A) { w = L[0] - L[3]; v = 0.5 * (L[0] + L[3]); vp = 0.5 * (L[2] + L[1]); }
    else if (c == KB_CH_P) { w = L[0] + L[1]; v = 0.5 * (L[0] - L[1]); vp = 0.5 * (L[2] - L[3]); }
    else { w = L[1] - L[3]; v = 0.5 * (L[0] + L[2]); vp = 0.5 * (L[1] + L[3]); }
}

// tanh(v / 2T); the argument as v times 1/(2T), a loop invariant of the callers (GB300's
// FP64 divide costs several FMA issue slots)
__device__ __forceinline__ double tanh_T(double v, double T) {
    if (T <= 0.0) return v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0);
    return tanh(v * (0.5 / T));
}

// Retarded and Keldysh parts of a line table at v (n points on the tan grid of scale A,
// linear in x, zero at x = +-1).
__device__ __forceinline__ void line_table(const double2* tR, const double2* tK, int n, double A, double v,
                                           double2& R, double2& K) {
    R = make_double2(0, 0);
    K = make_double2(0, 0);
    double t;
    int k = xstencil(v, n, A, t);
    if (k >= 0) { R = cadd(R, cscale(tR[k], 1.0 - t)); K = cadd(K, cscale(tK[k], 1.0 - t)); }
    if (k >= -1 && k + 1 <= n - 1) { R = cadd(R, cscale(tR[k + 1], t)); K = cadd(K, cscale(tK[k + 1], t)); }
}

// Katanin substitution S -> S + G dSigma G: the contour product with
// dSigma = [[0, dS^A], [dS^R, dS^K]] in the [[K, R], [A, 0]] layout of G
__device__ inline void add_katanin(const Model& m, double v, double2 GR, double2 GA, double2 GK, double2 P[2][2]) {
    double2 dR = make_double2(0, 0), dK = make_double2(0, 0);
    double t;
    int k = xstencil(v, m.n_dsig, m.A_dsig, t);
    if (k >= 0) { dR = cadd(dR, cscale(m.dsigR[k], 1.0 - t)); dK = cadd(dK, cscale(m.dsigK[k], 1.0 - t)); }
    if (k >= -1 && k + 1 <= m.n_dsig - 1) {
        dR = cadd(dR, cscale(m.dsigR[k + 1], t));
        dK = cadd(dK, cscale(m.dsigK[k + 1], t));
    }
    const double2 dA = cconj(dR);
    P[0][1] = cadd(P[0][1], cmul(cmul(GR, dR), GR));
    P[1][0] = cadd(P[1][0], cmul(cmul(GA, dA), GA));
    P[0][0] = cadd(P[0][0], cadd(cadd(cmul(cmul(GR, dR), GK), cmul(cmul(GK, dA), GA)), cmul(cmul(GR, dK), GA)));
}

// 2x2 Keldysh matrix of G (which = 0) or of the single-scale propagator S = dG/dΛ at fixed
// Σ of the flow scheme m.reg (which = 1) at frequency v; index [a][a'], 0 = classical,
// 1 = quantum: [[K, R], [A, 0]].  The interaction flow divides the bare inverse propagator
// by λ = m.lam: G^R = 1 / ((v - eps + iΔ) / λ - Σ^R), G^K = G^R [Σ^K - 2iΔ th / λ] G^A.
// With line tables (m.n_gt, m.n_st > 0) G and S are read from them instead (G^A = (G^R)*).
__device__ inline void prop2x2(const Model& m, int which, double v, double2 P[2][2]) {
    if (m.n_gt > 0 && (which == 0 || m.n_st > 0)) {
        double2 GR, GK;
        line_table(m.gtR, m.gtK, m.n_gt, m.A_gt, v, GR, GK);
        const double2 GA = cconj(GR);
        if (which == 0) {
            P[0][0] = GK;
            P[0][1] = GR;
            P[1][0] = GA;
        } else {
            double2 SR, SK;
            line_table(m.stR, m.stK, m.n_st, m.A_st, v, SR, SK);
            P[0][0] = SK;
            P[0][1] = SR;
            P[1][0] = cconj(SR);
            if (m.n_dsig > 0) add_katanin(m, v, GR, GA, GK, P);
        }
        P[1][1] = make_double2(0, 0);
        return;
    }
    double2 sR = make_double2(0, 0), sK = make_double2(0, 0);
    if (m.n_sig > 0) {
        double t;
        int k = xstencil(v, m.n_sig, m.A_sig, t);
        if (k >= 0) { sR = cadd(sR, cscale(m.sigR[k], 1.0 - t)); sK = cadd(sK, cscale(m.sigK[k], 1.0 - t)); }
        if (k >= -1 && k + 1 <= m.n_sig - 1) {
            sR = cadd(sR, cscale(m.sigR[k + 1], t));
            sK = cadd(sK, cscale(m.sigK[k + 1], t));
        }
    }
    const double lam = (m.reg == KB_REG_U) ? m.lam : 1.0;
    const double ilam = (m.reg == KB_REG_U) ? 1.0 / m.lam : 1.0;
    const double2 g0 = make_double2(v - m.eps, m.Delta);          // v - eps + i Delta
    double2 GR = cinv(make_double2(g0.x * ilam - sR.x, g0.y * ilam - sR.y));
    double2 GA = cconj(GR);
    double th = tanh_T(v, m.T);
    double2 mid = make_double2(sK.x, sK.y - 2.0 * m.Delta * th * ilam);
    if (which == 0) {
        P[0][0] = cmul(cmul(GR, mid), GA);
        P[0][1] = GR;
        P[1][0] = GA;
    } else if (m.n_st > 0) {
        // tabulated S with the model's G
        double2 SR, SK;
        line_table(m.stR, m.stK, m.n_st, m.A_st, v, SR, SK);
        P[0][0] = SK;
        P[0][1] = SR;
        P[1][0] = cconj(SR);
        if (m.n_dsig > 0) add_katanin(m, v, GR, GA, cmul(cmul(GR, mid), GA), P);
    } else {
        // S^R = -(G^R)^2 d[(G^R)^-1]/dΛ and dmid = d(mid)/dΛ per scheme
        double2 SR, dmid;
        if (m.reg == KB_REG_NONE) {
            SR = make_double2(0.0, 0.0);
            dmid = make_double2(0.0, 0.0);
        } else if (m.reg == KB_REG_U) {
            SR = cscale(cmul(cmul(GR, GR), g0), 1.0 / (lam * lam));
            dmid = make_double2(0.0, 2.0 * m.Delta * th / (lam * lam));
        } else if (m.reg == KB_REG_T) {
            const double c = cosh(v / (2.0 * m.T));
            const double dth = -v / (2.0 * m.T * m.T) / (c * c);      // d tanh(v/2T) / dT
            SR = make_double2(0.0, 0.0);
            dmid = make_double2(0.0, -2.0 * m.Delta * dth);
        } else {
            SR = cmul(make_double2(0.0, -1.0), cmul(GR, GR));
            dmid = make_double2(0.0, -2.0 * th);
        }
        double2 SA = cconj(SR);
        double2 t1 = cmul(cmul(SR, mid), GA);
        double2 t2 = cmul(cmul(GR, dmid), GA);
        double2 t3 = cmul(cmul(GR, mid), SA);
        P[0][0] = cadd(cadd(t1, t2), t3);
        P[0][1] = SR;
        P[1][0] = SA;
        if (m.n_dsig > 0) add_katanin(m, v, GR, GA, cmul(cmul(GR, mid), GA), P);
    }
    P[1][1] = make_double2(0, 0);
}

// Pi table entry (all 16 [B][D]) for node j at bosonic w, scaled by
// c_r * w_j * J_j / (2 pi i); at x_j = +-1 the limit of J * P(arg3) * P(arg4) is used:
// J / v''^2 -> pi / (2A), v'' * G -> λ [[0, 1], [1, 0]] times the sign of v'' in the
// argument (λ = 1 but in the interaction flow), v'' * S -> [[0, 1], [1, 0]] in the
// interaction flow (S^R -> 1/v) and 0 otherwise (Sec. II.G.6 tail reading).
// vnode: the node frequency v''_j = A tan(pi x_j / 2) when the caller has it (have_v), so
// that the tangent is not evaluated again.
// Channel R at compile time: the Keldysh indices (b3, b3', b4, b4') of the two lines map to
// the rows B and columns D of the table as in channel_maps (kb_api.cu), and with every
// index fixed at compile time the 2x2 propagator matrices stay in registers.
template <int R>
__device__ __forceinline__ void pi_entry_t(const Model& m, int pi_kind, double A, double w, double xj, double wj,
                                           double2 out[16], double vnode = 0.0, bool have_v = false) {
    constexpr double cr = (R == KB_CH_T) ? -1.0 : 1.0;
    double2 P3[2][2], P4[2][2], S3[2][2], S4[2][2];
    double scale;
    if (xj <= -1.0 || xj >= 1.0) {
        constexpr double s3 = 1.0, s4 = (R == KB_CH_P) ? -1.0 : 1.0;
        const double gl = (m.reg == KB_REG_U) ? m.lam : 1.0, sl = (m.reg == KB_REG_U) ? 1.0 : 0.0;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const double g = (a != b) ? 1.0 : 0.0;
                P3[a][b] = make_double2(g * gl * s3, 0);
                P4[a][b] = make_double2(g * gl * s4, 0);
                S3[a][b] = make_double2(g * sl * s3, 0);
                S4[a][b] = make_double2(g * sl * s4, 0);
            }
        scale = KB_PI / (2.0 * A);
    } else {
        const double tn = have_v ? vnode / A : tan(0.5 * KB_PI * xj);
        const double vpp = have_v ? vnode : A * tn;
        double a3, a4;
        if (R == KB_CH_P) { a3 = 0.5 * w + vpp; a4 = 0.5 * w - vpp; }
        else { a3 = vpp + 0.5 * w; a4 = vpp - 0.5 * w; }
        prop2x2(m, 0, a3, P3);
        prop2x2(m, 0, a4, P4);
        if (pi_kind == KB_PI_GS_SG) { prop2x2(m, 1, a3, S3); prop2x2(m, 1, a4, S4); }
        else {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) S3[a][b] = S4[a][b] = make_double2(0, 0);
        }
        scale = 0.5 * A * KB_PI * (1.0 + tn * tn);
    }
    // c_r * w_j * scale / (2 pi i) = -i * (c_r w_j scale / 2 pi)
    const double f = cr * wj * scale * (0.5 / KB_PI);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int b3 = q >> 3, b3p = (q >> 2) & 1, b4 = (q >> 1) & 1, b4p = q & 1;
        const int B = (R == KB_CH_A) ? 2 * b4p + b3 : (R == KB_CH_P ? 2 * b3 + b4 : 2 * b3p + b4);
        const int D = (R == KB_CH_A) ? 2 * b3p + b4 : (R == KB_CH_P ? 2 * b3p + b4p : 2 * b4p + b3);
        double2 v;
        // G^{2|2} = S^{2|2} = 0: a line with both indices quantum makes the entry vanish
        if ((b3 == 1 && b3p == 1) || (b4 == 1 && b4p == 1))
            v = make_double2(0.0, 0.0);
        else if (pi_kind == KB_PI_GS_SG)
            v = cadd(cmul(P3[b3][b3p], S4[b4][b4p]), cmul(S3[b3][b3p], P4[b4][b4p]));
        else
            v = cmul(P3[b3][b3p], P4[b4][b4p]);
        out[4 * B + D] = make_double2(f * v.y, -f * v.x);   // times -i f
    }
}

// The same for a channel known only at run time.
__device__ inline void pi_entry(const Model& m, const ChannelMaps& M, int r, int pi_kind, double A, double w,
                                double xj, double wj, double2 out[16], double vnode = 0.0, bool have_v = false) {
    (void)M;
    if (r == KB_CH_A) pi_entry_t<KB_CH_A>(m, pi_kind, A, w, xj, wj, out, vnode, have_v);
    else if (r == KB_CH_P) pi_entry_t<KB_CH_P>(m, pi_kind, A, w, xj, wj, out, vnode, have_v);
    else pi_entry_t<KB_CH_T>(m, pi_kind, A, w, xj, wj, out, vnode, have_v);
}

}  // namespace kb
