// Point evaluation of a stored vertex: the full vertex of a slot — the bare part and the
// asymptotic classes of its channels, each read at the point converted to its own channel
// variables (Sec. II.C.1) and interpolated linearly in x (Sec. II.G.7) — at arbitrary
// frequencies given in the variables of one channel.  The paper's post-processing reads
// such slices of the full vertex, e.g. the t-channel plane (w_t = 0, v_t, v'_t).
//
// The self-energy loop (Sec. II.D.2) closes the vertex with one propagator line:
//   Sigma^{a1'|a1}(v) = - int dv'/(2 pi i) sum Gamma_s^{a1' a2'|a1 a2}(v, v'|v, v') P^{a2|a2'}(v'),
//   Gamma_s = Gamma_ud + Gamma_uu, the vertex in t-channel variables (0, v, v'), P = G, the
//   single-scale propagator S of the flow scheme (the self-energy flow's loop(Gamma, S)) or
//   the line G dSigma G with one insertion of the dSigma tables (its multiloop t term),
// the sign of the Schwinger-Dyson equation's bare term (Sec. III.B), the v' integral the
// symmetric principal value at +-inf.  On the composite GL5 rule in x = (2/pi) atan(v'/A):
// the v'-independent part C(v) (R + K1_t + K2_t of both spin components) multiplies
// I_G = int dv' [G - M v'/(v'^2 + A^2)] (M = lim v' G; the subtracted term is odd), the rest
// D vanishes at x = +-1.  At x = +-1 the rule takes the limits: J [G - ...] -> (pi/2A) N_+-
// with N_+- = lim v'(v' G - M), and J D G -> +-M D_+-, D_+- the classes that decay through one
// argument ~ +-v', read at their edge node, times (n + 1)/2.
#include <cstdio>
#include <string>

#include "kb_fp64.cuh"

namespace kb {
namespace {

__global__ void k_vertex_eval(VertexDev V, Grids G, int r, int uu, int n, const double* __restrict__ f,
                              double2* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double w = f[3 * i], v = f[3 * i + 1], vp = f[3 * i + 2];
    double2 a[16], b[16];
    vertex_part_f64(V, G, r, uu != 0, false, false, w, v, vp, a);     // R + K1_r + K2'_r
    vertex_part_f64(V, G, r, uu != 0, false, true, w, v, vp, b);      // K2_r + K3_r + other channels
#pragma unroll
    for (int o = 0; o < 16; ++o) out[(size_t)16 * i + o] = make_double2(a[o].x + b[o].x, a[o].y + b[o].y);
}

// f * (class k of channel c at its edge node along `axis` (0 = w, 2 = v'), side > 0 the last
// node, interpolated in the other arguments) * (n_axis + 1)/2, into acc (components with
// a1 <-> a2 exchanged when swap12)
__device__ void acc_class_edge(const VertexDev& V, const Grids& G, int c, int k, int axis, int side, double w,
                               double v, double f, bool swap12, double2 acc[16]) {
    // the loop needs K1 along w and K2', K3 along v' only
    if (!((k == 0 && axis == 0) || ((k == 2 || k == 3) && axis == 2))) return;
    const void* D = V.cls[c][k];
    if (!D) return;
    const int dt = V.dt[c][k];
    int nw, nv;
    if (k == 0) { nw = G.n1; nv = 1; }
    else if (k < 3) { nw = G.n2w; nv = G.n2v; }
    else { nw = G.n3w; nv = G.n3v; }
    // the free arguments: w (axis 2) and, for K3, v
    int kw = 0, kv = 0;
    double tw = 0.0, tv = 0.0;
    if (axis != 0) { kw = xstencil(w, nw, G.A, tw); if (kw == -2) return; }
    if (k == 3) { kv = xstencil(v, nv, G.A, tv); if (kv == -2) return; }
    const int n_ax = (axis == 0) ? nw : nv;
    const int i_ax = side > 0 ? n_ax - 1 : 0;
    const double g0 = f * 0.5 * (n_ax + 1);
    const int nb_w = (axis == 0) ? 1 : 2, nb_v = (k == 3) ? 2 : 1;
    for (int a = 0; a < nb_w; ++a) {
        int iw = (axis == 0) ? i_ax : kw + a;
        if (iw < 0 || iw > nw - 1) continue;
        double fw = (axis == 0) ? 1.0 : (a ? tw : 1.0 - tw);
        for (int b = 0; b < nb_v; ++b) {
            int iv = (k == 3) ? kv + b : 0;
            if (k == 3 && (iv < 0 || iv > nv - 1)) continue;
            double fv = (k == 3) ? (b ? tv : 1.0 - tv) : 1.0;
            size_t base;
            if (k == 0) base = (size_t)iw * 16;
            else if (k == 2) base = ((size_t)iw * nv + i_ax) * 16;               // K2'(w, v')
            else base = (((size_t)iw * nv + iv) * nv + i_ax) * 16;               // K3(w, v, v')
            const double g = g0 * fw * fv;
#pragma unroll
            for (int o = 0; o < 16; ++o) {
                int src = swap12 ? ((o & 12) | ((o & 1) << 1) | ((o >> 1) & 1)) : o;
                double2 val = ld_c(D, dt, base + src);
                acc[o].x = fma(g, val.x, acc[o].x);
                acc[o].y = fma(g, val.y, acc[o].y);
            }
        }
    }
}

// D_+- of Gamma_s = 2 Gamma_ud(v, v'|v, v') - Gamma_ud(v, v'|v', v) at v' -> side * inf (of
// Gamma_ud alone when UD_ONLY); each channel's exchanged term comes from its crossing
// partner's data (a <-> t, p -> p).  Direct legs: t (0, v, v'), a (v - v', ...), p (v + v', ...);
// exchanged legs: t (v' - v, ...), a (0, v, v'), p (v + v', ...).
template <bool UD_ONLY>
__device__ void loop_edge(const VertexDev& V, const Grids& G, double nu, int side, double2 E[16]) {
    constexpr double fd = UD_ONLY ? 1.0 : 2.0;
#pragma unroll
    for (int o = 0; o < 16; ++o) E[o] = make_double2(0.0, 0.0);
    if ((V.mask >> KB_CH_T) & 1) {
        acc_class_edge(V, G, KB_CH_T, 2, 2, side, 0.0, nu, fd, false, E);     // K2'_t(0, v')
        acc_class_edge(V, G, KB_CH_T, 3, 2, side, 0.0, nu, fd, false, E);     // K3_t(0, v, v')
        if (!UD_ONLY) {
            acc_class_edge(V, G, KB_CH_A, 2, 2, side, 0.0, nu, -1.0, true, E);    // K2'_a(0, v'), exchanged
            acc_class_edge(V, G, KB_CH_A, 3, 2, side, 0.0, nu, -1.0, true, E);    // K3_a(0, v, v'), exchanged
        }
    }
    if ((V.mask >> KB_CH_A) & 1) {
        acc_class_edge(V, G, KB_CH_A, 0, 0, -side, 0.0, 0.0, fd, false, E);   // K1_a(v - v')
        if (!UD_ONLY) acc_class_edge(V, G, KB_CH_T, 0, 0, side, 0.0, 0.0, -1.0, true, E);   // K1_t(v' - v), exchanged
    }
    if ((V.mask >> KB_CH_P) & 1) {
        acc_class_edge(V, G, KB_CH_P, 0, 0, side, 0.0, 0.0, fd, false, E);    // K1_p(v + v')
        if (!UD_ONLY) acc_class_edge(V, G, KB_CH_P, 0, 0, side, 0.0, 0.0, -1.0, true, E);   // K1_p(v + v'), exchanged
    }
}

// S[a1'][a1] += f sum_{a2, a2'} Gam[a1' a2'|a1 a2] P[a2][a2']
__device__ __forceinline__ void loop_contract(const double2 Gam[16], const double2 P[2][2], double f, double2 S[4]) {
#pragma unroll
    for (int a1p = 0; a1p < 2; ++a1p)
#pragma unroll
        for (int a1 = 0; a1 < 2; ++a1) {
            double2 s = make_double2(0.0, 0.0);
#pragma unroll
            for (int a2p = 0; a2p < 2; ++a2p)
#pragma unroll
                for (int a2 = 0; a2 < 2; ++a2) cfma(s, Gam[8 * a1p + 4 * a2p + 2 * a1 + a2], P[a2][a2p]);
            S[2 * a1p + a1].x = fma(f, s.x, S[2 * a1p + a1].x);
            S[2 * a1p + a1].y = fma(f, s.y, S[2 * a1p + a1].y);
        }
}

constexpr int LOOP_THREADS = 256;

// Asymptotics of the line P (which 0: G, 1: S of the flow scheme) with Sigma tables vanishing
// at x = +-1: M = lim v' P = mm [[0, 1], [1, 0]] and N_+- = lim v'(v' P - M) with
// N^R = nR, N^A = nR*, N^K_+- = -+ i nK (N^{qq} = 0):
//   G: mm = lam, nR = lam (eps - i Delta), nK = 2 lam Delta;
//   S, hybridisation flow (S^R = -i G^R G^R): mm = 0, nR = -i, nK = 2;
//   S, interaction flow (S = G / lam at this order): mm = 1, nR = eps - i Delta, nK = 2 Delta;
//   S, temperature flow: all zero (S^R = 0, S^K falls exponentially); no-flow scheme: S = 0.
// The Katanin term G dSigma G falls like 1/v'^3 and adds nothing.
// The line with one insertion of the dSigma tables, G dSigma G (which 2), falls like 1/v'^3:
// all zero.
struct LineTail {
    double mm, nK;
    double2 nR;
};
__device__ __forceinline__ LineTail line_tail(const Model& m, int which) {
    const double lam = (m.reg == KB_REG_U) ? m.lam : 1.0;
    if (which == 2) return {0.0, 0.0, make_double2(0.0, 0.0)};
    if (which == 0) return {lam, 2.0 * lam * m.Delta, make_double2(lam * m.eps, -lam * m.Delta)};
    if (m.reg == KB_REG_U) return {1.0, 2.0 * m.Delta, make_double2(m.eps, -m.Delta)};
    if (m.reg == KB_REG_T || m.reg == KB_REG_NONE) return {0.0, 0.0, make_double2(0.0, 0.0)};
    return {0.0, 2.0, make_double2(0.0, -1.0)};
}

// G dSigma G at v: the contour product with dSigma = [[0, dS^A], [dS^R, dS^K]] (the dSigma
// tables, linear in x, zero at x = +-1) in the [[K, R], [A, 0]] layout of G; zero without tables.
__device__ void line_with_insertion(const Model& m, double v, double2 P[2][2]) {
    double2 Gm[2][2];
    prop2x2(m, 0, v, Gm);
    double2 dR = make_double2(0, 0), dK = make_double2(0, 0);
    if (m.n_dsig > 0) {
        double t;
        int k = xstencil(v, m.n_dsig, m.A_dsig, t);
        if (k >= 0) { dR = cadd(dR, cscale(m.dsigR[k], 1.0 - t)); dK = cadd(dK, cscale(m.dsigK[k], 1.0 - t)); }
        if (k >= -1 && k + 1 <= m.n_dsig - 1) {
            dR = cadd(dR, cscale(m.dsigR[k + 1], t));
            dK = cadd(dK, cscale(m.dsigK[k + 1], t));
        }
    }
    const double2 GR = Gm[0][1], GA = Gm[1][0], GK = Gm[0][0], dA = cconj(dR);
    P[0][1] = cmul(cmul(GR, dR), GR);
    P[1][0] = cmul(cmul(GA, dA), GA);
    P[0][0] = cadd(cadd(cmul(cmul(GR, dR), GK), cmul(cmul(GK, dA), GA)), cmul(cmul(GR, dK), GA));
    P[1][1] = make_double2(0, 0);
}

// One block per output frequency; threads stride over the interior nodes 1 .. nq-2.  UD_ONLY:
// the up-down vertex alone (the closed line carries the spin opposite to the external one, as
// in the Schwinger-Dyson equation's bubble forms).
template <bool UD_ONLY>
__global__ void __launch_bounds__(LOOP_THREADS) k_loop(VertexDev V, Grids G, Model m, int which, int n,
                                                       const double* __restrict__ nus,
                                                       const double* __restrict__ xq,
                                                       const double* __restrict__ wq, double2* __restrict__ out) {
    const int i = blockIdx.x;
    if (i >= n) return;
    const double nu = nus[i], A = G.A;
    const int nq = G.nq;
    const LineTail tl = line_tail(m, which);
    double2 acc[8];                       // [0..3] int D G over [a1'][a1], [4..7] I_G over [a2][a2']
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int j = 1 + threadIdx.x; j < nq - 1; j += LOOP_THREADS) {
        const double tn = tan(0.5 * KB_PI * xq[j]);
        const double nup = A * tn, f = wq[j] * (0.5 * A * KB_PI * (1.0 + tn * tn));
        double2 P[2][2];
        if (which == 2) line_with_insertion(m, nup, P);
        else prop2x2(m, which, nup, P);
        P[1][1] = make_double2(0.0, 0.0);
        const double sub = tl.mm * nup / (nup * nup + A * A);
        acc[4].x = fma(f, P[0][0].x, acc[4].x);         acc[4].y = fma(f, P[0][0].y, acc[4].y);
        acc[5].x = fma(f, P[0][1].x - sub, acc[5].x);   acc[5].y = fma(f, P[0][1].y, acc[5].y);
        acc[6].x = fma(f, P[1][0].x - sub, acc[6].x);   acc[6].y = fma(f, P[1][0].y, acc[6].y);
        double2 Dv[16];
        vertex_part_f64(V, G, KB_CH_T, false, true, true, 0.0, nu, nup, Dv);    // up-down
        loop_contract(Dv, P, f, acc);
        if (!UD_ONLY) {
            vertex_part_f64(V, G, KB_CH_T, true, true, true, 0.0, nu, nup, Dv);     // up-up
            loop_contract(Dv, P, f, acc);
        }
    }
    // block reduction: warp shuffles, then one slot per warp in shared memory
    __shared__ double2 red[LOOP_THREADS / 32][8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
        for (int d = 16; d > 0; d >>= 1) {
            acc[q].x += __shfl_down_sync(0xffffffffu, acc[q].x, d);
            acc[q].y += __shfl_down_sync(0xffffffffu, acc[q].y, d);
        }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 8; ++q) red[warp][q] = acc[q];
    __syncthreads();
    if (threadIdx.x != 0) return;
    double2 S[4], IG[2][2];
    for (int q = 0; q < 4; ++q) {
        S[q] = make_double2(0.0, 0.0);
        double2 t = make_double2(0.0, 0.0);
        for (int k = 0; k < LOOP_THREADS / 32; ++k) { S[q] = cadd(S[q], red[k][q]); t = cadd(t, red[k][4 + q]); }
        IG[q >> 1][q & 1] = t;
    }
    // the rule's end nodes of I_P: (pi/2A) N_-+ (x = -1 with weight wq[0], x = +1 with wq[nq-1])
    const double c0 = wq[0] * KB_PI / (2.0 * A), c1 = wq[nq - 1] * KB_PI / (2.0 * A);
    IG[0][0].y += (c0 - c1) * tl.nK;
    IG[0][1] = cadd(IG[0][1], cscale(tl.nR, c0 + c1));
    IG[1][0] = cadd(IG[1][0], cscale(cconj(tl.nR), c0 + c1));
    double2 Cv[16];
    vertex_part_f64(V, G, KB_CH_T, false, true, false, 0.0, nu, 0.0, Cv);
    loop_contract(Cv, IG, 1.0, S);
    if (!UD_ONLY) {
        vertex_part_f64(V, G, KB_CH_T, true, true, false, 0.0, nu, 0.0, Cv);
        loop_contract(Cv, IG, 1.0, S);
    }
    // end nodes of int D P: +-M D_+-
    double2 Mm[2][2] = {{make_double2(0.0, 0.0), make_double2(tl.mm, 0.0)},
                        {make_double2(tl.mm, 0.0), make_double2(0.0, 0.0)}};
    double2 E[16];
    loop_edge<UD_ONLY>(V, G, nu, +1, E);
    loop_contract(E, Mm, wq[nq - 1], S);
    loop_edge<UD_ONLY>(V, G, nu, -1, E);
    loop_contract(E, Mm, -wq[0], S);
    // Sigma = -S / (2 pi i) = i S / (2 pi)
    const double s = 1.0 / (2.0 * KB_PI);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[(size_t)4 * i + q] = make_double2(-S[q].y * s, S[q].x * s);
}

}  // namespace
}  // namespace kb

using namespace kb;

extern "C" kb_status kb_vertex_eval(kb_ctx* ctx, int slot, int channel, int spin_uu, int n, const double* freqs,
                                    void* out, void* stream) {
    if (!ctx) return KB_ERR_ARG;
    if (slot < 0 || slot >= KB_MAX_SLOTS || channel < 0 || channel > 2 || n < 0 || (n > 0 && (!freqs || !out))) {
        ctx->err = "kb_vertex_eval: bad slot, channel, count or pointer";
        return KB_ERR_ARG;
    }
    if (!ctx->grids_set || !ctx->slot_set[slot]) {
        ctx->err = "kb_vertex_eval: set the grids and the vertex first";
        return KB_ERR_STATE;
    }
    if (n == 0) return KB_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return KB_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    {
        KB_LAUNCH(ctx, st, "k_vertex_eval");
        k_vertex_eval<<<(n + 127) / 128, 128, 0, st>>>(ctx->slots[slot], ctx->g, channel, spin_uu, n, freqs,
                                                       static_cast<double2*>(out));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("kb_vertex_eval: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}

extern "C" kb_status kb_loop(kb_ctx* ctx, int slot, int which, int n, const double* nus, void* out,
                             void* stream) {
    if (!ctx) return KB_ERR_ARG;
    const int line = which & 3;
    const bool ud_only = (which & KB_LOOP_UD_ONLY) != 0;
    if (slot < 0 || slot >= KB_MAX_SLOTS || which < 0 || (which & ~(3 | KB_LOOP_UD_ONLY)) || line > 2 || n < 0 ||
        (n > 0 && (!nus || !out))) {
        ctx->err = "kb_loop: bad slot, line, count or pointer";
        return KB_ERR_ARG;
    }
    if (!ctx->grids_set || !ctx->model_set || !ctx->slot_set[slot]) {
        ctx->err = "kb_loop: set the grids, the model and the vertex first";
        return KB_ERR_STATE;
    }
    if (line == 1 && ctx->m.n_gt > 0 && ctx->m.n_st == 0) {
        ctx->err = "kb_loop: G is tabulated, so the S line needs an S table";
        return KB_ERR_STATE;
    }
    if (n == 0) return KB_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return KB_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    {
        KB_LAUNCH(ctx, st, "k_loop");
        if (ud_only)
            k_loop<true><<<n, LOOP_THREADS, 0, st>>>(ctx->slots[slot], ctx->g, ctx->m, line, n, nus, ctx->d_xq,
                                                     ctx->d_wq, static_cast<double2*>(out));
        else
            k_loop<false><<<n, LOOP_THREADS, 0, st>>>(ctx->slots[slot], ctx->g, ctx->m, line, n, nus, ctx->d_xq,
                                                      ctx->d_wq, static_cast<double2*>(out));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("kb_loop: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}
