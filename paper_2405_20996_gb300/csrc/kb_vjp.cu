// Adjoint (vector-jacobian product) of the plain FP64 bubble.
//
// Convention: gradients of a real loss L on the real embedding, bar(z) = dL/dRe z +
// i dL/dIm z.  Per output class and chunk of bosonic frequencies the forward is
//   B[w] = L[w] R'[w]^T,  L = left tile, R' = Pi-folded right tile (kb_fp64.cu),
// so with Gbar[w][(v, A)][(v', C)] = alpha * bar(out)[..][c(A, C)]:
//   bar(L)[m][k]  = sum_n Gbar[m][n] conj(R'[n][k])             (k_zgemm_gen)
//   bar(R')[n][k] = sum_m conj(L[m][k]) Gbar[m][n]              (k_zgemm_gen)
//   bar(R)[D][C]  = sum_B conj(Pi[B][D]) bar(R')[C][B]           (k_vjp_right)
//   bar(Pi)[B][D] = sum_{v', C, s} conj(R[D][C]) bar(R')[C][B]   (k_vjp_right)
// and the tile gradients are scattered through the transpose of the interpolation, the
// class split, the channel conversion and the up-up exchange into the gradient slots
// (atomic FP64 adds).  The Pi gradient is pulled back to G^R at the two sample frequencies
// of every (w, node), with G^A = (G^R)* and G^K = tanh(v/2T)(G^R - G^A) (FDR, Sec. II.C.4).
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "kb_fp64.cuh"

namespace kb {
namespace {

__device__ __forceinline__ void atomic_cadd(double2* p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

// Transpose of acc_class_f64: grad(c, k)[corner][src(o)] += f * weight * bar[o].
__device__ void acc_class_adj_f64(const VertexDev& Gd, const Grids& G, int c, int k, double w, double v, double vp,
                                  double f, bool swap12, const double2 bar[16]) {
    double2* D = const_cast<double2*>(reinterpret_cast<const double2*>(Gd.cls[c][k]));
    if (!D) return;
    int nw, nv;
    if (k == 0) { nw = G.n1; nv = 1; }
    else if (k < 3) { nw = G.n2w; nv = G.n2v; }
    else { nw = G.n3w; nv = G.n3v; }
    double tw, tv = 0, tp = 0;
    int kw = xstencil(w, nw, G.A, tw);
    if (kw == -2) return;
    int kv = 0, kp = 0;
    if (k == 1 || k == 3) { kv = xstencil(v, nv, G.A, tv); if (kv == -2) return; }
    if (k == 2) { kv = xstencil(vp, nv, G.A, tv); if (kv == -2) return; }
    if (k == 3) { kp = xstencil(vp, nv, G.A, tp); if (kp == -2) return; }
    int nb_v = (k == 0) ? 1 : 2, nb_p = (k == 3) ? 2 : 1;
    for (int a = 0; a < 2; ++a) {
        int iw = kw + a;
        if (iw < 0 || iw > nw - 1) continue;
        double fw = a ? tw : 1.0 - tw;
        for (int b = 0; b < nb_v; ++b) {
            int iv = kv + b;
            double fv = 1.0;
            if (k != 0) { if (iv < 0 || iv > nv - 1) continue; fv = b ? tv : 1.0 - tv; }
            for (int e = 0; e < nb_p; ++e) {
                int ip = kp + e;
                double fp = 1.0;
                if (k == 3) { if (ip < 0 || ip > nv - 1) continue; fp = e ? tp : 1.0 - tp; }
                size_t base;
                if (k == 0) base = (size_t)iw * 16;
                else if (k < 3) base = ((size_t)iw * nv + iv) * 16;
                else base = (((size_t)iw * nv + iv) * nv + ip) * 16;
                double g = f * fw * fv * fp;
                if (g == 0.0) continue;
#pragma unroll
                for (int o = 0; o < 16; ++o) {
                    int src = swap12 ? ((o & 12) | ((o & 1) << 1) | ((o >> 1) & 1)) : o;
                    atomic_cadd(D + base + src, cscale(bar[o], g));
                }
            }
        }
    }
}

// Transpose of vertex_part_f64 (the bare part is a fixed parameter: no gradient).
__device__ void vertex_part_adj_f64(const VertexDev& V, const VertexDev& Gd, const Grids& G, int r, bool uu,
                                    bool right, bool nupart, double w, double v, double vp, const double2 bar[16]) {
    int k_free = right ? 1 : 2, k_dep = right ? 2 : 1;
    int ka = nupart ? k_dep : 0, kb2 = nupart ? 3 : k_free;
    if ((V.mask >> r) & 1) {
        int sr = (r == KB_CH_A) ? KB_CH_T : (r == KB_CH_T ? KB_CH_A : KB_CH_P);
        double xw = (r == KB_CH_P) ? w : -w, xvp = (r == KB_CH_P) ? -vp : vp;
        for (int q = 0; q < 2; ++q) {
            int k = q ? kb2 : ka;
            acc_class_adj_f64(Gd, G, r, k, w, v, vp, 1.0, false, bar);
            if (uu) acc_class_adj_f64(Gd, G, sr, k, xw, v, xvp, -1.0, true, bar);
        }
    }
    if (nupart) {
        double L[4];
        legs_of(r, w, v, vp, L);
        double S[4] = {L[0], L[1], L[3], L[2]};
        for (int c = 0; c < 3; ++c) {
            if (c == r || !((V.mask >> c) & 1)) continue;
            double wc, vc, pc;
            vars_of(c, L, wc, vc, pc);
            for (int k = 0; k < 4; ++k) acc_class_adj_f64(Gd, G, c, k, wc, vc, pc, 1.0, false, bar);
            if (uu) {
                int sc = (c == KB_CH_A) ? KB_CH_T : (c == KB_CH_T ? KB_CH_A : KB_CH_P);
                vars_of(sc, S, wc, vc, pc);
                for (int k = 0; k < 4; ++k) acc_class_adj_f64(Gd, G, sc, k, wc, vc, pc, -1.0, true, bar);
            }
        }
    }
}

// Gbar[wl][(vL, A)][(vR, C)] = alpha * bar(out)[class element][cO[A][C]]
__global__ void k_vjp_gbar(ClassJob J, int cls, const void* gout, int dt, double alpha, double2* __restrict__ Gb) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)J.nw_chunk * J.nL * J.nR * 16;
    if (idx >= total) return;
    int o = idx % 16;
    size_t rest = idx / 16;
    int vR = rest % J.nR;
    rest /= J.nR;
    int vL = rest % J.nL;
    int wl = rest / J.nL;
    const ChannelMaps& M = c_maps[J.r];
    int A = 0, C = 0;
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 4; ++c)
            if (M.cO[a][c] == o) { A = a; C = c; }
    size_t w = J.w0 + wl, e;
    if (cls == KB_K1) e = w * 16 + o;
    else if (cls == KB_K2) e = (w * J.nL + vL) * 16 + o;
    else if (cls == KB_K2P) e = (w * J.nR + vR) * 16 + o;
    else e = ((w * J.nL + vL) * J.nR + vR) * 16 + o;
    double2 g = ld_c(gout, dt, e);
    int Mrows = 4 * J.nL, Ncols = 4 * J.nR;
    Gb[((size_t)wl * Mrows + 4 * vL + A) * Ncols + 4 * vR + C] = cscale(g, alpha);
}

// Batched strided complex GEMM: C[b][i][j] = sum_l opA(A[b][i][l]) opB(B[b][l][j]), op =
// identity or complex conjugate, every operand addressed by element strides.  32x32 output
// tile, 256 threads with 2x2 outputs each, l in chunks of 16 through shared memory.
struct GemmDesc {
    int I, J, L;
    long long sAb, sAi, sAl, sBb, sBl, sBj, sCb, sCi;
    bool conjA, conjB;
};

__global__ void __launch_bounds__(256) k_zgemm_gen(const double2* __restrict__ A, const double2* __restrict__ B,
                                                   double2* __restrict__ C, GemmDesc d) {
    __shared__ double2 sA[16][33], sB[16][33];
    int b = blockIdx.z;
    int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const double2* Ab = A + b * d.sAb;
    const double2* Bb = B + b * d.sBb;
    int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double2 acc[2][2] = {};
    for (int l0 = 0; l0 < d.L; l0 += 16) {
        for (int t = threadIdx.x; t < 32 * 16; t += 256) {
            int ll = t / 32, rr = t % 32;
            int gi = i0 + rr, gj = j0 + rr, gl = l0 + ll;
            double2 a = make_double2(0, 0), bv = make_double2(0, 0);
            if (gi < d.I && gl < d.L) a = Ab[gi * d.sAi + gl * d.sAl];
            if (gj < d.J && gl < d.L) bv = Bb[gl * d.sBl + gj * d.sBj];
            sA[ll][rr] = d.conjA ? cconj(a) : a;
            sB[ll][rr] = d.conjB ? cconj(bv) : bv;
        }
        __syncthreads();
#pragma unroll
        for (int ll = 0; ll < 16; ++ll) {
            double2 a0 = sA[ll][ty], a1 = sA[ll][ty + 16];
            double2 b0 = sB[ll][tx], b1 = sB[ll][tx + 16];
            cfma(acc[0][0], a0, b0);
            cfma(acc[0][1], a0, b1);
            cfma(acc[1][0], a1, b0);
            cfma(acc[1][1], a1, b1);
        }
        __syncthreads();
    }
    for (int i = 0; i < 2; ++i)
        for (int jj = 0; jj < 2; ++jj) {
            int gi = i0 + ty + 16 * i, gj = j0 + tx + 16 * jj;
            if (gi < d.I && gj < d.J) C[b * d.sCb + gi * d.sCi + gj] = acc[i][jj];
        }
}

// One thread per (w, v, s, j) record of the left tile: bar(L) -> gradient slot.
__global__ void k_vjp_left(VertexDev V, VertexDev Gd, Grids G, ClassJob J, const double* __restrict__ xq,
                           const double2* __restrict__ gL) {
    // consecutive threads take different (v, s, w) of the same node: records that share
    // interpolation corners (adjacent nodes) sit in different warps, so the atomic adds of
    // one warp rarely collide on one address
    const size_t inner = (size_t)J.nw_chunk * J.ns * J.nL;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= inner * J.nq) return;
    const int j = (int)(idx / inner);
    size_t rest = idx % inner;
    const int vi = (int)(rest % J.nL);
    rest /= J.nL;
    const int s = (int)(rest % J.ns);
    const int wl = (int)(rest / J.ns);
    const ChannelMaps& M = c_maps[J.r];
    double w = grid_freq(J.w0 + wl, J.nw_grid, G.A);
    double vext = J.L_nu ? grid_freq(vi, J.nvL_grid, G.A) : 0.0;
    double xj = xq[j];
    double vpp = (xj <= -1.0) ? -INFINITY : (xj >= 1.0 ? INFINITY : G.A * tan(0.5 * KB_PI * xj));
    bool uu = (J.r == KB_CH_T) && (s == 0);
    size_t K = (size_t)4 * J.ns * J.nq;
    size_t kcol = ((size_t)s * J.nq + j) * 4;
    size_t rowbase = (size_t)wl * 4 * J.nL + (size_t)vi * 4;
    double2 bar[16];
    for (int A = 0; A < 4; ++A)
        for (int B = 0; B < 4; ++B) bar[M.cL[A][B]] = gL[(rowbase + A) * K + kcol + B];
    vertex_part_adj_f64(V, Gd, G, J.r, uu, false, J.L_nu, w, vext, vpp, bar);
}

// One thread per (w, v', s, j) record of the right tile: bar(R') -> bar(R) -> gradient slot,
// and (gPi != nullptr) bar(Pi)[w][j] += sum_C conj(R[D][C]) bar(R')[C][B].
// Launched twice when both are wanted: for the vertex gradient (want_vertex, gPi null) with
// consecutive threads on different (v, s, w) of one node, like k_vjp_left; for the Pi
// gradient (gPi) with consecutive threads on consecutive nodes, whose Pi entries differ.
__global__ void k_vjp_right(VertexDev V, VertexDev Gd, bool want_vertex, Grids G, ClassJob J,
                            const double* __restrict__ xq, const double2* __restrict__ Pi,
                            const double2* __restrict__ gRp, double2* __restrict__ gPi) {
    const size_t inner = (size_t)J.nw_chunk * J.ns * J.nR;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= inner * J.nq) return;
    int j, vi, s, wl;
    if (gPi) {
        j = (int)(idx % J.nq);
        size_t rest = idx / J.nq;
        vi = (int)(rest % J.nR);
        rest /= J.nR;
        s = (int)(rest % J.ns);
        wl = (int)(rest / J.ns);
    } else {
        j = (int)(idx / inner);
        size_t rest = idx % inner;
        vi = (int)(rest % J.nR);
        rest /= J.nR;
        s = (int)(rest % J.ns);
        wl = (int)(rest / J.ns);
    }
    const ChannelMaps& M = c_maps[J.r];
    double w = grid_freq(J.w0 + wl, J.nw_grid, G.A);
    double vext = J.R_nu ? grid_freq(vi, J.nvR_grid, G.A) : 0.0;
    double xj = xq[j];
    double vpp = (xj <= -1.0) ? -INFINITY : (xj >= 1.0 ? INFINITY : G.A * tan(0.5 * KB_PI * xj));
    bool uu = (J.r == KB_CH_T) && (s == 1);
    size_t K = (size_t)4 * J.ns * J.nq;
    size_t kcol = ((size_t)s * J.nq + j) * 4;
    size_t rowbase = (size_t)wl * 4 * J.nR + (size_t)vi * 4;
    double2 grp[4][4];   // [C][B]
    for (int C = 0; C < 4; ++C)
        for (int B = 0; B < 4; ++B) grp[C][B] = gRp[(rowbase + C) * K + kcol + B];
    const double2* P = Pi + ((size_t)wl * J.nq + j) * 16;
    if (want_vertex) {
        double2 bar[16];
        for (int D = 0; D < 4; ++D)
            for (int C = 0; C < 4; ++C) {
                double2 acc = make_double2(0, 0);
                for (int B = 0; B < 4; ++B) cfma(acc, cconj(P[4 * B + D]), grp[C][B]);
                bar[M.cR[D][C]] = acc;
            }
        vertex_part_adj_f64(V, Gd, G, J.r, uu, true, J.R_nu, w, vpp, vext, bar);
    }
    if (gPi) {
        double2 g[16];
        vertex_part_f64(V, G, J.r, uu, true, J.R_nu, w, vpp, vext, g);
        double2* dst = gPi + ((size_t)wl * J.nq + j) * 16;
        for (int B = 0; B < 4; ++B)
            for (int D = 0; D < 4; ++D) {
                double2 acc = make_double2(0, 0);
                for (int C = 0; C < 4; ++C) cfma(acc, cconj(g[M.cR[D][C]]), grp[C][B]);
                atomic_cadd(dst + 4 * B + D, acc);
            }
    }
}

// Pull bar(Pi) back to G^R at the two propagator arguments of every interior (w, node):
// Pi[B][D] = -i f P3[q0][q1] P4[q2][q3] with f = c_r w_j J_j / (2 pi) (see pi_entry), then
// bar(G^R) = bar(G^{1|2}) + conj(bar(G^{2|1})) + th (bar(G^{1|1}) - conj(bar(G^{1|1}))).
// gGR[w][j][side] (w on the class grid) accumulates.
__global__ void k_vjp_gr(Model m, ClassJob J, double A, const double* __restrict__ xq, const double* __restrict__ wq,
                         const double2* __restrict__ gPi, double2* __restrict__ gGR) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int wl = blockIdx.y;
    if (j >= J.nq || wl >= J.nw_chunk) return;
    double xj = xq[j];
    if (xj <= -1.0 || xj >= 1.0) return;      // the tail limit does not depend on G
    const ChannelMaps& M = c_maps[J.r];
    double w = grid_freq(J.w0 + wl, J.nw_grid, A);
    double tn = tan(0.5 * KB_PI * xj);
    double vpp = A * tn;
    double a3, a4;
    if (J.r == KB_CH_P) { a3 = 0.5 * w + vpp; a4 = 0.5 * w - vpp; }
    else { a3 = vpp + 0.5 * w; a4 = vpp - 0.5 * w; }
    double2 P3[2][2], P4[2][2];
    prop2x2(m, 0, a3, P3);
    prop2x2(m, 0, a4, P4);
    double cr = (J.r == KB_CH_T) ? -1.0 : 1.0;
    double f = cr * wq[j] * (0.5 * A * KB_PI * (1.0 + tn * tn)) / (2.0 * KB_PI);
    double2 b3[2][2] = {}, b4[2][2] = {};
    const double2* g = gPi + ((size_t)wl * J.nq + j) * 16;
    for (int B = 0; B < 4; ++B)
        for (int D = 0; D < 4; ++D) {
            const int* q = M.piq[B][D];
            double2 gb = g[4 * B + D];
            // d Pi / d P3 = -i f P4  ->  conj = i f conj(P4)
            double2 c4 = cconj(P4[q[2]][q[3]]), c3 = cconj(P3[q[0]][q[1]]);
            double2 if4 = make_double2(-f * c4.y, f * c4.x), if3 = make_double2(-f * c3.y, f * c3.x);
            cfma(b3[q[0]][q[1]], if4, gb);
            cfma(b4[q[2]][q[3]], if3, gb);
        }
    double th3 = tanh_T(a3, m.T), th4 = tanh_T(a4, m.T);
    auto pull = [](double2 bb[2][2], double th) {
        double2 r = cadd(bb[0][1], cconj(bb[1][0]));
        // th (z - conj z) = 2 i th Im z
        return cadd(r, make_double2(0.0, 2.0 * th * bb[0][0].y));
    };
    double2* dst = gGR + ((size_t)(J.w0 + wl) * J.nq + j) * 2;
    dst[0] = cadd(dst[0], pull(b3, th3));
    dst[1] = cadd(dst[1], pull(b4, th4));
}

}  // namespace
}  // namespace kb

using namespace kb;

void class_shape(const Grids& g, int cls, int& nw, int& nL, int& nR, int& nvg);

static bool g_vjp_maps_uploaded[64] = {};

kb_status kb_bubble_vjp_fp64(kb_ctx* ctx, int r, int sl, int sr, int sgo, int pi_kind, unsigned mask, double alpha,
                             int sgl, int sgr, void* const gGR[3], cudaStream_t st) {
    if (!g_vjp_maps_uploaded[ctx->device]) {
        ChannelMaps h[3] = {channel_maps(0), channel_maps(1), channel_maps(2)};
        KB_CUDA_TRY(ctx, cudaMemcpyToSymbol(c_maps, h, sizeof(h)));
        g_vjp_maps_uploaded[ctx->device] = true;
    }
    const Grids& g = ctx->g;
    int ns = (r == KB_CH_T) ? 2 : 1;
    size_t K = (size_t)4 * ns * g.nq;
    const VertexDev none{};
    const VertexDev& GL = sgl >= 0 ? ctx->slots[sgl] : none;
    const VertexDev& GR = sgr >= 0 ? ctx->slots[sgr] : none;
    for (int cls = 0; cls < 4; ++cls) {
        if (!((mask >> cls) & 1)) continue;
        double2* gtab = reinterpret_cast<double2*>(gGR ? gGR[cls == KB_K1 ? 0 : (cls == KB_K3 ? 2 : 1)] : nullptr);
        bool want_l = sgl >= 0, want_r = sgr >= 0, want_gr = gtab != nullptr;
        if (!want_l && !want_r && !want_gr) continue;
        int nw, nL, nR, nvg;
        class_shape(g, cls, nw, nL, nR, nvg);
        size_t tileL = (size_t)4 * nL * K, tileR = (size_t)4 * nR * K, nGb = (size_t)16 * nL * nR;
        size_t per_w = ((size_t)g.nq * 16 * (want_gr ? 2 : 1) + 2 * tileL + 2 * tileR + nGb) * sizeof(double2);
        int chunk = (int)std::max<size_t>(1, std::min<size_t>(nw, ctx->ws_limit / per_w));
        kb_status s = kb_ensure_workspace(ctx, per_w * chunk, st);
        if (s != KB_OK) return s;
        double2* Pi = static_cast<double2*>(ctx->ws.ptr);
        double2* Lt = Pi + (size_t)chunk * g.nq * 16;
        double2* Rt = Lt + (size_t)chunk * tileL;
        double2* gL = Rt + (size_t)chunk * tileR;
        double2* gRp = gL + (size_t)chunk * tileL;
        double2* Gb = gRp + (size_t)chunk * tileR;
        double2* gPi = want_gr ? Gb + (size_t)chunk * nGb : nullptr;
        for (int w0 = 0; w0 < nw; w0 += chunk) {
            ClassJob J;
            J.r = r; J.pi_kind = pi_kind; J.ns = ns; J.nq = g.nq;
            J.nw_chunk = std::min(chunk, nw - w0); J.w0 = w0; J.nw_grid = nw;
            J.nL = nL; J.nR = nR; J.nvL_grid = nvg; J.nvR_grid = nvg;
            J.L_nu = (cls == KB_K2 || cls == KB_K3);
            J.R_nu = (cls == KB_K2P || cls == KB_K3);
            int Mr = 4 * nL, Nc = 4 * nR;
            {
                KB_LAUNCH(ctx, st, "k_pi_table");
                k_pi_table<<<dim3((g.nq + 127) / 128, J.nw_chunk), 128, 0, st>>>(ctx->m, J, g.A, ctx->d_xq, ctx->d_wq, Pi);
            }
            {
                KB_LAUNCH(ctx, st, "k_gather_f64_left");
                k_gather_f64<false><<<dim3((g.nq + 127) / 128, nL * ns, J.nw_chunk), 128, 0, st>>>(
                    ctx->slots[sl], g, J, ctx->d_xq, Pi, Lt);
            }
            {
                KB_LAUNCH(ctx, st, "k_gather_f64_right");
                k_gather_f64<true><<<dim3((g.nq + 127) / 128, nR * ns, J.nw_chunk), 128, 0, st>>>(
                    ctx->slots[sr], g, J, ctx->d_xq, Pi, Rt);
            }
            {
                KB_LAUNCH(ctx, st, "k_vjp_gbar");
                size_t tot = (size_t)J.nw_chunk * nL * nR * 16;
                k_vjp_gbar<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(J, cls, ctx->slots[sgo].cls[r][cls],
                                                                         ctx->slots[sgo].dt[r][cls], alpha, Gb);
            }
            if (want_l) {
                GemmDesc d{Mr, (int)K, Nc, (long long)Mr * Nc, Nc, 1, (long long)tileR, (long long)K, 1,
                           (long long)tileL, (long long)K, false, true};
                {
                    KB_LAUNCH(ctx, st, "k_zgemm_gen");
                    k_zgemm_gen<<<dim3((unsigned)((K + 31) / 32), (Mr + 31) / 32, J.nw_chunk), 256, 0, st>>>(Gb, Rt, gL,
                                                                                                           d);
                }
                {
                    KB_LAUNCH(ctx, st, "k_vjp_left");
                    size_t tot = (size_t)J.nw_chunk * ns * nL * g.nq;
                    k_vjp_left<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(ctx->slots[sl], GL, g, J, ctx->d_xq, gL);
                }
            }
            if (want_r || want_gr) {
                GemmDesc d{Nc, (int)K, Mr, (long long)Mr * Nc, 1, Nc, (long long)tileL, (long long)K, 1,
                           (long long)tileR, (long long)K, false, true};
                {
                    KB_LAUNCH(ctx, st, "k_zgemm_gen");
                    k_zgemm_gen<<<dim3((unsigned)((K + 31) / 32), (Nc + 31) / 32, J.nw_chunk), 256, 0, st>>>(Gb, Lt, gRp,
                                                                                                           d);
                }
                if (want_gr)
                    KB_CUDA_TRY(ctx, cudaMemsetAsync(gPi, 0, (size_t)J.nw_chunk * g.nq * 16 * sizeof(double2), st));
                {
                    KB_LAUNCH(ctx, st, "k_vjp_right");
                    size_t tot = (size_t)J.nw_chunk * ns * nR * g.nq;
                    if (want_r)
                        k_vjp_right<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(ctx->slots[sr], GR, true, g, J,
                                                                                 ctx->d_xq, Pi, gRp, nullptr);
                    if (want_gr)
                        k_vjp_right<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(ctx->slots[sr], GR, false, g, J,
                                                                                 ctx->d_xq, Pi, gRp, gPi);
                }
                if (want_gr) {
                    KB_LAUNCH(ctx, st, "k_vjp_gr");
                    k_vjp_gr<<<dim3((g.nq + 127) / 128, J.nw_chunk), 128, 0, st>>>(ctx->m, J, g.A, ctx->d_xq, ctx->d_wq,
                                                                                 gPi, gtab);
                }
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { ctx->err = std::string("vjp launch: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
        }
    }
    return KB_OK;
}
