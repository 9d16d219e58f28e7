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
#include "kb_mixed.cuh"

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
                if (!kb_rec_ok((long long)(base / 16), (long long)nw * (k == 0 ? 1 : nv) * (k == 3 ? nv : 1),
                               KB_SITE_FP64_ADJ))
                    continue;
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


// ------------------------------------------------------------------------------------
// Mixed-precision adjoint: the same pipeline with the records of the complex64 vertex
// evaluated as the mixed forward evaluates them (double-float frequencies and stencils,
// FP32 interpolation, vertex_part_f32), FP32 tiles, products and GEMMs, and every sum
// over many terms — the scatter into the complex128 gradient slots through the transposed
// interpolation and the Pi gradient — accumulated with FP64 atomic adds.  The Pi table and
// its pull-back to G^R stay FP64.
// ------------------------------------------------------------------------------------

// Warp-cooperative scatter of one corner: lane L adds wgt * bar into record idx of D
// (idx < 0: nothing), component o of bar onto component o, or o with a1 <-> a2 when swap12.
// Consecutive lanes hold consecutive quadrature nodes, which mostly interpolate from the
// same records, so the lanes that share a record first sum their 32 reals by a butterfly
// reduce-scatter (lane L ends with real L of the sum) and then issue one FP64 atomic add
// each: one warp-wide atomic per distinct record instead of 32 per lane.  All 32 lanes of
// the warp must call it together.
__device__ __forceinline__ void warp_scatter(double2* __restrict__ D, int idx, float wgt, bool swap12,
                                             const float2 bar[16]) {
    const int lane = threadIdx.x & 31;
    unsigned todo = __ballot_sync(0xffffffffu, idx >= 0);
    while (todo) {
        const int lead = __ffs(todo) - 1;
        const int lidx = __shfl_sync(0xffffffffu, idx, lead);
        const bool mine = idx == lidx;
        todo &= ~__ballot_sync(0xffffffffu, mine);
        const float wm = mine ? wgt : 0.f;
        float v[32];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            // source component of destination e: kswap12 exchanges 1 <-> 2 within each group of 4
            const int q = e & 3;
            const float2 b = (q == 1) ? (swap12 ? bar[e + 1] : bar[e])
                                      : ((q == 2) ? (swap12 ? bar[e - 1] : bar[e]) : bar[e]);
            v[2 * e] = wm * b.x;
            v[2 * e + 1] = wm * b.y;
        }
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            const bool hi = (lane & d) != 0;
#pragma unroll
            for (int i = 0; i < d; ++i) {
                const float send = hi ? v[i] : v[i + d];
                const float keep = hi ? v[i + d] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, d);
            }
        }
        atomicAdd(reinterpret_cast<double*>(D + (size_t)lidx * 16) + lane, (double)v[0]);
    }
}

// Transpose of corners() for one class, warp-cooperatively: corner cc of every lane's
// stencil (valid: the lane's class applies) with the forward's FP32 weight.
__device__ __forceinline__ void corners_adj_warp(double2* __restrict__ D, bool valid, int nd, int k0, int k1, int k2,
                                                 float t0, float t1, float t2, int N0, int N1, int N2, float f,
                                                 bool swap12, const float2 bar[16]) {
    int kk[3] = {k0, k1, k2}, N[3] = {N0, N1, N2};
    float tt[3] = {t0, t1, t2};
    int st[3] = {1, 1, 1};
    if (nd == 2) st[0] = N[1];
    if (nd == 3) { st[1] = N[2]; st[0] = N[1] * N[2]; }
    const int base = kk[0] * st[0] + (nd >= 2 ? kk[1] * st[1] : 0) + (nd == 3 ? kk[2] * st[2] : 0);
#pragma unroll 1
    for (int cc = 0; cc < (1 << nd); ++cc) {
        float wgt = f;
        int of = base;
        bool ok = valid;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d < nd) {
                const bool bt = (cc >> d) & 1;
                ok = ok && (bt ? (kk[d] + 1 < N[d]) : (kk[d] >= 0));
                wgt *= bt ? tt[d] : 1.f - tt[d];
                of += bt ? st[d] : 0;
            }
        }
        const bool use = ok && wgt != 0.f && kb_rec_ok(of, (long long)N[0] * N[1] * N[2], KB_SITE_MIXED_ADJ);
        warp_scatter(D, use ? of : -1, wgt, swap12, bar);
    }
}

__device__ __forceinline__ double2* grad_ptr(const VertexF& VG, int ch, int k) {
    return reinterpret_cast<double2*>(const_cast<float2*>(vcls(VG, ch, k)));
}

// Transpose of vertex_part_f32 for the parts `what` (the bare part has no gradient), for
// the records of a warp (lanes with live = false contribute nothing; the control flow is
// uniform over the warp).  VG holds the gradient slot's complex128 classes (as pointers
// only) and the forward vertex's channel mask; a class the gradient slot lacks receives
// nothing.
template <int r>
__device__ void vertex_part_adj_f32(const VertexF& VG, const DfGrids& G, int parts, bool right, int what, df w, df v,
                                    df vp, const float2 bar[16], bool live) {
    const bool dir = parts & PARTS_UD, exch = parts & PARTS_X;
    const int k_free = right ? 1 : 2, k_dep = right ? 2 : 1;
    unsigned own = 0;
    if (what & 2) own |= 1u << 0;
    if (what & 4) own |= 1u << k_free;
    if (what & 8) own |= 1u << k_dep;
    if (what & 16) own |= 1u << 3;
    if (!((VG.mask >> r) & 1)) own = 0;
    const bool cross_l = (what & 32) && isfinite(v.h) && isfinite(vp.h);
    const bool cross = __any_sync(0xffffffffu, live && cross_l);
    constexpr int sr = (r == KB_CH_A) ? KB_CH_T : (r == KB_CH_T ? KB_CH_A : KB_CH_P);
#pragma unroll 1
    for (int grp = 0; grp < 6; ++grp) {
        int ch;
        unsigned classes;
        float f = 1.f;
        bool sw = false, ok = live;
        df gw, gv, gp;
        if (grp == 0) {
            if (!own || !dir) continue;
            ch = r; classes = own; gw = w; gv = v; gp = vp;
        } else if (grp == 1) {
            if (!own || !exch) continue;
            ch = sr; classes = own; f = -1.f; sw = true;
            gw = (r == KB_CH_P) ? w : df_neg(w); gv = v; gp = (r == KB_CH_P) ? df_neg(vp) : vp;
        } else {
            if (!cross || (grp < 4 ? !dir : !exch)) continue;
            const int c = (grp & 1) ? ((r == 2) ? 1 : 2) : ((r == 0) ? 1 : 0);
            if (!((VG.mask >> c) & 1)) continue;
            ok = ok && cross_l;
            df L[4];
            df_legs(r, w, v, vp, L);
            classes = 15;
            if (grp < 4) {
                ch = c;
                df_vars(c, L, gw, gv, gp);
            } else {
                ch = (c == KB_CH_A) ? KB_CH_T : (c == KB_CH_T ? KB_CH_A : KB_CH_P);
                df S4[4] = {L[0], L[1], L[3], L[2]};
                df_vars(ch, S4, gw, gv, gp);
                f = -1.f;
                sw = true;
            }
        }
        const Sten7 S = stencils7(VG, ch, classes, G, gw, gv, gp);
        if ((classes & 1) && vcls(VG, ch, 0))
            corners_adj_warp(grad_ptr(VG, ch, 0), ok && S.u0, 1, S.kw1, 0, 0, S.tw1, 0.f, 0.f, G.N1, 1, 1, f, sw, bar);
        if ((classes & 2) && vcls(VG, ch, 1))
            corners_adj_warp(grad_ptr(VG, ch, 1), ok && S.u1, 2, S.kw2, S.kv2, 0, S.tw2, S.tv2, 0.f, G.N2w, G.N2v, 1, f,
                             sw, bar);
        if ((classes & 4) && vcls(VG, ch, 2))
            corners_adj_warp(grad_ptr(VG, ch, 2), ok && S.u2, 2, S.kw2, S.kp2, 0, S.tw2, S.tp2, 0.f, G.N2w, G.N2v, 1, f,
                             sw, bar);
        if ((classes & 8) && vcls(VG, ch, 3))
            corners_adj_warp(grad_ptr(VG, ch, 3), ok && S.u3, 3, S.kw3, S.kv3, S.kp3, S.tw3, S.tv3, S.tp3, G.N3w, G.N3v,
                             G.N3v, f, sw, bar);
    }
}

// Frequencies and part selection of one tile record (w, external v, s, node j), as the
// FP64 tile kernels take them: the spin term of the t channel is up-up for the left s = 0
// and the right s = 1; the zero part reads R + K1_r + the external-free own class, the
// v-part the external-dependent own class, K3_r and the other channels.
struct RecArgs {
    df w, vext, vpp;
    int parts, what;
};
template <bool RIGHT>
__device__ __forceinline__ RecArgs rec_args(const DfGrids& G, const ClassJob& J, const df* __restrict__ wgrid,
                                            const df* __restrict__ vgrid, int wl, int vi, int s, int j) {
    RecArgs a;
    const bool nupart = RIGHT ? J.R_nu : J.L_nu;
    a.w = wgrid[J.w0 + wl];
    a.vext = nupart ? vgrid[vi] : df{0.f, 0.f};
    a.vpp = (G.n3v + G.N3v)[j];
    const bool uu = (J.r == KB_CH_T) && (RIGHT ? (s == 1) : (s == 0));
    a.parts = uu ? PARTS_UU : PARTS_UD;
    a.what = nupart ? (8 | 16 | 32) : (1 | 2 | 4);
    return a;
}

// One thread per (w, external v, s, j): the left tile L (FP32) or the Pi-folded right tile
// R' = sum_D Pi[B][D] R[D][C], as k_gather_f64.
template <bool RIGHT, int R>
__global__ void k_vjp_tile_f32(VertexF V, DfGrids G, ClassJob J, const df* __restrict__ wgrid,
                               const df* __restrict__ vgrid, const double2* __restrict__ Pi, float2* __restrict__ tile) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y % J.ns, vi = blockIdx.y / J.ns, wl = blockIdx.z;
    const int nrow = RIGHT ? J.nR : J.nL;
    if (j >= J.nq || vi >= nrow) return;
    const ChannelMaps& M = c_maps[R];
    const RecArgs a = rec_args<RIGHT>(G, J, wgrid, vgrid, wl, vi, s, j);
    float2 g[16];
    if (RIGHT) vertex_part_f32<R>(V, G, a.parts, true, a.what, a.w, a.vpp, a.vext, g);
    else vertex_part_f32<R>(V, G, a.parts, false, a.what, a.w, a.vext, a.vpp, g);
    const size_t K = (size_t)4 * J.ns * J.nq, kcol = ((size_t)s * J.nq + j) * 4;
    const size_t rowbase = (size_t)wl * 4 * nrow + (size_t)vi * 4;
    if (!RIGHT) {
        for (int A = 0; A < 4; ++A)
            for (int B = 0; B < 4; ++B) tile[(rowbase + A) * K + kcol + B] = g[M.cL[A][B]];
    } else {
        const double2* P = Pi + ((size_t)wl * J.nq + j) * 16;
        float2 pm[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) pm[i] = make_float2((float)P[i].x, (float)P[i].y);
        for (int C = 0; C < 4; ++C)
            for (int B = 0; B < 4; ++B) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int D = 0; D < 4; ++D) cmac2(acc, pm[4 * B + D], g[M.cR[D][C]]);
                tile[(rowbase + C) * K + kcol + B] = acc;
            }
    }
}

// Gbar (FP32) = alpha * bar(out), laid out as k_vjp_gbar.
__global__ void k_vjp_gbar_f32(ClassJob J, int cls, const void* gout, int dt, double alpha, float2* __restrict__ Gb) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)J.nw_chunk * J.nL * J.nR * 16) return;
    const int o = idx % 16;
    size_t rest = idx / 16;
    const int vR = rest % J.nR;
    rest /= J.nR;
    const int vL = rest % J.nL;
    const int wl = rest / J.nL;
    const ChannelMaps& M = c_maps[J.r];
    int A = 0, C = 0;
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 4; ++c)
            if (M.cO[a][c] == o) { A = a; C = c; }
    const size_t w = J.w0 + wl;
    size_t e;
    if (cls == KB_K1) e = w * 16 + o;
    else if (cls == KB_K2) e = (w * J.nL + vL) * 16 + o;
    else if (cls == KB_K2P) e = (w * J.nR + vR) * 16 + o;
    else e = ((w * J.nL + vL) * J.nR + vR) * 16 + o;
    const double2 g = ld_c(gout, dt, e);
    Gb[((size_t)wl * 4 * J.nL + 4 * vL + A) * (4 * J.nR) + 4 * vR + C] =
        make_float2((float)(alpha * g.x), (float)(alpha * g.y));
}

// k_zgemm_gen in FP32 (complex, FP32 accumulation over the short inner dimension 4 nL or
// 4 nR of the adjoint GEMMs).
__global__ void __launch_bounds__(256) k_cgemm_gen_f32(const float2* __restrict__ A, const float2* __restrict__ B,
                                                       float2* __restrict__ C, GemmDesc d) {
    __shared__ float2 sA[16][33], sB[16][33];
    const int b = blockIdx.z;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const float2* Ab = A + b * d.sAb;
    const float2* Bb = B + b * d.sBb;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float2 acc[2][2] = {};
    for (int l0 = 0; l0 < d.L; l0 += 16) {
        for (int t = threadIdx.x; t < 32 * 16; t += 256) {
            const int ll = t / 32, rr = t % 32;
            const int gi = i0 + rr, gj = j0 + rr, gl = l0 + ll;
            float2 a = make_float2(0.f, 0.f), bv = a;
            if (gi < d.I && gl < d.L) a = Ab[gi * d.sAi + gl * d.sAl];
            if (gj < d.J && gl < d.L) bv = Bb[gl * d.sBl + gj * d.sBj];
            if (d.conjA) a.y = -a.y;
            if (d.conjB) bv.y = -bv.y;
            sA[ll][rr] = a;
            sB[ll][rr] = bv;
        }
        __syncthreads();
#pragma unroll
        for (int ll = 0; ll < 16; ++ll) {
            const float2 a0 = sA[ll][ty], a1 = sA[ll][ty + 16];
            const float2 b0 = sB[ll][tx], b1 = sB[ll][tx + 16];
            cmac2(acc[0][0], a0, b0);
            cmac2(acc[0][1], a0, b1);
            cmac2(acc[1][0], a1, b0);
            cmac2(acc[1][1], a1, b1);
        }
        __syncthreads();
    }
    for (int i = 0; i < 2; ++i)
        for (int jj = 0; jj < 2; ++jj) {
            const int gi = i0 + ty + 16 * i, gj = j0 + tx + 16 * jj;
            if (gi < d.I && gj < d.J) C[b * d.sCb + gi * d.sCi + gj] = acc[i][jj];
        }
}

// Warp w of a scatter launch: record row (wl, v, s) and nodes 32 b .. 32 b + 31 of it, one
// node per lane (rows of nrow external points; nblk = ceil(nq / 32) blocks per row).
struct WarpRec {
    int wl, vi, s, j;
    bool live, in;
};
__device__ __forceinline__ WarpRec warp_record(const ClassJob& J, int nrow) {
    WarpRec q;
    const int nblk = (J.nq + 31) / 32;
    const size_t gw = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t rows = (size_t)J.nw_chunk * J.ns * nrow;
    q.in = gw < rows * nblk;                       // uniform over the warp
    const size_t row = q.in ? gw / nblk : 0;
    q.j = (int)(gw % nblk) * 32 + (int)(threadIdx.x & 31);
    q.live = q.in && q.j < J.nq;
    q.j = min(q.j, J.nq - 1);
    q.vi = (int)(row % nrow);
    q.s = (int)((row / nrow) % J.ns);
    q.wl = (int)(row / nrow / J.ns);
    return q;
}

// bar(L) -> gradient slot, one warp per 32 consecutive nodes of a (w, v, s) row.
template <int R>
__global__ void k_vjp_left_f32(VertexF VG, DfGrids G, ClassJob J, const df* __restrict__ wgrid,
                               const df* __restrict__ vgrid, const float2* __restrict__ gL) {
    const WarpRec q = warp_record(J, J.nL);
    if (!q.in) return;
    const ChannelMaps& M = c_maps[R];
    const RecArgs a = rec_args<false>(G, J, wgrid, vgrid, q.wl, q.vi, q.s, q.j);
    const size_t K = (size_t)4 * J.ns * J.nq, kcol = ((size_t)q.s * J.nq + q.j) * 4;
    const size_t rowbase = (size_t)q.wl * 4 * J.nL + (size_t)q.vi * 4;
    float2 bar[16];
    for (int A = 0; A < 4; ++A)
        for (int B = 0; B < 4; ++B)
            bar[M.cL[A][B]] = q.live ? gL[(rowbase + A) * K + kcol + B] : make_float2(0.f, 0.f);
    vertex_part_adj_f32<R>(VG, G, a.parts, false, a.what, a.w, a.vext, a.vpp, bar, q.live);
}

// bar(R') -> bar(R)[D][C] = sum_B conj(Pi[B][D]) bar(R')[C][B] -> gradient slot, one warp per
// 32 consecutive nodes of a (w, v', s) row.
template <int R>
__global__ void k_vjp_right_f32(VertexF VG, DfGrids G, ClassJob J, const df* __restrict__ wgrid,
                                const df* __restrict__ vgrid, const double2* __restrict__ Pi,
                                const float2* __restrict__ gRp) {
    const WarpRec q = warp_record(J, J.nR);
    if (!q.in) return;
    const ChannelMaps& M = c_maps[R];
    const RecArgs a = rec_args<true>(G, J, wgrid, vgrid, q.wl, q.vi, q.s, q.j);
    const size_t K = (size_t)4 * J.ns * J.nq, kcol = ((size_t)q.s * J.nq + q.j) * 4;
    const size_t rowbase = (size_t)q.wl * 4 * J.nR + (size_t)q.vi * 4;
    const double2* P = Pi + ((size_t)q.wl * J.nq + q.j) * 16;
    float2 bar[16];
    for (int D = 0; D < 4; ++D)
        for (int C = 0; C < 4; ++C) {
            float2 acc = make_float2(0.f, 0.f);
            if (q.live)
                for (int B = 0; B < 4; ++B)
                    cmac2(acc, make_float2((float)P[4 * B + D].x, -(float)P[4 * B + D].y),
                          gRp[(rowbase + C) * K + kcol + B]);
            bar[M.cR[D][C]] = acc;
        }
    vertex_part_adj_f32<R>(VG, G, a.parts, true, a.what, a.w, a.vpp, a.vext, bar, q.live);
}

// bar(Pi)[w][j][B][D] += sum_C conj(R[D][C]) bar(R')[C][B], one thread per (w, v', s, j)
// record with consecutive threads on consecutive nodes (whose Pi entries differ).
template <int R>
__global__ void k_vjp_pi_f32(VertexF V, DfGrids G, ClassJob J, const df* __restrict__ wgrid,
                             const df* __restrict__ vgrid, const float2* __restrict__ gRp, double2* __restrict__ gPi) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)J.nw_chunk * J.ns * J.nR * J.nq) return;
    const int j = (int)(idx % J.nq);
    size_t rest = idx / J.nq;
    const int vi = (int)(rest % J.nR);
    rest /= J.nR;
    const int s = (int)(rest % J.ns);
    const int wl = (int)(rest / J.ns);
    const ChannelMaps& M = c_maps[R];
    const RecArgs a = rec_args<true>(G, J, wgrid, vgrid, wl, vi, s, j);
    const size_t K = (size_t)4 * J.ns * J.nq, kcol = ((size_t)s * J.nq + j) * 4;
    const size_t rowbase = (size_t)wl * 4 * J.nR + (size_t)vi * 4;
    float2 g[16];
    vertex_part_f32<R>(V, G, a.parts, true, a.what, a.w, a.vpp, a.vext, g);
    double2* dst = gPi + ((size_t)wl * J.nq + j) * 16;
    for (int B = 0; B < 4; ++B)
        for (int D = 0; D < 4; ++D) {
            float2 acc = make_float2(0.f, 0.f);
            for (int C = 0; C < 4; ++C) {
                const float2 rv = g[M.cR[D][C]];
                cmac2(acc, make_float2(rv.x, -rv.y), gRp[(rowbase + C) * K + kcol + B]);
            }
            atomic_cadd(dst + 4 * B + D, make_double2(acc.x, acc.y));
        }
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


// Mixed-precision adjoint (kb_bubble_vjp with KB_PREC_MIXED): the pipeline of
// kb_bubble_vjp_fp64 with FP32 tiles and GEMMs on the complex64 vertex.
template <int R>
static kb_status vjp_mixed_impl(kb_ctx* ctx, int sl, int sr, int sgo, int pi_kind, unsigned mask, double alpha,
                                int sgl, int sgr, void* const gGR[3], cudaStream_t st) {
    VertexF VL, VRt;
    if (!kb_slot_f32(ctx, sl, VL) || !kb_slot_f32(ctx, sr, VRt)) return KB_ERR_ARG;
    const VertexDev none{};
    auto grad_view = [&](int gs, const VertexDev& fwd) {
        const VertexDev& Gd = gs >= 0 ? ctx->slots[gs] : none;
        VertexF F;
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 4; ++k) F.cls[c][k] = reinterpret_cast<const float2*>(Gd.cls[c][k]);
        F.has_R = 0;
        F.mask = fwd.mask;
        F.bare = 0.f;
        return F;
    };
    const VertexF GVL = grad_view(sgl, ctx->slots[sl]), GVR = grad_view(sgr, ctx->slots[sr]);
    const Grids& g = ctx->g;
    const int ns = (R == KB_CH_T) ? 2 : 1;
    const size_t K = (size_t)4 * ns * g.nq;
    const size_t ntab = (size_t)g.n1 + g.n2w + g.n2v + g.n3w + g.n3v + g.nq;
    const size_t tab_bytes = (ntab * sizeof(df) + 255) / 256 * 256;
    for (int cls = 0; cls < 4; ++cls) {
        if (!((mask >> cls) & 1)) continue;
        double2* gtab = reinterpret_cast<double2*>(gGR ? gGR[cls == KB_K1 ? 0 : (cls == KB_K3 ? 2 : 1)] : nullptr);
        const bool want_l = sgl >= 0, want_r = sgr >= 0, want_gr = gtab != nullptr;
        if (!want_l && !want_r && !want_gr) continue;
        int nw, nL, nR, nvg;
        class_shape(g, cls, nw, nL, nR, nvg);
        const size_t tileL = (size_t)4 * nL * K, tileR = (size_t)4 * nR * K, nGb = (size_t)16 * nL * nR;
        const size_t per_w = (size_t)g.nq * 16 * sizeof(double2) * (want_gr ? 2 : 1) +
                             (2 * tileL + 2 * tileR + nGb) * sizeof(float2);
        const int chunk = (int)std::max<size_t>(1, std::min<size_t>(nw, ctx->ws_limit / per_w));
        kb_status s = kb_ensure_workspace(ctx, tab_bytes + per_w * chunk, st);
        if (s != KB_OK) return s;
        char* ws = static_cast<char*>(ctx->ws.ptr);
        DfGrids G;
        kb_mixed_tables(ctx, reinterpret_cast<df*>(ws), G, st);
        double2* Pi = reinterpret_cast<double2*>(ws + tab_bytes);
        double2* gPi = Pi + (size_t)chunk * g.nq * 16;
        float2* Lt = reinterpret_cast<float2*>(gPi + (want_gr ? (size_t)chunk * g.nq * 16 : 0));
        float2* Rt = Lt + (size_t)chunk * tileL;
        float2* gL = Rt + (size_t)chunk * tileR;
        float2* gRp = gL + (size_t)chunk * tileL;
        float2* Gb = gRp + (size_t)chunk * tileR;
        const df* wgrid = cls == KB_K1 ? G.n1 : (cls == KB_K3 ? G.n3w : G.n2w);
        const df* vgrid = cls == KB_K3 ? G.n3v : G.n2v;
        for (int w0 = 0; w0 < nw; w0 += chunk) {
            ClassJob J;
            J.r = R; J.pi_kind = pi_kind; J.ns = ns; J.nq = g.nq;
            J.nw_chunk = std::min(chunk, nw - w0); J.w0 = w0; J.nw_grid = nw;
            J.nL = nL; J.nR = nR; J.nvL_grid = nvg; J.nvR_grid = nvg;
            J.L_nu = (cls == KB_K2 || cls == KB_K3);
            J.R_nu = (cls == KB_K2P || cls == KB_K3);
            const int Mr = 4 * nL, Nc = 4 * nR;
            {
                KB_LAUNCH(ctx, st, "k_pi_table");
                k_pi_table<<<dim3((g.nq + 127) / 128, J.nw_chunk), 128, 0, st>>>(ctx->m, J, g.A, ctx->d_xq, ctx->d_wq, Pi);
            }
            {
                KB_LAUNCH(ctx, st, "k_vjp_tile_f32_left");
                k_vjp_tile_f32<false, R><<<dim3((g.nq + 127) / 128, nL * ns, J.nw_chunk), 128, 0, st>>>(
                    VL, G, J, wgrid, vgrid, Pi, Lt);
            }
            {
                KB_LAUNCH(ctx, st, "k_vjp_tile_f32_right");
                k_vjp_tile_f32<true, R><<<dim3((g.nq + 127) / 128, nR * ns, J.nw_chunk), 128, 0, st>>>(
                    VRt, G, J, wgrid, vgrid, Pi, Rt);
            }
            {
                KB_LAUNCH(ctx, st, "k_vjp_gbar_f32");
                const size_t tot = (size_t)J.nw_chunk * nL * nR * 16;
                k_vjp_gbar_f32<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(J, cls, ctx->slots[sgo].cls[R][cls],
                                                                             ctx->slots[sgo].dt[R][cls], alpha, Gb);
            }
            if (want_l) {
                GemmDesc d{Mr, (int)K, Nc, (long long)Mr * Nc, Nc, 1, (long long)tileR, (long long)K, 1,
                           (long long)tileL, (long long)K, false, true};
                {
                    KB_LAUNCH(ctx, st, "k_cgemm_gen_f32");
                    k_cgemm_gen_f32<<<dim3((unsigned)((K + 31) / 32), (Mr + 31) / 32, J.nw_chunk), 256, 0, st>>>(
                        Gb, Rt, gL, d);
                }
                {
                    KB_LAUNCH(ctx, st, "k_vjp_left_f32");
                    const size_t tot = (size_t)J.nw_chunk * ns * nL * ((g.nq + 31) / 32) * 32;
                    k_vjp_left_f32<R><<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(GVL, G, J, wgrid, vgrid, gL);
                }
            }
            if (want_r || want_gr) {
                GemmDesc d{Nc, (int)K, Mr, (long long)Mr * Nc, 1, Nc, (long long)tileL, (long long)K, 1,
                           (long long)tileR, (long long)K, false, true};
                {
                    KB_LAUNCH(ctx, st, "k_cgemm_gen_f32");
                    k_cgemm_gen_f32<<<dim3((unsigned)((K + 31) / 32), (Nc + 31) / 32, J.nw_chunk), 256, 0, st>>>(
                        Gb, Lt, gRp, d);
                }
                if (want_gr)
                    KB_CUDA_TRY(ctx, cudaMemsetAsync(gPi, 0, (size_t)J.nw_chunk * g.nq * 16 * sizeof(double2), st));
                if (want_r) {
                    KB_LAUNCH(ctx, st, "k_vjp_right_f32");
                    const size_t tot = (size_t)J.nw_chunk * ns * nR * ((g.nq + 31) / 32) * 32;
                    k_vjp_right_f32<R><<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(GVR, G, J, wgrid, vgrid, Pi,
                                                                                     gRp);
                }
                if (want_gr) {
                    {
                        KB_LAUNCH(ctx, st, "k_vjp_pi_f32");
                        const size_t tot = (size_t)J.nw_chunk * ns * nR * g.nq;
                        k_vjp_pi_f32<R><<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(VRt, G, J, wgrid, vgrid, gRp,
                                                                                      gPi);
                    }
                    KB_LAUNCH(ctx, st, "k_vjp_gr");
                    k_vjp_gr<<<dim3((g.nq + 127) / 128, J.nw_chunk), 128, 0, st>>>(ctx->m, J, g.A, ctx->d_xq, ctx->d_wq,
                                                                                 gPi, gtab);
                }
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { ctx->err = std::string("mixed vjp launch: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
        }
    }
    return KB_OK;
}

kb_status kb_bubble_vjp_mixed(kb_ctx* ctx, int r, int sl, int sr, int sgo, int pi_kind, unsigned mask, double alpha,
                              int sgl, int sgr, void* const gGR[3], cudaStream_t st) {
    if (!g_vjp_maps_uploaded[ctx->device]) {
        ChannelMaps h[3] = {channel_maps(0), channel_maps(1), channel_maps(2)};
        KB_CUDA_TRY(ctx, cudaMemcpyToSymbol(c_maps, h, sizeof(h)));
        g_vjp_maps_uploaded[ctx->device] = true;
    }
    if (r == KB_CH_A) return vjp_mixed_impl<KB_CH_A>(ctx, sl, sr, sgo, pi_kind, mask, alpha, sgl, sgr, gGR, st);
    if (r == KB_CH_P) return vjp_mixed_impl<KB_CH_P>(ctx, sl, sr, sgo, pi_kind, mask, alpha, sgl, sgr, gGR, st);
    return vjp_mixed_impl<KB_CH_T>(ctx, sl, sr, sgo, pi_kind, mask, alpha, sgl, sgr, gGR, st);
}
