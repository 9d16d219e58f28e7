// Mixed-precision device helpers: double-float (pair of FP32) frequency arithmetic and an
// FP32 vertex gather whose interpolation weights are accurate to ~1e-7 even on fine grids.
//
// Why double-float: a vertex class is interpolated linearly in x = (2/pi) atan(v/A)
// (Sec. II.G.7).  The weight of a node is (x - X_k)(N+1)/2; with x in plain FP32 its
// absolute error (~6e-8) is amplified by (N+1)/2, which for a 401-point grid of random
// data would be a 1e-5 relative error.  Here the frequency sums are exact to ~1e-14
// (two-sum), the cell is found exactly by comparing against the node frequencies, and the
// fraction uses atan(a) - atan(b) = atan((a - b)/(1 + ab)) with a - b formed in
// double-float, so the weight carries only the FP32 relative error of a small number.
#pragma once
#include "kb_dev.cuh"

namespace kb {

struct df {
    float h, l;
};

__device__ __forceinline__ df df_make(double x) {
    float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ df df_add(df a, df b) {
    float s = __fadd_rn(a.h, b.h);
    float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_half(df a) { return {0.5f * a.h, 0.5f * a.l}; }
__device__ __forceinline__ bool df_lt(df a, df b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }

// Node tables of the class grids (double-float), in device memory.
struct DfGrids {
    const df* n1;     // K1 bosonic
    const df* n2w;    // K2 bosonic
    const df* n2v;    // K2 fermionic
    const df* n3w;    // K3 bosonic
    const df* n3v;    // K3 fermionic
    int N1, N2w, N2v, N3w, N3v;
    float A;
};

// Cell estimate x ~ (2/pi) atan(v/A) of a frequency, shared by all grids that read it.
// It only has to land within one cell of the true one (the cell is then fixed by exact
// double-float comparisons with the node frequencies), so a short odd polynomial in
// u = min(|y|, 1/|y|), y = v/A, does: (2/pi) atan(u) ~ u (c0 + c1 u^2 + c2 u^4 + c3 u^6),
// least-squares fit on [0, 1] (csrc/fit_atan_estimate.py), max error 5.2e-5 in x, i.e.
// below 0.03 cells for grids of up to 1000 points; atan(y) = pi/2 - atan(1/y) for y > 1.
__device__ __forceinline__ float x_est(float v, float invA) {
    const float y = fabsf(v) * invA;
    const bool big = y > 1.f;
    const float u = big ? __fdividef(1.f, y) : y;
    const float u2 = u * u;
    const float p = u * fmaf(u2, fmaf(u2, fmaf(u2, -0.02481973f, 0.09311505f), -0.2044664f), 0.63611925f);
    return copysignf(big ? 1.f - p : p, v);
}

// atan(z) for the small arguments of the stencil fraction: the odd Taylor series to z^15
// (relative error below z^16/17, 1.1e-9 at |z| = 0.33); larger |z| (grids of fewer than
// nine points, or the cells next to x = +-1 on such grids) take atanf.
__device__ __forceinline__ float atan_frac(float z) {
    if (fabsf(z) > 0.33f) return atanf(z);
    const float z2 = z * z;
    float p = fmaf(z2, -1.f / 15.f, 1.f / 13.f);
    p = fmaf(z2, p, -1.f / 11.f);
    p = fmaf(z2, p, 1.f / 9.f);
    p = fmaf(z2, p, -1.f / 7.f);
    p = fmaf(z2, p, 1.f / 5.f);
    p = fmaf(z2, p, -1.f / 3.f);
    p = fmaf(z2, p, 1.f);
    return z * p;
}

// Stencil on an N-point grid with zero-valued virtual nodes at x = +-1 from the cell
// estimate x: returns the lower node k in [-1, N-1] and the fraction t toward node k+1.
// The fraction relative to the estimated node uses atan(a) - atan(b) = atan((a - b)/(1 + ab))
// with a - b formed in double-float: x - X_k = (2/pi) atan((v - v_k) A / (A^2 + v v_k)),
// and for k = -1 (v < 0) x + 1 = (2/pi) atan(-A/v).  It is accurate to the FP32 relative
// error of t itself, so the estimate only has to be within one cell: t < 0 or t >= 1
// moves k by one (t + 1, t - 1 are then exact to FP32 rounding).
__device__ __forceinline__ int stencil_x(df v, float x, const df* __restrict__ nodes, int N, float A, float& t) {
    int k = (int)floorf((x + 1.0f) * (0.5f * (float)(N + 1))) - 1;
    k = max(-1, min(k, N - 1));
    if (k < 0 && !(v.h < 0.f)) k = 0;
    const float scale = (float)(N + 1) * 0.318309886183790672f;
    float z;
    if (k < 0) {
        z = __fdividef(-A, v.h);
    } else {
        df nk = nodes[k];
        df d = df_sub(v, nk);
        z = __fdividef((d.h + d.l) * A, fmaf(v.h, nk.h, A * A));
    }
    t = atan_frac(z) * scale;
    if (t < 0.f && k >= 0) { --k; t += 1.f; }
    else if (t >= 1.f && k < N - 1) { ++k; t -= 1.f; }
    t = fminf(fmaxf(t, 0.f), 1.f);
    return k;
}

// acc += x * y (complex), two packed FMAs
__device__ __forceinline__ void cmac2(float2& acc, float2 x, float2 y) {
    acc = __ffma2_rn(make_float2(x.x, x.x), y, acc);
    acc = __ffma2_rn(make_float2(-x.y, x.y), make_float2(y.y, y.x), acc);
}

// legs (v1', v2', v1, v2) and channel variables in double-float (Sec. II.C.1)
__device__ __forceinline__ void df_legs(int r, df w, df v, df vp, df L[4]) {
    df hw = df_half(w);
    if (r == KB_CH_A) { L[0] = df_add(v, hw); L[3] = df_sub(v, hw); L[2] = df_add(vp, hw); L[1] = df_sub(vp, hw); }
    else if (r == KB_CH_P) { L[0] = df_add(hw, v); L[1] = df_sub(hw, v); L[2] = df_add(hw, vp); L[3] = df_sub(hw, vp); }
    else { L[1] = df_add(vp, hw); L[3] = df_sub(vp, hw); L[0] = df_sub(v, hw); L[2] = df_add(v, hw); }
}
__device__ __forceinline__ void df_vars(int c, const df L[4], df& w, df& v, df& vp) {
    if (c == KB_CH_A) { w = df_sub(L[0], L[3]); v = df_half(df_add(L[0], L[3])); vp = df_half(df_add(L[2], L[1])); }
    else if (c == KB_CH_P) { w = df_add(L[0], L[1]); v = df_half(df_sub(L[0], L[1])); vp = df_half(df_sub(L[2], L[3])); }
    else { w = df_sub(L[1], L[3]); v = df_half(df_add(L[0], L[2])); vp = df_half(df_add(L[1], L[3])); }
}

// Compile-time Keldysh index maps of channel R (same as channel_maps in kb_api.cu):
// left tile L[A][B] = Gamma1^{cL(A,B)}, right tile R[D][C] = Gamma2^{cR(D,C)}, output cO(A,C).
template <int R>
__host__ __device__ constexpr int cmap(int X, int Y) {
    return R == KB_CH_A ? 8 * (X >> 1) + 4 * (Y >> 1) + 2 * (Y & 1) + (X & 1)
         : R == KB_CH_P ? 8 * (X >> 1) + 4 * (X & 1) + 2 * (Y >> 1) + (Y & 1)
                        : 8 * (X >> 1) + 4 * (Y >> 1) + 2 * (X & 1) + (Y & 1);
}

// Vertex in device form for the mixed path (complex64 classes only).
struct VertexF {
    const float2* cls[3][4];
    int has_R, mask;
    float bare;
};

// Class pointer of channel ch (a runtime value) without indexing the parameter struct at run
// time, which would copy it to local memory: a chain of selects over the 12 entries.
__device__ __forceinline__ const float2* vcls(const VertexF& V, int ch, int k) {
    const float2* p = nullptr;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (c == ch && q == k) p = V.cls[c][q];
    return p;
}

// Corners of one class: nd dimensions with lower nodes kk[d], fractions tt[d] and sizes N[d]
// (row-major data, 16 complex components per record); the corner code exists once.  Two
// records are loaded before either is applied; ONE: one record at a time (fewer registers,
// for the K3 tile kernel, which runs more CTAs per SM instead).
template <bool ONE = false>
__device__ __forceinline__ void corners(const float2* __restrict__ D, int nd, int k0, int k1, int k2, float t0,
                                        float t1, float t2, int N0, int N1, int N2, float f, bool swap12,
                                        float2 acc[16]) {
    int kk[3] = {k0, k1, k2}, N[3] = {N0, N1, N2};
    float tt[3] = {t0, t1, t2};
    int st[3] = {1, 1, 1};
    if (nd == 2) st[0] = N[1];
    if (nd == 3) { st[1] = N[2]; st[0] = N[1] * N[2]; }
    int base = kk[0] * st[0] + (nd >= 2 ? kk[1] * st[1] : 0) + (nd == 3 ? kk[2] * st[2] : 0);
    int ncorner = 1 << nd;   // even
    if (ONE) {
#pragma unroll 1
        for (int c = 0; c < ncorner; ++c) {
            float wgt = f;
            int of = base;
            bool ok = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d < nd) {
                    bool bt = (c >> d) & 1;
                    ok = ok && (bt ? (kk[d] + 1 < N[d]) : (kk[d] >= 0));
                    wgt *= bt ? tt[d] : 1.f - tt[d];
                    of += bt ? st[d] : 0;
                }
            }
            if (!(ok && wgt != 0.f && kb_rec_ok(of, (long long)N[0] * N[1] * N[2], KB_SITE_MIXED_REC))) continue;
            float4 u[8];
            const float4* q = reinterpret_cast<const float4*>(D + (size_t)of * 16);
#pragma unroll
            for (int i = 0; i < 8; ++i) u[i] = __ldg(q + i);
            const float2 g = make_float2(wgt, wgt);
#pragma unroll
            for (int grp = 0; grp < 4; ++grp) {
                float2 a0 = make_float2(u[2 * grp].x, u[2 * grp].y), a1 = make_float2(u[2 * grp].z, u[2 * grp].w);
                float2 a2 = make_float2(u[2 * grp + 1].x, u[2 * grp + 1].y);
                float2 a3 = make_float2(u[2 * grp + 1].z, u[2 * grp + 1].w);
                if (swap12) {
                    float2 t0 = a1; a1 = a2; a2 = t0;
                }
                acc[4 * grp + 0] = __ffma2_rn(g, a0, acc[4 * grp + 0]);
                acc[4 * grp + 1] = __ffma2_rn(g, a1, acc[4 * grp + 1]);
                acc[4 * grp + 2] = __ffma2_rn(g, a2, acc[4 * grp + 2]);
                acc[4 * grp + 3] = __ffma2_rn(g, a3, acc[4 * grp + 3]);
            }
        }
        return;
    }
    // two corners per iteration: both records are loaded before either is applied
#pragma unroll 1
    for (int c = 0; c < ncorner; c += 2) {
        float wg[2];
        int off[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            int cc = c + e;
            float wgt = f;
            int of = base;
            bool ok = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d < nd) {
                    bool bt = (cc >> d) & 1;
                    ok = ok && (bt ? (kk[d] + 1 < N[d]) : (kk[d] >= 0));
                    wgt *= bt ? tt[d] : 1.f - tt[d];
                    of += bt ? st[d] : 0;
                }
            }
            bool use = ok && wgt != 0.f && kb_rec_ok(of, (long long)N[0] * N[1] * N[2], KB_SITE_MIXED_REC);
            wg[e] = use ? wgt : 0.f;
            off[e] = use ? of : -1;
        }
        float4 u0[8], u1[8];
        const float4* q0 = reinterpret_cast<const float4*>(D + (size_t)max(off[0], 0) * 16);
        const float4* q1 = reinterpret_cast<const float4*>(D + (size_t)max(off[1], 0) * 16);
#pragma unroll
        for (int i = 0; i < 8; ++i) u0[i] = off[0] >= 0 ? __ldg(q0 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 8; ++i) u1[i] = off[1] >= 0 ? __ldg(q1 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 g0 = make_float2(wg[0], wg[0]), g1 = make_float2(wg[1], wg[1]);
#pragma unroll
        for (int grp = 0; grp < 4; ++grp) {
            float2 a0 = make_float2(u0[2 * grp].x, u0[2 * grp].y), a1 = make_float2(u0[2 * grp].z, u0[2 * grp].w);
            float2 a2 = make_float2(u0[2 * grp + 1].x, u0[2 * grp + 1].y);
            float2 a3 = make_float2(u0[2 * grp + 1].z, u0[2 * grp + 1].w);
            float2 b0 = make_float2(u1[2 * grp].x, u1[2 * grp].y), b1 = make_float2(u1[2 * grp].z, u1[2 * grp].w);
            float2 b2 = make_float2(u1[2 * grp + 1].x, u1[2 * grp + 1].y);
            float2 b3 = make_float2(u1[2 * grp + 1].z, u1[2 * grp + 1].w);
            if (swap12) {
                float2 t0 = a1; a1 = a2; a2 = t0;
                float2 t1 = b1; b1 = b2; b2 = t1;
            }
            acc[4 * grp + 0] = __ffma2_rn(g1, b0, __ffma2_rn(g0, a0, acc[4 * grp + 0]));
            acc[4 * grp + 1] = __ffma2_rn(g1, b1, __ffma2_rn(g0, a1, acc[4 * grp + 1]));
            acc[4 * grp + 2] = __ffma2_rn(g1, b2, __ffma2_rn(g0, a2, acc[4 * grp + 2]));
            acc[4 * grp + 3] = __ffma2_rn(g1, b3, __ffma2_rn(g0, a3, acc[4 * grp + 3]));
        }
    }
}

// Stencils of one channel's classes at (w, v, vp): K1 on the K1 grid, K2/K2' on the K2
// grids, K3 on the K3 grids; flags say which classes contribute.
struct Sten7 {
    int kw1, kw2, kw3, kv2, kv3, kp2, kp3;
    float tw1, tw2, tw3, tv2, tv3, tp2, tp3;
    bool u0, u1, u2, u3;
};

__device__ __forceinline__ Sten7 stencils7(const VertexF& V, int ch, unsigned classes, const DfGrids& G, df gw, df gv,
                                           df gp) {
    Sten7 S;
    const bool fw = isfinite(gw.h), fv = isfinite(gv.h), fp = isfinite(gp.h);
    const float ia = 1.f / G.A;
    const float xw = fw ? x_est(gw.h, ia) : 0.f, xv = fv ? x_est(gv.h, ia) : 0.f, xp = fp ? x_est(gp.h, ia) : 0.f;
    S.u0 = (classes & 1) && vcls(V, ch, 0) && fw;
    S.u1 = (classes & 2) && vcls(V, ch, 1) && fw && fv;
    S.u2 = (classes & 4) && vcls(V, ch, 2) && fw && fp;
    S.u3 = (classes & 8) && vcls(V, ch, 3) && fw && fv && fp;
    S.tw1 = S.tw2 = S.tw3 = S.tv2 = S.tv3 = S.tp2 = S.tp3 = 0.f;
    S.kw1 = S.kw2 = S.kw3 = S.kv2 = S.kv3 = S.kp2 = S.kp3 = 0;
    if (S.u0) S.kw1 = stencil_x(gw, xw, G.n1, G.N1, G.A, S.tw1);
    if (S.u1 || S.u2) S.kw2 = stencil_x(gw, xw, G.n2w, G.N2w, G.A, S.tw2);
    if (S.u1) S.kv2 = stencil_x(gv, xv, G.n2v, G.N2v, G.A, S.tv2);
    if (S.u2) S.kp2 = stencil_x(gp, xp, G.n2v, G.N2v, G.A, S.tp2);
    if (S.u3) {
        S.kw3 = stencil_x(gw, xw, G.n3w, G.N3w, G.A, S.tw3);
        S.kv3 = stencil_x(gv, xv, G.n3v, G.N3v, G.A, S.tv3);
        S.kp3 = stencil_x(gp, xp, G.n3v, G.N3v, G.A, S.tp3);
    }
    return S;
}

template <bool ONE = false>
__device__ __forceinline__ void apply7(const VertexF& V, int ch, const Sten7& S, const DfGrids& G, float f, bool sw,
                                       float2 out[16]) {
    if (S.u0) corners<ONE>(vcls(V, ch, 0), 1, S.kw1, 0, 0, S.tw1, 0.f, 0.f, G.N1, 1, 1, f, sw, out);
    if (S.u1) corners<ONE>(vcls(V, ch, 1), 2, S.kw2, S.kv2, 0, S.tw2, S.tv2, 0.f, G.N2w, G.N2v, 1, f, sw, out);
    if (S.u2) corners<ONE>(vcls(V, ch, 2), 2, S.kw2, S.kp2, 0, S.tw2, S.tp2, 0.f, G.N2w, G.N2v, 1, f, sw, out);
    if (S.u3) corners<ONE>(vcls(V, ch, 3), 3, S.kw3, S.kv3, S.kp3, S.tw3, S.tv3, S.tp3, G.N3w, G.N3v, G.N3v, f, sw, out);
}

// Parts of the vertex relative to channel r at r-variables (w, v, vp), FP32 accumulation.
// what bits: 1 = R, 2 = K1_r, 4 = ext-free own class (K2'_r left / K2_r right),
// 8 = ext-dependent own class (K2_r left / K2'_r right), 16 = K3_r, 32 = other channels.
// parts: PARTS_UD = the up-down component (direct lookups); PARTS_X = the exchanged term
// of the up-up component alone, -gamma_{sigma(c)}^ud(1'2'|21) channel by channel
// (crossing partner a <-> t, p -> p); PARTS_UU = both, the up-up component.  Since
// up-up = up-down + exchanged term, a caller that needs both spin components evaluates
// PARTS_UD once and then adds PARTS_X onto it (accumulate = true).
// The argument that may be infinite is the quadrature frequency v''; infinite arguments
// make a class read zero, and the other channels then vanish as well.
// All stencils of a group of lookups are computed before its corner loads so that the
// independent stencil computations overlap.
constexpr int PARTS_UD = 1, PARTS_X = 2, PARTS_UU = 3;

template <int r, bool ONE = false>
__device__ __forceinline__ void vertex_part_f32(const VertexF& V, const DfGrids& G, int parts, bool right, int what,
                                                df w, df v, df vp, float2 out[16], bool accumulate = false) {
    const bool dir = parts & PARTS_UD, exch = parts & PARTS_X;
    if (!accumulate) {
#pragma unroll
        for (int o = 0; o < 16; ++o) out[o] = make_float2(0.f, 0.f);
    }
    // the bare part is even under a1 <-> a2, so its up-up value R(12) - R(21) is zero
    if ((what & 1) && V.has_R && dir != exch) {
        const float u = dir ? V.bare : -V.bare;
#pragma unroll
        for (int o = 0; o < 16; ++o) out[o].x += (__popc(o) & 1) ? u : 0.f;
    }
    int k_free = right ? 1 : 2, k_dep = right ? 2 : 1;
    unsigned own = 0;
    if (what & 2) own |= 1u << 0;
    if (what & 4) own |= 1u << k_free;
    if (what & 8) own |= 1u << k_dep;
    if (what & 16) own |= 1u << 3;
    if (!((V.mask >> r) & 1)) own = 0;
    bool cross = (what & 32) && isfinite(v.h) && isfinite(vp.h);
    constexpr int sr = (r == KB_CH_A) ? KB_CH_T : (r == KB_CH_T ? KB_CH_A : KB_CH_P);
    // lookup groups: 0 own direct, 1 own exchanged, 2/3 other channels direct,
    // 4/5 their exchanged partners
#pragma unroll 1
    for (int grp = 0; grp < 6; ++grp) {
        int ch;
        unsigned classes;
        float f = 1.f;
        bool sw = false;
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
            int c = (grp & 1) ? ((r == 2) ? 1 : 2) : ((r == 0) ? 1 : 0);   // the two channels != r
            if (!((V.mask >> c) & 1)) continue;
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
        Sten7 S = stencils7(V, ch, classes, G, gw, gv, gp);
        apply7<ONE>(V, ch, S, G, f, sw, out);
    }
}


// ------------------------------------------------------------------------------------
// Other channels' part of a vertex seen from channel r, by lookup group.
// ------------------------------------------------------------------------------------

// Channel read by lookup group g of channel r (compile time): g = 0, 1 the two channels
// c != r, direct; g = 2, 3 their exchanged partners (crossing partner a <-> t, p -> p).
template <int r, int g>
__host__ __device__ constexpr int group_channel() {
    return g < 2 ? ((g & 1) ? (r == KB_CH_T ? KB_CH_P : KB_CH_T) : (r == KB_CH_A ? KB_CH_P : KB_CH_A))
                 : ((g & 1) ? (r == KB_CH_T ? KB_CH_P : KB_CH_A)
                            : (r == KB_CH_A ? KB_CH_P : KB_CH_T));
}
// The channel c != r whose inclusion in the vertex decides group g.
template <int r, int g>
__host__ __device__ constexpr int group_source() {
    return (g & 1) ? (r == KB_CH_T ? KB_CH_P : KB_CH_T) : (r == KB_CH_A ? KB_CH_P : KB_CH_A);
}

// Component of the looked-up record that lands on component c under the exchange of the
// Keldysh indices a1 <-> a2 (bits 1 and 0 of c); an involution.
__host__ __device__ constexpr int kswap12(int c) { return (c & 12) | ((c & 1) << 1) | ((c >> 1) & 1); }

// ------------------------------------------------------------------------------------
// Corner lists: the interpolation of a lookup written out by the thread that found the
// stencil, read by the lanes that hold the record components.  Compact form: per class the
// record index of its first corner (the others follow at fixed offsets of the grid strides)
// and per corner its weight, so that a reading lane takes 4 bytes per corner plus 16 per
// lookup from shared memory.
// ------------------------------------------------------------------------------------

// The 18 corners of one channel's classes from its stencils, times f: base = record index of
// the first corner of K1 (kw1), K2 (kw2 N2v + kv2), K2' (kw2 N2v + kp2) and K3
// ((kw3 N3v + kv3) N3v + kp3); the weights in pairs whose second corner is the next record:
// wt[0] K1 (kw1, kw1 + 1); wt[1 + bw] K2 (bw, 0), (bw, 1); wt[3 + bw] K2' likewise;
// wt[5 + 2 bw + bv] K3 (bw, bv, 0), (bw, bv, 1).  Corner (bw, bv) of K2 is record
// base + bw N2v + bv, corner (bw, bv, bp) of K3 is base + bw N3v^2 + bv N3v + bp.  A corner
// outside its grid or of an absent class has weight 0 and is not read.
__device__ __forceinline__ void corner_weights18(const Sten7& S, const DfGrids& G, float f, int4* base, float2* wt,
                                                 int stride) {
    *base = make_int4(S.kw1, S.kw2 * G.N2v + S.kv2, S.kw2 * G.N2v + S.kp2, (S.kw3 * G.N3v + S.kv3) * G.N3v + S.kp3);
    auto lin = [](bool ok, float w) { return ok ? w : 0.f; };
    wt[0] = make_float2(lin(S.u0 && S.kw1 >= 0, f * (1.f - S.tw1)), lin(S.u0 && S.kw1 + 1 < G.N1, f * S.tw1));
#pragma unroll
    for (int bw = 0; bw < 2; ++bw) {
        const bool okw = bw ? S.kw2 + 1 < G.N2w : S.kw2 >= 0;
        const float fw = f * (bw ? S.tw2 : 1.f - S.tw2);
        wt[(1 + bw) * stride] = make_float2(lin(S.u1 && okw && S.kv2 >= 0, fw * (1.f - S.tv2)),
                                            lin(S.u1 && okw && S.kv2 + 1 < G.N2v, fw * S.tv2));
        wt[(3 + bw) * stride] = make_float2(lin(S.u2 && okw && S.kp2 >= 0, fw * (1.f - S.tp2)),
                                            lin(S.u2 && okw && S.kp2 + 1 < G.N2v, fw * S.tp2));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int bw = q >> 1, bv = q & 1;
        const bool ok = S.u3 && (bw ? S.kw3 + 1 < G.N3w : S.kw3 >= 0) && (bv ? S.kv3 + 1 < G.N3v : S.kv3 >= 0);
        const float fwv = f * (bw ? S.tw3 : 1.f - S.tw3) * (bv ? S.tv3 : 1.f - S.tv3);
        wt[(5 + q) * stride] = make_float2(lin(ok && S.kp3 >= 0, fwv * (1.f - S.tp3)),
                                           lin(ok && S.kp3 + 1 < G.N3v, fwv * S.tp3));
    }
}

__device__ __forceinline__ void no_corners18(int4* base, float2* wt, int stride) {
    *base = make_int4(0, 0, 0, 0);
#pragma unroll
    for (int i = 0; i < 9; ++i) wt[i * stride] = make_float2(0.f, 0.f);
}

// Corner list of lookup group g of the other channels' part seen from channel r at the
// r-variables (w, v, vp), with the group (and so the channel) known only at run time: one
// copy of the stencil code serves every group (four inlined copies measured slower, from
// instruction fetch), the class pointers are selected without indexing the parameter
// struct.  An exchanged group (g >= 2) carries the factor -1; its Keldysh index swap
// a1 <-> a2 is applied by the reader.
template <int r>
__device__ __forceinline__ void group_corners_rt(const VertexF& V, const DfGrids& Gr, int g, df w, df v, df vp,
                                                 int4* base, float2* wt, int stride) {
    const int c = (g & 1) ? ((r == KB_CH_T) ? KB_CH_P : KB_CH_T) : ((r == KB_CH_A) ? KB_CH_P : KB_CH_A);
    if (!((V.mask >> c) & 1)) { no_corners18(base, wt, stride); return; }
    df L[4];
    df_legs(r, w, v, vp, L);
    df gw, gv, gp;
    int ch = c;
    if (g < 2) {
        df_vars(c, L, gw, gv, gp);
    } else {
        ch = (c == KB_CH_A) ? KB_CH_T : (c == KB_CH_T ? KB_CH_A : KB_CH_P);
        df S4[4] = {L[0], L[1], L[3], L[2]};
        df_vars(ch, S4, gw, gv, gp);
    }
    corner_weights18(stencils7(V, ch, 15, Gr, gw, gv, gp), Gr, g < 2 ? 1.f : -1.f, base, wt, stride);
}

// Bosonic stencils of a lookup group, tabulated.  The other channels' transfer frequency
// seen from channel r is v + v'', v'' - v or v - v'' (Sec. II.C.1 parametrisations): it does
// not depend on the bosonic frequency w of channel r, so its three stencils (K1, K2 and K3
// bosonic grids) are found once per (group, v, node) and shared by every w.  Packed as
// (t on the K1 grid, t on the K2 grid, t on the K3 grid, bits) with bits = (k1 + 1) |
// (k2 + 1) << 11 | (k3 + 1) << 21, bit 31 set when the frequency is not finite; this needs
// N1 <= 2046 and N2w, N3w <= 1022.
constexpr int BSTEN_MAX_N1 = 2046, BSTEN_MAX_NW = 1022;

__device__ __forceinline__ Sten7 stencils7_tab(const VertexF& V, int ch, const DfGrids& G, float4 bt, df gv, df gp) {
    Sten7 S;
    const unsigned b = __float_as_uint(bt.w);
    const bool fw = !(b >> 31), fv = isfinite(gv.h), fp = isfinite(gp.h);
    const float ia = 1.f / G.A;
    const float xv = fv ? x_est(gv.h, ia) : 0.f, xp = fp ? x_est(gp.h, ia) : 0.f;
    S.u0 = vcls(V, ch, 0) && fw;
    S.u1 = vcls(V, ch, 1) && fw && fv;
    S.u2 = vcls(V, ch, 2) && fw && fp;
    S.u3 = vcls(V, ch, 3) && fw && fv && fp;
    S.tw1 = S.tw2 = S.tw3 = S.tv2 = S.tv3 = S.tp2 = S.tp3 = 0.f;
    S.kw1 = S.kw2 = S.kw3 = S.kv2 = S.kv3 = S.kp2 = S.kp3 = 0;
    if (S.u0) { S.kw1 = (int)(b & 2047u) - 1; S.tw1 = bt.x; }
    if (S.u1 || S.u2) { S.kw2 = (int)((b >> 11) & 1023u) - 1; S.tw2 = bt.y; }
    if (S.u1) S.kv2 = stencil_x(gv, xv, G.n2v, G.N2v, G.A, S.tv2);
    if (S.u2) S.kp2 = stencil_x(gp, xp, G.n2v, G.N2v, G.A, S.tp2);
    if (S.u3) {
        S.kw3 = (int)((b >> 21) & 1023u) - 1;
        S.tw3 = bt.z;
        S.kv3 = stencil_x(gv, xv, G.n3v, G.N3v, G.A, S.tv3);
        S.kp3 = stencil_x(gp, xp, G.n3v, G.N3v, G.A, S.tp3);
    }
    return S;
}

// Channel variables of lookup group g of channel r at the r-variables (w, v, vp): the
// channel read and its (w, v, vp); an exchanged group reads the crossing partner at the
// legs with v1 <-> v2 exchanged.
template <int r>
__device__ __forceinline__ int group_vars(int g, df w, df v, df vp, df& gw, df& gv, df& gp) {
    const int c = (g & 1) ? ((r == KB_CH_T) ? KB_CH_P : KB_CH_T) : ((r == KB_CH_A) ? KB_CH_P : KB_CH_A);
    df L[4];
    df_legs(r, w, v, vp, L);
    if (g < 2) {
        df_vars(c, L, gw, gv, gp);
        return c;
    }
    const int ch = (c == KB_CH_A) ? KB_CH_T : (c == KB_CH_T ? KB_CH_A : KB_CH_P);
    df S4[4] = {L[0], L[1], L[3], L[2]};
    df_vars(ch, S4, gw, gv, gp);
    return ch;
}

// group_corners_rt with the bosonic stencils taken from the table entry bt.
template <int r>
__device__ __forceinline__ void group_corners_tab(const VertexF& V, const DfGrids& Gr, int g, df w, df v, df vp,
                                                  float4 bt, int4* base, float2* wt, int stride) {
    const int c = (g & 1) ? ((r == KB_CH_T) ? KB_CH_P : KB_CH_T) : ((r == KB_CH_A) ? KB_CH_P : KB_CH_A);
    if (!((V.mask >> c) & 1)) { no_corners18(base, wt, stride); return; }
    df gw, gv, gp;
    const int ch = group_vars<r>(g, w, v, vp, gw, gv, gp);
    corner_weights18(stencils7_tab(V, ch, Gr, bt, gv, gp), Gr, g < 2 ? 1.f : -1.f, base, wt, stride);
}

// One pair of corners (records p and p + 1, record index i0 and i0 + 1 of a class of n
// records) of a lane group's gather: lane l reads the 16-byte piece l of each record with a
// nonzero weight (p already points at piece l).
__device__ __forceinline__ void corner_pair(const float4* p, float2 w, float2& a0, float2& a1, long long i0,
                                            long long n) {
    if (w.x != 0.f && kb_rec_ok(i0, n, KB_SITE_K2_GATHER)) {
        const float4 u = __ldg(p);
        a0 = __ffma2_rn(make_float2(w.x, w.x), make_float2(u.x, u.y), a0);
        a1 = __ffma2_rn(make_float2(w.x, w.x), make_float2(u.z, u.w), a1);
    }
    if (w.y != 0.f && kb_rec_ok(i0 + 1, n, KB_SITE_K2_GATHER)) {
        const float4 u = __ldg(p + 8);
        a0 = __ffma2_rn(make_float2(w.y, w.y), make_float2(u.x, u.y), a0);
        a1 = __ffma2_rn(make_float2(w.y, w.y), make_float2(u.z, u.w), a1);
    }
}

// Gather of one compact corner list by a group of 8 lanes: lane l accumulates components
// 2l, 2l+1 (one 16-byte piece of every corner record), acc += sum_k w_k rec_k[2l .. 2l+1],
// so that one warp-wide load delivers the full records of the 4 nodes its lane groups hold.
// With SPLIT the K1 and K2 corners accumulate into s0, s1 instead (the t channel reuses
// them for the exchanged p group, which has the same K1 and K2 corners); with SKIP12 they
// are left out (that exchanged group, whose caller adds them from the direct group).
template <int ch, bool SPLIT = false, bool SKIP12 = false>
__device__ __forceinline__ void gather_list(const VertexF& V, const DfGrids& G, const int4* __restrict__ base,
                                            const float2* __restrict__ wt, int stride, int l, float2& a0,
                                            float2& a1, float2* s0 = nullptr, float2* s1 = nullptr) {
    const int4 b = *base;
    float2 w[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) w[i] = wt[i * stride];
    const float4* c1 = reinterpret_cast<const float4*>(V.cls[ch][0]) + l;
    const float4* c2 = reinterpret_cast<const float4*>(V.cls[ch][1]) + l;
    const float4* c2p = reinterpret_cast<const float4*>(V.cls[ch][2]) + l;
    const float4* c3 = reinterpret_cast<const float4*>(V.cls[ch][3]) + l;
    const size_t s2 = (size_t)G.N2v * 8, s3 = (size_t)G.N3v * 8, s33 = (size_t)G.N3v * G.N3v * 8;
    const long long n1 = G.N1, n2 = (long long)G.N2w * G.N2v, n3 = (long long)G.N3w * G.N3v * G.N3v;
    const long long v2 = G.N2v, v3 = G.N3v, v33 = (long long)G.N3v * G.N3v;
    if (SPLIT) {
        corner_pair(c1 + (size_t)b.x * 8, w[0], *s0, *s1, b.x, n1);
        corner_pair(c2 + (size_t)b.y * 8, w[1], *s0, *s1, b.y, n2);
        corner_pair(c2 + (size_t)b.y * 8 + s2, w[2], *s0, *s1, b.y + v2, n2);
    } else if (!SKIP12) {
        corner_pair(c1 + (size_t)b.x * 8, w[0], a0, a1, b.x, n1);
        corner_pair(c2 + (size_t)b.y * 8, w[1], a0, a1, b.y, n2);
        corner_pair(c2 + (size_t)b.y * 8 + s2, w[2], a0, a1, b.y + v2, n2);
    }
    corner_pair(c2p + (size_t)b.z * 8, w[3], a0, a1, b.z, n2);
    corner_pair(c2p + (size_t)b.z * 8 + s2, w[4], a0, a1, b.z + v2, n2);
    const float4* p3 = c3 + (size_t)b.w * 8;
    corner_pair(p3, w[5], a0, a1, b.w, n3);
    corner_pair(p3 + s3, w[6], a0, a1, b.w + v3, n3);
    corner_pair(p3 + s33, w[7], a0, a1, b.w + v33, n3);
    corner_pair(p3 + s33 + s3, w[8], a0, a1, b.w + v33 + v3, n3);
}

// Host helpers of the mixed path (kb_mixed.cu) shared with its adjoint (kb_vjp.cu): the
// FP32 view of a slot (false, with the context's error set, unless every attached class is
// complex64 and 16-byte aligned), and the double-float node tables of the class grids and
// the quadrature written into tab (n1 + n2w + n2v + n3w + n3v + nq entries) with G pointing
// into them.
bool kb_slot_f32(kb_ctx* ctx, int slot, VertexF& F);
void kb_mixed_tables(kb_ctx* ctx, df* tab, DfGrids& G, cudaStream_t st);

}  // namespace kb
