// FP64 vertex evaluation and the forward tile kernels of the plain path, shared by the
// bubble (kb_fp64.cu) and its adjoint (kb_vjp.cu).  Everything here has internal linkage,
// so each translation unit holds its own copy (including the channel-map constants, which
// each unit uploads itself).
#pragma once
#include "kb_dev.cuh"

namespace kb {
namespace {

// ------------------------------------------------------------------------------------
// Vertex evaluation in FP64 (16 Keldysh components at once)
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double2 ld_c(const void* p, int dt, size_t i) {
    if (dt == KB_DT_C128) return reinterpret_cast<const double2*>(p)[i];
    float2 f = reinterpret_cast<const float2*>(p)[i];
    return make_double2(f.x, f.y);
}

// acc[o] += f * class(c, k)(w, v, vp)[src(o)], src(o) = o or o with (a1 <-> a2) when swap12
__device__ void acc_class_f64(const VertexDev& V, const Grids& G, int c, int k, double w, double v, double vp,
                              double f, bool swap12, double2 acc[16]) {
    const void* D = V.cls[c][k];
    if (!D) return;
    int dt = V.dt[c][k];
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
                if (!kb_rec_ok((long long)(base / 16), (long long)nw * (k == 0 ? 1 : nv) * (k == 3 ? nv : 1),
                               KB_SITE_FP64_REC))
                    continue;
                double g = f * fw * fv * fp;
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
}

// Part of Gamma (spin up-down, or up-up when uu) relative to channel r at r-variables
// (w, v, vp): zero part (R + K1_r + [K2'_r left | K2_r right]) or v-part
// ([K2_r left | K2'_r right] + K3_r + the other included channels at converted
// frequencies).  Up-up, channel by channel: gamma_c^uu(1'2'|12) = gamma_c^ud(1'2'|12) -
// gamma_{sigma(c)}^ud(1'2'|21) with sigma: a <-> t, p -> p; the exchanged own-channel term
// is read at (w, v, vp) -> (-w, v, vp) (a, t) or (w, v, -vp) (p).
__device__ void vertex_part_f64(const VertexDev& V, const Grids& G, int r, bool uu, bool right, bool nupart,
                                double w, double v, double vp, double2 out[16]) {
#pragma unroll
    for (int o = 0; o < 16; ++o) out[o] = make_double2(0, 0);
    if (!nupart && !uu && V.has_R) {
#pragma unroll
        for (int o = 0; o < 16; ++o) out[o].x = (__popc(o) & 1) ? V.bare : 0.0;
    }
    int k_free = right ? 1 : 2, k_dep = right ? 2 : 1;
    int ka = nupart ? k_dep : 0, kb2 = nupart ? 3 : k_free;
    if ((V.mask >> r) & 1) {
        int sr = (r == KB_CH_A) ? KB_CH_T : (r == KB_CH_T ? KB_CH_A : KB_CH_P);
        double xw = (r == KB_CH_P) ? w : -w, xvp = (r == KB_CH_P) ? -vp : vp;
        for (int q = 0; q < 2; ++q) {
            int k = q ? kb2 : ka;
            acc_class_f64(V, G, r, k, w, v, vp, 1.0, false, out);
            if (uu) acc_class_f64(V, G, sr, k, xw, v, xvp, -1.0, true, out);
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
            for (int k = 0; k < 4; ++k) acc_class_f64(V, G, c, k, wc, vc, pc, 1.0, false, out);
            if (uu) {
                int sc = (c == KB_CH_A) ? KB_CH_T : (c == KB_CH_T ? KB_CH_A : KB_CH_P);
                vars_of(sc, S, wc, vc, pc);
                for (int k = 0; k < 4; ++k) acc_class_f64(V, G, sc, k, wc, vc, pc, -1.0, true, out);
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Kernels
// ------------------------------------------------------------------------------------
struct ClassJob {
    int r, pi_kind, ns;          // channel, pair kind, spin terms (2 for t)
    int nq;
    int nw_chunk, w0;            // bosonic indices [w0, w0 + nw_chunk) of the class grid
    int nw_grid;                 // size of the class's bosonic grid
    int nL, nR;                  // external fermionic points of the left / right tile (1 = zero part)
    int nvL_grid, nvR_grid;      // grid sizes of those axes
    bool L_nu, R_nu;             // which part each side uses
};

__constant__ ChannelMaps c_maps[3];

__device__ __forceinline__ double grid_freq(int i, int n, double A) {
    return A * tan(0.5 * KB_PI * (-1.0 + 2.0 * (i + 1) / (double)(n + 1)));
}

// Pi[wl][j][16]
__global__ void k_pi_table(Model m, ClassJob J, double A, const double* __restrict__ xq,
                           const double* __restrict__ wq, double2* __restrict__ Pi) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int wl = blockIdx.y;
    if (j >= J.nq || wl >= J.nw_chunk) return;
    double w = grid_freq(J.w0 + wl, J.nw_grid, A);
    double2 e[16];
    pi_entry(m, c_maps[J.r], J.r, J.pi_kind, A, w, xq[j], wq[j], e);
    double2* o = Pi + ((size_t)wl * J.nq + j) * 16;
#pragma unroll
    for (int i = 0; i < 16; ++i) o[i] = e[i];
}

// One thread per (w, external v, s, j).  Writes the 4x4 block of the tile.
template <bool RIGHT>
__global__ void k_gather_f64(VertexDev V, Grids G, ClassJob J, const double* __restrict__ xq,
                             const double2* __restrict__ Pi, double2* __restrict__ tile) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int s = blockIdx.y % J.ns;
    int vi = blockIdx.y / J.ns;
    int wl = blockIdx.z;
    int nrow = RIGHT ? J.nR : J.nL;
    if (j >= J.nq || vi >= nrow) return;
    const ChannelMaps& M = c_maps[J.r];
    bool nupart = RIGHT ? J.R_nu : J.L_nu;
    int nvg = RIGHT ? J.nvR_grid : J.nvL_grid;
    double w = grid_freq(J.w0 + wl, J.nw_grid, G.A);
    double vext = nupart ? grid_freq(vi, nvg, G.A) : 0.0;
    double xj = xq[j];
    double vpp = (xj <= -1.0) ? -INFINITY : (xj >= 1.0 ? INFINITY : G.A * tan(0.5 * KB_PI * xj));
    // spin of this term: t channel left s=0 up-up, s=1 up-down; right s=0 up-down, s=1 up-up
    bool uu = (J.r == KB_CH_T) && (RIGHT ? (s == 1) : (s == 0));
    double2 g[16];
    if (RIGHT) vertex_part_f64(V, G, J.r, uu, true, nupart, w, vpp, vext, g);
    else vertex_part_f64(V, G, J.r, uu, false, nupart, w, vext, vpp, g);
    size_t K = (size_t)4 * J.ns * J.nq;
    size_t kcol = ((size_t)s * J.nq + j) * 4;
    size_t rowbase = ((size_t)wl * 4 * nrow + (size_t)vi * 4);
    if (!RIGHT) {
        for (int A = 0; A < 4; ++A) {
            double2* dst = tile + (rowbase + A) * K + kcol;
            for (int B = 0; B < 4; ++B) dst[B] = g[M.cL[A][B]];
        }
    } else {
        const double2* P = Pi + ((size_t)wl * J.nq + j) * 16;
        double2 pm[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) pm[i] = P[i];
        for (int C = 0; C < 4; ++C) {
            double2* dst = tile + (rowbase + C) * K + kcol;
            for (int B = 0; B < 4; ++B) {
                double2 acc = make_double2(0, 0);
#pragma unroll
                for (int D = 0; D < 4; ++D) cfma(acc, pm[4 * B + D], g[M.cR[D][C]]);
                dst[B] = acc;
            }
        }
    }
}

}  // namespace
}  // namespace kb
