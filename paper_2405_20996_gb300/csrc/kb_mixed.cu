// Mixed-precision path: propagators, Pi and the high-frequency tail in FP64; vertex gather
// in FP32 with double-float frequency arithmetic (kb_mixed.cuh); contractions with FP32
// products.  Per channel r:
//   k_mx_tables   double-float node tables of the class grids and the quadrature
//   k_mx_prep     per (w, node) on the K2 grid: N_s = Pi R0_s and M_s = L0_s Pi (4x4,
//                 FP64 then FP32); on the K3 grid: Pi in FP32 for folding the right tile
//   k_mx_k1       K1(w) = sum_j L0 Pi R0, one CTA per w
//   k_mx_sumj     column sums over j of N_s, M_s (for the v-independent own class)
//   k_mx_k2<R>    K2 (K2') = sum_j [v-part of Gamma1] N  (M [v'-part of Gamma2]), gather
//                 fused with the contraction, no tile in memory
//   k_mx_tile3<R> K3 tiles: left L[(v,A)][(s,j,B)], right R' = Pi R, as four FP32 planes
//                 (re hi, re lo, im hi, im lo; hi = TF32-rounded value, lo = remainder)
//   K3 contraction: tcgen05 3xTF32 (kb_tc.cu) or the SIMT reference k_mx_cgemm
//   k_mx_scatter3 out <- alpha B + beta out for K3
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "kb_mixed.cuh"

namespace kb {

// ------------------------------------------------------------------------------------
// tables
// ------------------------------------------------------------------------------------
__global__ void k_mx_tables(int n1, int n2w, int n2v, int n3w, int n3v, int nq, double A, const double* __restrict__ xq,
                            df* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int sizes[6] = {n1, n2w, n2v, n3w, n3v, nq};
    int off = 0;
    for (int g = 0; g < 6; ++g) {
        if (i < off + sizes[g]) {
            int k = i - off;
            double x = (g < 5) ? -1.0 + 2.0 * (k + 1) / (double)(sizes[g] + 1) : xq[k];
            df v;
            if (x <= -1.0) v = {-INFINITY, 0.f};
            else if (x >= 1.0) v = {INFINITY, 0.f};
            else v = df_make(A * tan(0.5 * KB_PI * x));
            out[i] = v;
            return;
        }
        off += sizes[g];
    }
}

struct MixedJob {
    int r, pi_kind, ns, nq;
    ChannelMaps M;
    double alpha, beta;
};

__device__ __forceinline__ double2 c64to128(float2 a) { return make_double2(a.x, a.y); }

// Zero part of a vertex as seen by the K1/K2 tables (own channel only, FP32 gather).
// left: R + K1_r + K2'_r(w, v''); right: R + K1_r + K2_r(w, v'').
template <int r>
__device__ __forceinline__ void zero_part(const VertexF& V, const DfGrids& G, bool uu, bool right, df w, df vpp,
                                          float2 out[16]) {
    df zero = {0.f, 0.f};
    const int parts = uu ? PARTS_UU : PARTS_UD;
    if (right) vertex_part_f32<r>(V, G, parts, true, 1 | 2 | 4, w, vpp, zero, out);
    else vertex_part_f32<r>(V, G, parts, false, 1 | 2 | 4, w, zero, vpp, out);
}

// Per (w in K2 grid, j): N_s = Pi R0_s, M_s = L0_s Pi;  Nt/Mt layout [w][s][j][16] float2.
// Right spin order s: 0 up-down, 1 up-up (t); left: 0 up-up, 1 up-down (t).
template <int R>
__global__ void __launch_bounds__(128) k_mx_prep_k2(VertexF VL, VertexF VR, DfGrids G, Model m, MixedJob J, const double* __restrict__ xq,
                             const double* __restrict__ wq, const df* __restrict__ wgrid, float2* __restrict__ Nt,
                             float2* __restrict__ Mt) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int wi = blockIdx.y;
    if (j >= J.nq) return;
    const df* qn = G.n3v + G.N3v;   // quadrature nodes follow the K3 fermionic grid in the table
    df w = wgrid[wi], vpp = qn[j];
    float2 Pf[16];
    {
        double2 Pi[16];
        pi_entry_t<R>(m, J.pi_kind, G.A, (double)w.h + (double)w.l, xq[j], wq[j], Pi,
                     (double)G.n3v[G.N3v + j].h + (double)G.n3v[G.N3v + j].l, true);
#pragma unroll
        for (int i = 0; i < 16; ++i) Pf[i] = make_float2((float)Pi[i].x, (float)Pi[i].y);
    }
    constexpr int NS = (R == KB_CH_T) ? 2 : 1;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        float2 R0[16], L0[16];
        bool uuR = (R == KB_CH_T) && s == 1, uuL = (R == KB_CH_T) && s == 0;
        zero_part<R>(VR, G, uuR, true, w, vpp, R0);
        zero_part<R>(VL, G, uuL, false, w, vpp, L0);
        float2* n = Nt + (((size_t)wi * J.ns + s) * J.nq + j) * 16;
        float2* mm = Mt + (((size_t)wi * J.ns + s) * J.nq + j) * 16;
#pragma unroll
        for (int X = 0; X < 4; ++X)
#pragma unroll
            for (int Y = 0; Y < 4; ++Y) {
                float2 an = make_float2(0.f, 0.f), am = make_float2(0.f, 0.f);
#pragma unroll
                for (int Z = 0; Z < 4; ++Z) {
                    cmac2(an, Pf[4 * X + Z], R0[cmap<R>(Z, Y)]);   // N[B=X][C=Y] = sum_D Pi[B][D] R0[D][C]
                    cmac2(am, L0[cmap<R>(X, Z)], Pf[4 * Z + Y]);   // M[A=X][D=Y] = sum_B L0[A][B] Pi[B][D]
                }
                n[4 * X + Y] = an;
                mm[4 * X + Y] = am;
            }
    }
}

// Pi on the K3 bosonic grid, FP64 -> FP32: Pt[w][j][16]
__global__ void k_mx_pi3(DfGrids G, Model m, MixedJob J, const double* __restrict__ xq, const double* __restrict__ wq,
                         float2* __restrict__ Pt) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int wi = blockIdx.y;
    if (j >= J.nq) return;
    df w = G.n3w[wi];
    double2 Pi[16];
    pi_entry(m, J.M, J.r, J.pi_kind, G.A, (double)w.h + (double)w.l, xq[j], wq[j], Pi,
                     (double)G.n3v[G.N3v + j].h + (double)G.n3v[G.N3v + j].l, true);
    float2* o = Pt + ((size_t)wi * J.nq + j) * 16;
#pragma unroll
    for (int i = 0; i < 16; ++i) o[i] = make_float2((float)Pi[i].x, (float)Pi[i].y);
}

// Block-wide sum of 16 complex numbers per thread into FP64 (result valid in thread 0).
template <int NT>
__device__ __forceinline__ void block_sum16(const float2 v[16], double2 res[16], double* sh) {
    // sh: NT/32 * 32 doubles
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 0; o < 16; ++o) {
        double x = v[o].x, y = v[o].y;
        for (int d = 16; d > 0; d >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, d);
            y += __shfl_xor_sync(0xffffffffu, y, d);
        }
        if (lane == 0) { sh[wid * 32 + 2 * o] = x; sh[wid * 32 + 2 * o + 1] = y; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int o = 0; o < 16; ++o) {
            double x = 0, y = 0;
            for (int wv = 0; wv < NT / 32; ++wv) { x += sh[wv * 32 + 2 * o]; y += sh[wv * 32 + 2 * o + 1]; }
            res[o] = make_double2(x, y);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void store_out(void* out, int dt, size_t e, double2 v, double alpha, double beta) {
    if (dt == KB_DT_C128) {
        double2* p = reinterpret_cast<double2*>(out) + e;
        double2 o = beta != 0.0 ? *p : make_double2(0, 0);
        *p = make_double2(alpha * v.x + beta * o.x, alpha * v.y + beta * o.y);
    } else {
        float2* p = reinterpret_cast<float2*>(out) + e;
        float2 o = beta != 0.0 ? *p : make_float2(0, 0);
        *p = make_float2((float)(alpha * v.x + beta * o.x), (float)(alpha * v.y + beta * o.y));
    }
}

// K1(w) = sum_j sum_s L0_s Pi R0_s.  Grid (w of the K1 grid, node slice): each CTA of 128
// threads sums its slice of the nodes and writes an FP64 partial; k_mx_k1_fin adds the
// slices in order and stores.
// half (p channel, a crossing-symmetric vertex bubbled with itself): the summand at -v'' is
// the one at v'' with both Keldysh pairs of the output exchanged (crossing exchanges the
// pairs of L0 and R0, and Pi_p(w, -v'') is Pi_p(w, v'') with its two lines exchanged), so
// only the nodes v'' >= 0 are summed, the centre node v'' = 0 at half weight, and
// k_mx_k1_fin adds the sum to its pair-exchanged image.
constexpr int K1_SLICES = 8;

template <int R>
__global__ void __launch_bounds__(128) k_mx_k1(VertexF VL, VertexF VR, DfGrids G, Model m, MixedJob J,
                                               const double* __restrict__ xq, const double* __restrict__ wq,
                                               double2* __restrict__ part, int w_off, int half) {
    __shared__ double sh[4 * 32];
    int wi = w_off + blockIdx.x, sl = blockIdx.y;
    const df* qn = G.n3v + G.N3v;
    df w = G.n1[wi];
    const int jlo = half ? (J.nq - 1) / 2 : 0;
    const int per = (J.nq - jlo + K1_SLICES - 1) / K1_SLICES;
    const int jb = jlo + sl * per, je = min(J.nq, jb + per);
    float2 acc[16];
    for (int o = 0; o < 16; ++o) acc[o] = make_float2(0, 0);
    for (int j = jb + threadIdx.x; j < je; j += blockDim.x) {
        float2 Pf[16];
        {
            double2 Pi[16];
            pi_entry_t<R>(m, J.pi_kind, G.A, (double)w.h + (double)w.l, xq[j], wq[j], Pi,
                     (double)G.n3v[G.N3v + j].h + (double)G.n3v[G.N3v + j].l, true);
            const double hw = (half && j == jlo) ? 0.5 : 1.0;
#pragma unroll
            for (int i = 0; i < 16; ++i) Pf[i] = make_float2((float)(hw * Pi[i].x), (float)(hw * Pi[i].y));
        }
        constexpr int NS = (R == KB_CH_T) ? 2 : 1;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            float2 R0[16], L0[16];
            zero_part<R>(VR, G, (R == KB_CH_T) && s == 1, true, w, qn[j], R0);
            zero_part<R>(VL, G, (R == KB_CH_T) && s == 0, false, w, qn[j], L0);
#pragma unroll
            for (int B = 0; B < 4; ++B)
#pragma unroll
                for (int C = 0; C < 4; ++C) {
                    float2 nf = make_float2(0.f, 0.f);
#pragma unroll
                    for (int D = 0; D < 4; ++D) cmac2(nf, Pf[4 * B + D], R0[cmap<R>(D, C)]);
#pragma unroll
                    for (int A = 0; A < 4; ++A) cmac2(acc[4 * A + C], L0[cmap<R>(A, B)], nf);
                }
        }
    }
    double2 res[16];
    block_sum16<128>(acc, res, sh);
    if (threadIdx.x == 0)
        for (int o = 0; o < 16; ++o) part[((size_t)blockIdx.x * K1_SLICES + sl) * 16 + o] = res[o];
}

__global__ void k_mx_k1_fin(MixedJob J, const double2* __restrict__ part, void* out, int odt, int w_off, int nw,
                            int half) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw * 16) return;
    int wl = i / 16, o = i % 16, A = o / 4, C = o % 4;
    double x = 0, y = 0;
    for (int sl = 0; sl < K1_SLICES; ++sl) {
        double2 p = part[((size_t)wl * K1_SLICES + sl) * 16 + o];
        x += p.x;
        y += p.y;
    }
    if (half) {
        // the image at -v'': rows and columns with the two indices of their pair exchanged
        const int oi = 4 * (((A & 1) << 1) | (A >> 1)) + (((C & 1) << 1) | (C >> 1));
        for (int sl = 0; sl < K1_SLICES; ++sl) {
            double2 p = part[((size_t)wl * K1_SLICES + sl) * 16 + oi];
            x += p.x;
            y += p.y;
        }
    }
    store_out(out, odt, (size_t)(w_off + wl) * 16 + J.M.cO[A][C], make_double2(x, y), J.alpha, J.beta);
}

// Column sums over j of the K2-grid tables: S[t][w][s][16], t = 0 (N) or 1 (M).
// Column sums over j of the K2-grid tables: S[t][w][s][16], t = 0 (N) or 1 (M).
__global__ void k_mx_sumj(const float2* __restrict__ Nt, const float2* __restrict__ Mt, int nq, int ns,
                          double2* __restrict__ S) {
    __shared__ double sh[4 * 32];
    int wi = blockIdx.x, s = blockIdx.y, t = blockIdx.z;
    const float2* T = (t == 0 ? Nt : Mt) + ((size_t)wi * ns + s) * nq * 16;
    float2 acc[16];
    for (int o = 0; o < 16; ++o) acc[o] = make_float2(0, 0);
    for (int j = threadIdx.x; j < nq; j += blockDim.x)
        for (int o = 0; o < 16; ++o) { acc[o].x += T[(size_t)j * 16 + o].x; acc[o].y += T[(size_t)j * 16 + o].y; }
    double2 res[16];
    block_sum16<128>(acc, res, sh);
    if (threadIdx.x == 0) {
        double2* o = S + (((size_t)t * gridDim.x + wi) * ns + s) * 16;
        for (int i = 0; i < 16; ++i) o[i] = res[i];
    }
}

// Node-weighted sums of a K2-grid table: Ntil[t][w][s][m][16] = sum_j phi_m(v''_j) T_t(w, s, j)
// over the interior nodes, phi_m the linear hat function of K3 grid node m in x (the same
// stencil as the gathers, so the weights agree exactly).  The own K3 class of a K2 record is
// K3_r(w, v, v'') with (w, v) fixed per output point, a function of v'' alone, so
//   sum_j K3_r(w, v, v''_j) T(w, j) = sum_m K3_r(w, v, X_m) Ntil(w, m):
// the own K3 lookups leave the node loop of k_mx_k2.  t = 0: N table (left), 1: M (right).
__device__ __forceinline__ int first_not_below(const df* __restrict__ qn, int lo, int hi, df x) {
    // first j in [lo, hi] with qn[j] >= x (hi + 1 if none); qn increasing
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        if (df_lt(qn[mid], x)) lo = mid + 1;
        else hi = mid - 1;
    }
    return lo;
}

// Stencil of every quadrature node on the K3 fermionic grid (lower node, fraction), the same
// for every w, spin and component of k_mx_ntilde.
__global__ void k_mx_nstencil(DfGrids G, int nq, int2* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq) return;
    const df* qn = G.n3v + G.N3v;
    float tt = 0.f;
    int k = -2;
    if (j > 0 && j < nq - 1) k = stencil_x(qn[j], x_est(qn[j].h, 1.f / G.A), G.n3v, G.N3v, G.A, tt);
    out[j] = make_int2(k, __float_as_int(tt));
}

__global__ void k_mx_ntilde(const float2* __restrict__ Nt, const float2* __restrict__ Mt, DfGrids G, int nq, int ns,
                            int t0, const int2* __restrict__ nst, double2* __restrict__ out) {
    // four threads per (grid node m, Keldysh component o) of one (w, s, table), each taking
    // every fourth node of m's range; their sums are added by shuffles (a warp holds one m)
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int wi = blockIdx.y, s = blockIdx.z % ns, t = t0 + blockIdx.z / ns;
    const int m = idx >> 6, o = (idx >> 2) & 15, q = idx & 3;
    if (m >= G.N3v) return;
    const float2* T = (t == 0 ? Nt : Mt) + ((size_t)wi * ns + s) * nq * 16 + o;
    const df* qn = G.n3v + G.N3v;
    // nodes whose stencil can touch grid node m lie between X_{m-1} and X_{m+1}
    int jl = (m == 0) ? 1 : first_not_below(qn, 1, nq - 2, G.n3v[m - 1]) - 1;
    int jh = (m == G.N3v - 1) ? nq - 2 : first_not_below(qn, 1, nq - 2, G.n3v[m + 1]);
    jl = max(jl, 1);
    jh = min(jh, nq - 2);
    double ax = 0.0, ay = 0.0;
    for (int j = jl + q; j <= jh; j += 4) {
        const int2 st = __ldg(nst + j);
        const int k = st.x;
        const float tt = __int_as_float(st.y);
        const float ph = (k == m) ? 1.f - tt : ((k + 1 == m) ? tt : 0.f);
        const float2 x = __ldg(T + (size_t)j * 16);
        ax = fma((double)ph, (double)x.x, ax);
        ay = fma((double)ph, (double)x.y, ay);
    }
    ax += __shfl_xor_sync(0xffffffffu, ax, 1);
    ay += __shfl_xor_sync(0xffffffffu, ay, 1);
    ax += __shfl_xor_sync(0xffffffffu, ax, 2);
    ay += __shfl_xor_sync(0xffffffffu, ay, 2);
    if (q == 0) out[((((size_t)t * G.N2w + wi) * ns + s) * G.N3v + m) * 16 + o] = make_double2(ax, ay);
}

// Loads of the propagator-vertex tables in the contraction: each element is used by one
// instruction (four lanes at once), so it is read without allocating in L1, which keeps L1
// for the vertex records the gathers reuse.
__device__ __forceinline__ float2 ld_stream(const float2* p) {
    float2 v;
    asm("ld.global.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

__device__ __forceinline__ float4 ld_stream4(const float4* p) {
    float4 v;
    asm("ld.global.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

// Record cache of a vertex for the K2 (RIGHT = false) or K2' (RIGHT = true) contraction of
// channel R: the records the node loop of k_mx_k2 gathers — the other channels' part of the
// vertex at (w, v, v''_j) (left) or (w, v''_j, v') (right), FP32 — for every (w, v) of the
// K2 grids and every interior node j = 1 .. nq-2.  Layout: the interior nodes of one (w, v)
// in blocks of 32 (the last one padded), and within a block node-minor:
//   float4 index ((((w N2v + v) nblk + b) NS + s) 8 + p) 32 + l,   node j = 1 + 32 b + l,
// p the 16-byte piece of the 16-component record and s the spin record of the t channel
// (up-down, then up-up), so that 32 lanes reading the same piece read 512 contiguous bytes.
__host__ __device__ constexpr int rc_blocks(int nq) { return (nq - 2 + 31) / 32; }

template <bool RIGHT, int R>
__global__ void __launch_bounds__(128) k_mx_cache_k2(VertexF V, DfGrids G, int nq, float2* __restrict__ cache) {
    constexpr int NS = (R == KB_CH_T) ? 2 : 1;
    const int wi = blockIdx.z, vi = blockIdx.y;
    const int jj = blockIdx.x * 128 + threadIdx.x;            // interior node index j - 1
    if (jj >= nq - 2) return;
    const int j = jj + 1, b = jj >> 5, l = jj & 31;
    const df* qn = G.n3v + G.N3v;
    const df w = G.n2w[wi], ve = G.n2v[vi];
    float2 g[16];
    if (RIGHT) vertex_part_f32<R>(V, G, PARTS_UD, true, 32, w, qn[j], ve, g);
    else vertex_part_f32<R>(V, G, PARTS_UD, false, 32, w, ve, qn[j], g);
    float4* dst = reinterpret_cast<float4*>(cache) +
                  ((((size_t)wi * G.N2v + vi) * rc_blocks(nq) + b) * NS) * 8 * 32 + l;
#pragma unroll
    for (int i = 0; i < 8; ++i) dst[i * 32] = make_float4(g[2 * i].x, g[2 * i].y, g[2 * i + 1].x, g[2 * i + 1].y);
    if (NS == 2) {
        if (RIGHT) vertex_part_f32<R>(V, G, PARTS_X, true, 32, w, qn[j], ve, g, true);
        else vertex_part_f32<R>(V, G, PARTS_X, false, 32, w, ve, qn[j], g, true);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            dst[(8 + i) * 32] = make_float4(g[2 * i].x, g[2 * i].y, g[2 * i + 1].x, g[2 * i + 1].y);
    }
}

// The rest of a K2 (K2') output point after the node loop, for a thread holding the partial
// sum acc of component (A, C) = (o >> 2, o & 3), o = tid & 15: the own K3 class through the
// node-weighted sums, the own v-dependent class times the node sums, the reduction over the
// 8 thread groups and the store.
template <bool RIGHT, int R>
__device__ __forceinline__ void k2_tail(const VertexF& V, const DfGrids& G, const MixedJob& J,
                                        const double2* __restrict__ Ssum, const double2* __restrict__ Ntil, void* out,
                                        int odt, int wi, int vi, df w, df ve, float2 acc,
                                        float2 (*rec)[128][17], float2 (*red)[16]) {
    constexpr int NS = (R == KB_CH_T) ? 2 : 1;
    // the work is done by the first 128 threads; a larger block (k_mx_k2's producer warps)
    // only joins the barriers
    const int tid = threadIdx.x, o = tid & 15, q = tid >> 4;
    const bool act = tid < 128;
    const int A = o >> 2, C = o & 3;
    // own K3 class through the node-weighted sums: records at the K3 grid nodes X_m,
    // [0] up-down (pairs with N_0 + N_1, or N_0 for a, p), [1] the exchanged term of the
    // t channel's up-up component (pairs with N_0 left, N_1 right)
    {
        const double2* Nb = Ntil + (((size_t)(RIGHT ? 1 : 0) * G.N2w + wi) * NS) * G.N3v * 16;
#pragma unroll 1
        for (int m0 = 0; m0 < G.N3v; m0 += 128) {
            const int m = m0 + tid;
            if (act && m < G.N3v) {
                float2 g[16];
                if (RIGHT) vertex_part_f32<R>(V, G, PARTS_UD, true, 16, w, G.n3v[m], ve, g);
                else vertex_part_f32<R>(V, G, PARTS_UD, false, 16, w, ve, G.n3v[m], g);
#pragma unroll
                for (int c = 0; c < 16; ++c) rec[0][tid][c] = g[c];
                if (NS == 2) {
                    if (RIGHT) vertex_part_f32<R>(V, G, PARTS_X, true, 16, w, G.n3v[m], ve, g);
                    else vertex_part_f32<R>(V, G, PARTS_X, false, 16, w, ve, G.n3v[m], g);
#pragma unroll
                    for (int c = 0; c < 16; ++c) rec[NS - 1][tid][c] = g[c];
                }
            }
            __syncthreads();
            const int nrec = min(128, G.N3v - m0);
#pragma unroll 1
            for (int rr = q; act && rr < nrec; rr += 8) {
                const double2* n0 = Nb + (size_t)(m0 + rr) * 16;
                const double2* n1 = n0 + (size_t)G.N3v * 16;
                if (!RIGHT) {
#pragma unroll
                    for (int B = 0; B < 4; ++B) {
                        double2 a = n0[4 * B + C];
                        if (NS == 2) {
                            double2 b = n1[4 * B + C];
                            cmac2(acc, rec[0][rr][cmap<R>(A, B)], make_float2((float)(a.x + b.x), (float)(a.y + b.y)));
                            cmac2(acc, rec[NS - 1][rr][cmap<R>(A, B)], make_float2((float)a.x, (float)a.y));
                        } else {
                            cmac2(acc, rec[0][rr][cmap<R>(A, B)], make_float2((float)a.x, (float)a.y));
                        }
                    }
                } else {
#pragma unroll
                    for (int D = 0; D < 4; ++D) {
                        double2 a = n0[4 * A + D];
                        if (NS == 2) {
                            double2 b = n1[4 * A + D];
                            cmac2(acc, make_float2((float)(a.x + b.x), (float)(a.y + b.y)), rec[0][rr][cmap<R>(D, C)]);
                            cmac2(acc, make_float2((float)b.x, (float)b.y), rec[NS - 1][rr][cmap<R>(D, C)]);
                        } else {
                            cmac2(acc, make_float2((float)a.x, (float)a.y), rec[0][rr][cmap<R>(D, C)]);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    // own ext-dependent class: own(w, v) * sum_j N(w, j) (or sum_j M(w, j) * own(w, v'))
    if (q == 0) {
        df zero = {0.f, 0.f};
        float2 g[16];
#pragma unroll 1
        for (int s = 0; s < NS; ++s) {
            // s = 0: up-down on both sides for a, p; for t the up-down record (left s = 1,
            // right s = 0) comes first, then the exchanged term turns it into up-up
            const int parts = (s == 0) ? PARTS_UD : PARTS_X;
            if (RIGHT) vertex_part_f32<R>(V, G, parts, true, 8, w, zero, ve, g, s > 0);
            else vertex_part_f32<R>(V, G, parts, false, 8, w, ve, zero, g, s > 0);
            const int st = (NS == 1) ? 0 : (RIGHT ? s : 1 - s);
            const double2* S = Ssum + (((size_t)(RIGHT ? 1 : 0) * G.N2w + wi) * NS + st) * 16;
#pragma unroll
            for (int B = 0; B < 4; ++B) {
                if (!RIGHT) {
                    double2 sv = S[4 * B + C];
                    cmac2(acc, g[cmap<R>(A, B)], make_float2((float)sv.x, (float)sv.y));
                } else {
                    double2 sv = S[4 * A + B];
                    cmac2(acc, make_float2((float)sv.x, (float)sv.y), g[cmap<R>(B, C)]);
                }
            }
        }
    }
    if (act) red[q][o] = acc;
    __syncthreads();
    if (q == 0) {
        double re = 0, im = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) { re += red[k][o].x; im += red[k][o].y; }
        store_out(out, odt, ((size_t)wi * G.N2v + vi) * 16 + cmap<R>(A, C), make_double2(re, im), J.alpha, J.beta);
    }
}

// Bosonic stencils of the K2 gather's lookup groups per (group, v of the K2 grid, node):
// tab[(g * N2v + v) * nq + j] (see stencils7_tab); left side (K2) with (v, v'') = (v, node),
// right side (K2') with (node, v).  The transfer frequencies do not depend on w, which is set
// to 0 here.
template <bool RIGHT, int R>
__global__ void k_mx_bsten(DfGrids G, int nq, float4* __restrict__ tab) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, vi = blockIdx.y, g = blockIdx.z;
    if (j >= nq) return;
    const df* qn = G.n3v + G.N3v;
    const df zero = {0.f, 0.f};
    df gw, gv, gp;
    if (RIGHT) group_vars<R>(g, zero, qn[j], G.n2v[vi], gw, gv, gp);
    else group_vars<R>(g, zero, G.n2v[vi], qn[j], gw, gv, gp);
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned bits = 1u << 31;
    if (isfinite(gw.h)) {
        const float xw = x_est(gw.h, 1.f / G.A);
        const int k1 = stencil_x(gw, xw, G.n1, G.N1, G.A, o.x);
        const int k2 = stencil_x(gw, xw, G.n2w, G.N2w, G.A, o.y);
        const int k3 = stencil_x(gw, xw, G.n3w, G.N3w, G.A, o.z);
        bits = (unsigned)(k1 + 1) | ((unsigned)(k2 + 1) << 11) | ((unsigned)(k3 + 1) << 21);
    }
    o.w = __uint_as_float(bits);
    tab[((size_t)g * G.N2v + vi) * nq + j] = o;
}

// K2 (RIGHT = false): out(w, v)[A][C] = sum_j sum_s sum_B L_s(w, v, v''_j)[A][B] N_s(w, j)[B][C]
//   with L the v-dependent part of Gamma1 without its own K2 class, plus
//   K2own_s(w, v)[A][B] * SN_s(w)[B][C]  (the own K2 class does not depend on v'').
// K2' (RIGHT = true): out(w, v')[A][C] = sum_j sum_s sum_D M_s(w, j)[A][D] R_s(w, v''_j, v')[D][C]
//   + SM_s(w)[A][D] * K2'own_s(w, v')[D][C].
// One CTA per (w, v) with two warp roles working on chunks of CH = 128 / NG interior nodes
// (NG lookup groups: the two other channels, and for t their exchanged partners), the
// chunks' shared-memory buffers double-buffered so that the roles overlap:
//   producers (K2_PROD threads, warps 4-7), one chunk ahead: the corner lists, one
//      (node, group) item at a time — the stencils of the group's classes (the bosonic ones
//      from the k_mx_bsten table), its 18 corner weights and 4 class base records (a
//      reading lane then takes 4 bytes per corner) — and the chunk's rows of the
//      propagator-vertex table (t: combined per spin record);
//   consumers (K2_CONS threads, warps 0-3): 8 lanes per node, lane l reading the 16-byte
//      piece l (components 2l, 2l+1) of every corner record, so one warp-wide load covers the
//      full records of 4 nodes and each quarter-warp reads one 128-byte line (the L1 delivers
//      one line per quarter-warp and cycle, so this is the fewest wavefronts a corner can
//      cost); each lane multiplies its two interpolated components into the table rows they
//      meet and keeps 8 partial outputs across all nodes.
// Hand-over through named barriers: FULL(b) (producers arrive, consumers wait) and EMPTY(b)
// (consumers arrive, producers wait), each generation completed by all K2_THREADS threads.
// The corner lists are latency-bound ALU work and the gather is bound by the L1 data stage,
// so the two overlap instead of alternating.  Then the partials are reduced over lanes and
// warps into the (A, C)-per-thread layout of k2_tail, which adds the own classes and stores.
// The endpoint nodes contribute only through the own class and are not gathered.  (Reading
// each record once for a run of neighbouring nodes, by one thread or by a lane group, cut the
// L1 traffic but cost more instructions than it saved, measured on the a channel.)
constexpr int K2_CONS = 128, K2_PROD = 128, K2_THREADS = K2_CONS + K2_PROD;
constexpr int K2_BAR_FULL = 1, K2_BAR_EMPTY = 3;    // named barriers 1, 2 and 3, 4

// named barrier ID0 + b (b = 0 or 1) with all K2_THREADS threads taking part; the IDs are
// immediates so that the kernel reserves only the barriers it uses
template <int ID0>
__device__ __forceinline__ void nbar_sync(int b) {
    if (b) asm volatile("bar.sync %0, %1;" ::"n"(ID0 + 1), "n"(K2_THREADS) : "memory");
    else asm volatile("bar.sync %0, %1;" ::"n"(ID0), "n"(K2_THREADS) : "memory");
}
template <int ID0>
__device__ __forceinline__ void nbar_arrive(int b) {
    if (b) asm volatile("bar.arrive %0, %1;" ::"n"(ID0 + 1), "n"(K2_THREADS) : "memory");
    else asm volatile("bar.arrive %0, %1;" ::"n"(ID0), "n"(K2_THREADS) : "memory");
}

// one chunk buffer: class bases int4[NG][CH], weights float2[NG][9][CH], table rows
// float4[NS][CH][9]
template <int R>
__host__ __device__ constexpr size_t k2_buf_bytes() {
    constexpr int NS = (R == KB_CH_T) ? 2 : 1;
    constexpr int CH = 128 / (2 * NS);
    return (size_t)2 * NS * CH * (sizeof(int4) + 9 * sizeof(float2)) + (size_t)NS * CH * 9 * sizeof(float4);
}
template <int R>
__host__ __device__ constexpr size_t k2_smem_bytes() {
    constexpr int NS = (R == KB_CH_T) ? 2 : 1;
    constexpr size_t loop = 2 * k2_buf_bytes<R>();
    constexpr size_t tail = (size_t)NS * 128 * 17 * sizeof(float2);
    return loop > tail ? loop : tail;
}

template <bool RIGHT, int R>
__global__ void __launch_bounds__(K2_THREADS, 3) k_mx_k2(VertexF V, DfGrids G, MixedJob J, const float2* __restrict__ Tab,
                                                      const double2* __restrict__ Ssum, const double2* __restrict__ Ntil,
                                                      void* out, int odt, int w_off, int v_off,
                                                      const float4* __restrict__ bst) {
    constexpr int NS = (R == KB_CH_T) ? 2 : 1;
    constexpr int NG = 2 * NS;
    constexpr int CH = 128 / NG;
    constexpr size_t BUF = k2_buf_bytes<R>();
    constexpr size_t BASE_BYTES = (size_t)NG * CH * sizeof(int4);
    constexpr size_t CL_BYTES = BASE_BYTES + (size_t)NG * 9 * CH * sizeof(float2);
    extern __shared__ __align__(16) unsigned char k2_smem[];
    __shared__ float2 red[8][16];
    const int wi = w_off + blockIdx.y, vi = v_off + blockIdx.x;
    const df* qn = G.n3v + G.N3v;
    const df w = G.n2w[wi], ve = G.n2v[vi];
    const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31, gi = lane >> 3, l = lane & 7;
    const int nch = (J.nq - 2 + CH - 1) / CH;          // chunks of the interior nodes 1 .. nq-2
    // partial outputs of a consumer lane: left o[e][C] belongs to out[X_e][C], right o[e][A]
    // to out[A][Y_e]
    float2 o[2][4];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int c = 0; c < 4; ++c) o[e][c] = make_float2(0.f, 0.f);
    if (tid >= K2_CONS) {
        // producers: corner lists and table rows of chunk c into buffer c & 1
        const int pt = tid - K2_CONS;
        const float2* T0 = Tab + ((size_t)wi * NS) * J.nq * 16;
        const float2* T1 = T0 + (size_t)J.nq * 16;
#pragma unroll 1
        for (int c = 0; c < nch; ++c) {
            const int b = c & 1, j0 = 1 + c * CH;
            if (c >= 2) nbar_sync<K2_BAR_EMPTY>(b);                 // chunk c - 2 consumed
            unsigned char* buf = k2_smem + b * BUF;
            int4* cb = reinterpret_cast<int4*>(buf);                      // [g][n] class bases
            float2* cw = reinterpret_cast<float2*>(buf + BASE_BYTES);     // [g][pair][n] weights
            float4* trow = reinterpret_cast<float4*>(buf + CL_BYTES);     // [s][n][9]
            // (node, group) items; a warp's items share g
#pragma unroll 1
            for (int it = pt; it < NG * CH; it += K2_PROD) {
                const int n = it % CH, g = it / CH, j = j0 + n;
                int4* bd = cb + g * CH + n;
                float2* wd = cw + (size_t)g * 9 * CH + n;
                if (j < J.nq - 1 && bst) {
                    const float4 bt = bst[((size_t)g * G.N2v + vi) * J.nq + j];
                    if (RIGHT) group_corners_tab<R>(V, G, g, w, qn[j], ve, bt, bd, wd, CH);
                    else group_corners_tab<R>(V, G, g, w, ve, qn[j], bt, bd, wd, CH);
                } else if (j < J.nq - 1) {
                    if (RIGHT) group_corners_rt<R>(V, G, g, w, qn[j], ve, bd, wd, CH);
                    else group_corners_rt<R>(V, G, g, w, ve, qn[j], bd, wd, CH);
                } else {
                    no_corners18(bd, wd, CH);
                }
            }
            // table rows; t: left (T0 + T1, T0) pairs with (up-down, exchanged term) since
            // up-up = up-down + exchanged term and the sum is uu T0 + ud T1; right (T0 + T1, T1)
#pragma unroll 1
            for (int it = pt; it < CH * 8; it += K2_PROD) {
                const int n = it >> 3, piece = it & 7, j = j0 + n;
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f), bb = a;
                if (j < J.nq - 1) {
                    a = ld_stream4(reinterpret_cast<const float4*>(T0 + (size_t)j * 16) + piece);
                    if (NS == 2) bb = ld_stream4(reinterpret_cast<const float4*>(T1 + (size_t)j * 16) + piece);
                }
                if (NS == 1) {
                    trow[n * 9 + piece] = a;
                } else {
                    trow[n * 9 + piece] = make_float4(a.x + bb.x, a.y + bb.y, a.z + bb.z, a.w + bb.w);
                    trow[(CH + n) * 9 + piece] = RIGHT ? bb : a;
                }
            }
            nbar_arrive<K2_BAR_FULL>(b);                                // chunk c ready
        }
        // the consumers' releases of the last two chunks, so that every barrier generation
        // is completed
#pragma unroll 1
        for (int c = nch >= 2 ? nch - 2 : 0; c < nch; ++c) nbar_sync<K2_BAR_EMPTY>(c & 1);
    } else {
        // consumers: this lane's record components 2l + e as matrix entries (X_e, Y_e) of
        // channel R's map
        int Xe[2], Ye[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            int xy = 0;
            for (int q = 0; q < 16; ++q)
                if (cmap<R>(q >> 2, q & 3) == 2 * l + e) xy = q;
            Xe[e] = xy >> 2;
            Ye[e] = xy & 3;
        }
#pragma unroll 1
        for (int c = 0; c < nch; ++c) {
            const int b = c & 1;
            nbar_sync<K2_BAR_FULL>(b);                                  // chunk c ready
            const unsigned char* buf = k2_smem + b * BUF;
            const int4* cb = reinterpret_cast<const int4*>(buf);
            const float2* cw = reinterpret_cast<const float2*>(buf + BASE_BYTES);
            const float4* trow = reinterpret_cast<const float4*>(buf + CL_BYTES);
            // gather and contraction, 4 nodes per warp at a time
#pragma unroll 1
            for (int n = wp * 4 + gi; n < CH; n += 16) {
                float2 d0 = make_float2(0.f, 0.f), d1 = d0, x0 = d0, x1 = d0;
                gather_list<group_channel<R, 0>()>(V, G, cb + n, cw + n, CH, l, d0, d1);
                if (NS == 2) {
                    // t: group 3, the exchanged partner of group 1 (p at the legs with 1 and 2
                    // exchanged: the same w_p and v_p, v'_p negated), has group 1's K1 and K2
                    // corners with weights of opposite sign, so they are read once: group 1's
                    // K1 + K2 sum s is added to d and subtracted from the exchanged groups'
                    // sum y.  The exchanged groups are read like the direct ones (lane l holds
                    // components 2l, 2l+1 of the sum), and the exchanged term x = kswap12(y - s)
                    // (components 4m + 1 and 4m + 2 exchanged) is formed by one lane-pair
                    // shuffle: lanes l and l ^ 1 hold 4m, 4m+1 and 4m+2, 4m+3
                    float2 s0 = make_float2(0.f, 0.f), s1 = s0, y0 = s0, y1 = s0;
                    gather_list<group_channel<R, 1>(), true>(V, G, cb + CH + n, cw + 9 * CH + n, CH, l, d0, d1,
                                                             &s0, &s1);
                    d0 = make_float2(d0.x + s0.x, d0.y + s0.y);
                    d1 = make_float2(d1.x + s1.x, d1.y + s1.y);
                    gather_list<group_channel<R, 2>()>(V, G, cb + 2 * CH + n, cw + 2 * 9 * CH + n, CH, l, y0, y1);
                    gather_list<group_channel<R, 3>(), false, true>(V, G, cb + 3 * CH + n, cw + 3 * 9 * CH + n, CH,
                                                                    l, y0, y1);
                    y0 = make_float2(y0.x - s0.x, y0.y - s0.y);
                    y1 = make_float2(y1.x - s1.x, y1.y - s1.y);
                    const bool odd = l & 1;
                    const float2 send = odd ? y0 : y1;
                    const float2 recv = make_float2(__shfl_xor_sync(0xffffffffu, send.x, 1),
                                                    __shfl_xor_sync(0xffffffffu, send.y, 1));
                    x0 = odd ? recv : y0;
                    x1 = odd ? y1 : recv;
                } else {
                    gather_list<group_channel<R, 1>()>(V, G, cb + CH + n, cw + 9 * CH + n, CH, l, d0, d1);
                }
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const float2 dv = e ? d1 : d0, xv = e ? x1 : x0;
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        const float4* tr = trow + (s * CH + n) * 9;
                        const float2 rv = s == 0 ? dv : xv;
                        if (!RIGHT) {
                            // row Y_e of the table: components 4 Y_e .. 4 Y_e + 3
                            const float4 p0 = tr[2 * Ye[e]], p1 = tr[2 * Ye[e] + 1];
                            cmac2(o[e][0], rv, make_float2(p0.x, p0.y));
                            cmac2(o[e][1], rv, make_float2(p0.z, p0.w));
                            cmac2(o[e][2], rv, make_float2(p1.x, p1.y));
                            cmac2(o[e][3], rv, make_float2(p1.z, p1.w));
                        } else {
                            // column X_e of the table: components 4 A + X_e
#pragma unroll
                            for (int A = 0; A < 4; ++A) {
                                const float4 p = tr[2 * A + (Xe[e] >> 1)];
                                cmac2(o[e][A], (Xe[e] & 1) ? make_float2(p.z, p.w) : make_float2(p.x, p.y), rv);
                            }
                        }
                    }
                }
            }
            nbar_arrive<K2_BAR_EMPTY>(b);                               // chunk c consumed
        }
        // sum over the four node groups of a warp
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float2 v = o[e][c];
                v.x += __shfl_xor_sync(0xffffffffu, v.x, 8);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, 8);
                v.x += __shfl_xor_sync(0xffffffffu, v.x, 16);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, 16);
                o[e][c] = v;
            }
    }
    __syncthreads();                                                    // every buffer is free
    // sum over the lanes and warps that hold parts of the same output
    float2* part = reinterpret_cast<float2*>(k2_smem);                   // [warp][l][e][4]
    if (tid < K2_CONS && gi == 0) {
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int c = 0; c < 4; ++c) part[((wp * 8 + l) * 2 + e) * 4 + c] = o[e][c];
    }
    __syncthreads();
    float2 acc = make_float2(0.f, 0.f);
    if (tid < 16) {
        const int A = tid >> 2, C = tid & 3;
        for (int ll = 0; ll < 8; ++ll)
            for (int e = 0; e < 2; ++e) {
                int xy = 0;
                for (int q = 0; q < 16; ++q)
                    if (cmap<R>(q >> 2, q & 3) == 2 * ll + e) xy = q;
                const bool mine = RIGHT ? ((xy & 3) == C) : ((xy >> 2) == A);
                if (!mine) continue;
                const int c = RIGHT ? A : C;
                for (int ww = 0; ww < 4; ++ww) {
                    const float2 v = part[((ww * 8 + ll) * 2 + e) * 4 + c];
                    acc.x += v.x;
                    acc.y += v.y;
                }
            }
    }
    __syncthreads();
    k2_tail<RIGHT, R>(V, G, J, Ssum, Ntil, out, odt, wi, vi, w, ve, acc,
                      reinterpret_cast<float2 (*)[128][17]>(k2_smem), red);
}

// K2 / K2' from the record cache (k_mx_cache_k2): the same sums as k_mx_k2, with each
// thread taking whole records — its node's 16-component record(s), read from the cache's
// node-minor blocks (a warp's 16-byte loads cover 512 contiguous bytes), and its node's
// propagator-vertex table row, which the warp loads coalesced into padded shared memory —
// and all 16 outputs of a record in registers (64 complex MACs per record).  The 128 partial
// outputs are then reduced into the (A, C)-per-thread layout of k2_tail.
template <bool RIGHT, int R>
__global__ void __launch_bounds__(128, 4) k_mx_k2_rc(VertexF V, DfGrids G, MixedJob J, const float2* __restrict__ Tab,
                                                  const double2* __restrict__ Ssum, const double2* __restrict__ Ntil,
                                                  void* out, int odt, int w_off, int v_off,
                                                  const float2* __restrict__ cache) {
    constexpr int NS = (R == KB_CH_T) ? 2 : 1;
    // the node loop stages table rows (per warp 32 rows, 16 bytes padding) in the memory that
    // holds the partial sums and the tail's records afterwards
    constexpr size_t REC_BYTES = (size_t)NS * 128 * 17 * sizeof(float2), ROW_BYTES = 4 * 32 * 9 * sizeof(float4);
    __shared__ __align__(16) unsigned char sm_raw[REC_BYTES > ROW_BYTES ? REC_BYTES : ROW_BYTES];
    __shared__ float2 red[8][16];
    float2 (*rec)[128][17] = reinterpret_cast<float2 (*)[128][17]>(sm_raw);
    float4 (*trow)[32][9] = reinterpret_cast<float4 (*)[32][9]>(sm_raw);
    const int wi = w_off + blockIdx.y, vi = v_off + blockIdx.x;
    const df w = G.n2w[wi], ve = G.n2v[vi];
    const int tid = threadIdx.x, wp = tid >> 5, ln = tid & 31;
    const int nblk = rc_blocks(J.nq);
    const float2* T0 = Tab + ((size_t)wi * NS) * J.nq * 16;
    const float2* T1 = T0 + (size_t)J.nq * 16;
    const float4* base = reinterpret_cast<const float4*>(cache) + ((size_t)wi * G.N2v + vi) * nblk * NS * 8 * 32;
    float2 o16[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o16[c] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int b = wp; b < nblk; b += 4) {                // warp-uniform loop over node blocks
        const int j = 1 + 32 * b + ln;
        const bool valid = j < J.nq - 1;
#pragma unroll
        for (int pass = 0; pass < NS; ++pass) {
            // pass 0 pairs table 0 with the up-down record (right) or the up-up one (left of t);
            // pass 1 table 1 with the other spin record
            const int srec = (NS == 1) ? 0 : (RIGHT ? pass : 1 - pass);
            const float2* Tt = pass == 0 ? T0 : T1;
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int idx = q * 32 + ln, n = idx >> 3, piece = idx & 7;
                const int jn = min(1 + 32 * b + n, J.nq - 1);
                trow[wp][n][piece] = ld_stream4(reinterpret_cast<const float4*>(Tt + (size_t)jn * 16) + piece);
            }
            __syncwarp();
            float2 rv[16], tv[16];
            const float4* rp = base + ((size_t)b * NS + srec) * 8 * 32 + ln;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float4 u = ld_stream4(rp + i * 32);
                if (!valid) u = make_float4(0.f, 0.f, 0.f, 0.f);
                rv[2 * i] = make_float2(u.x, u.y);
                rv[2 * i + 1] = make_float2(u.z, u.w);
                const float4 t = trow[wp][ln][i];
                tv[2 * i] = make_float2(t.x, t.y);
                tv[2 * i + 1] = make_float2(t.z, t.w);
            }
#pragma unroll
            for (int A = 0; A < 4; ++A)
#pragma unroll
                for (int C = 0; C < 4; ++C)
#pragma unroll
                    for (int B = 0; B < 4; ++B) {
                        if (!RIGHT) cmac2(o16[4 * A + C], rv[cmap<R>(A, B)], tv[4 * B + C]);
                        else cmac2(o16[4 * A + C], tv[4 * A + B], rv[cmap<R>(B, C)]);
                    }
        }
    }
    // partials of the 128 threads -> thread (q, o) sums those of threads q, q + 8, ...
    __syncthreads();                                   // every warp is done with its table rows
#pragma unroll
    for (int c = 0; c < 16; ++c) rec[0][tid][c] = o16[c];
    __syncthreads();
    const int o = tid & 15, q = tid >> 4;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float2 v = rec[0][q + 8 * i][o];
        acc.x += v.x;
        acc.y += v.y;
    }
    __syncthreads();
    k2_tail<RIGHT, R>(V, G, J, Ssum, Ntil, out, odt, wi, vi, w, ve, acc, rec, red);
}

// TF32 split of an FP32 value: hi rounded to the 10-bit TF32 mantissa, lo = x - hi
// (exact in FP32).
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    hi = __uint_as_float(u);
    lo = x - hi;
}

// K3 tiles.  Left: row (v, A), col k = (s*nq + j)*4 + B, value Gamma1_s^{cL[A][B]}(w, v, v''_j)
// (v-dependent part incl. the own K2 class).  Right: row (v', C), same k, value
// sum_D Pi[B][D] Gamma2_s^{cR[D][C]}(w, v''_j, v').  Four planes per tile:
// [plane][row][k], plane = 2*(re 0 / im 1) + (hi 0 / lo 1), each plane rows x K floats.
// Keldysh component permutations of the symmetry images (c = 8 b1' + 4 b2' + 2 b1 + b2):
// conjugation (a1'a2'|a1a2) -> (a1a2|a1'a2'); crossing -> (a2'a1'|a2a1); the conjugation sign
// is (-1)^(1 + number of quantum indices + 4).
__host__ __device__ constexpr int perm_c(int c) { return ((c & 3) << 2) | (c >> 2); }
__host__ __device__ constexpr int perm_x(int c) {
    return (((c >> 2) & 1) << 3) | (((c >> 3) & 1) << 2) | ((c & 1) << 1) | ((c >> 1) & 1);
}
__host__ __device__ constexpr int popc4c(int c) { return (c & 1) + ((c >> 1) & 1) + ((c >> 2) & 1) + ((c >> 3) & 1); }
__host__ __device__ constexpr float sign_c(int c) { return (popc4c(c) & 1) ? 1.f : -1.f; }

__device__ __forceinline__ void write_planes(float* base, size_t plane, size_t row, size_t K, size_t col,
                                             const float2 v[4]) {
    float4 rh, rl, ih, il;
    tf32_split(v[0].x, rh.x, rl.x); tf32_split(v[1].x, rh.y, rl.y);
    tf32_split(v[2].x, rh.z, rl.z); tf32_split(v[3].x, rh.w, rl.w);
    tf32_split(v[0].y, ih.x, il.x); tf32_split(v[1].y, ih.y, il.y);
    tf32_split(v[2].y, ih.z, il.z); tf32_split(v[3].y, ih.w, il.w);
    *reinterpret_cast<float4*>(base + 0 * plane + row * K + col) = rh;
    *reinterpret_cast<float4*>(base + 1 * plane + row * K + col) = rl;
    *reinterpret_cast<float4*>(base + 2 * plane + row * K + col) = ih;
    *reinterpret_cast<float4*>(base + 3 * plane + row * K + col) = il;
}

// K3 tiles.  Left: row (v, A), col k = (s*nq + j)*4 + B, value Gamma1_s^{cL[A][B]}(w, v, v''_j)
// (v-dependent part incl. the own K2 class).  Right: row (v', C), same k, value
// sum_D Pi[B][D] Gamma2_s^{cR[D][C]}(w, v''_j, v').  Four planes per tile:
// [plane][row][k], plane = 2*(re 0 / im 1) + (hi 0 / lo 1), each plane rows x K floats.
// MODE 0: left tile, 1: right tile, 2: both from one gather of the left record, the right
// record being its symmetry image at the same w (a, p: conjugation; t: conjugation after
// crossing, with the spin terms up-down <-> up-down, up-up <-> up-up).
// Rows: the left tile holds v = vh .. N3v-1 (rowsL = 4 (N3v - vh) rows), the right tile all
// v' (rowsR = 4 N3v rows).  vh > 0 (p channel, MODE 2): only the crossing-independent half
// v >= 0 of the output is computed; the right tile rows v' < 0 then come from the same
// records through crossing, Gamma2(w, -v'', -v) = X[Gamma2(w, v'', v)], written at the
// mirrored node nq-1-j (the node set is symmetric under v'' -> -v'').
template <int MODE, int R>
__global__ void __launch_bounds__(128, 6) k_mx_tile3(VertexF V, DfGrids G, MixedJob J, int w0, int wt0, int vh,
                                                  int rowsL, int rowsR, const float2* __restrict__ Pt,
                                                  float* __restrict__ tile, float* __restrict__ tileR, int dform = 0) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int NS = (R == KB_CH_T) ? 2 : 1;
    constexpr bool RIGHT = (MODE == 1);
    int vi = vh + blockIdx.y, wl = blockIdx.z;
    if (j >= J.nq) return;
    const df* qn = G.n3v + G.N3v;
    df w = G.n3w[w0 + wl], ve = G.n3v[vi];
    // dform (t): one record per side, the density combination up-up + up-down
    const size_t K = (size_t)4 * (dform ? 1 : NS) * J.nq;
    const size_t planeL = (size_t)rowsL * K, planeR = (size_t)rowsR * K;
    const float2* P = Pt + ((size_t)(w0 + wl) * J.nq + j) * 16;
    const int vm = G.N3v - 1 - vi;                 // mirrored row of the crossing image
    const bool mirror = (MODE == 2) && (R == KB_CH_P) && vh > 0 && vm != vi;
    const int jm = J.nq - 1 - j;
    const float2* Pm = Pt + ((size_t)(w0 + wl) * J.nq + jm) * 16;
    float2 g[16];
    // t channel: the up-down record first, then the exchanged term turns it into the
    // up-up record (one set of direct lookups for both spin terms).  Spin index s of the
    // tile columns: left s = 0 up-up, s = 1 up-down; right s = 0 up-down, s = 1 up-up.
#pragma unroll 1
    for (int pass = 0; pass < NS; ++pass) {
        const int parts = pass == 0 ? PARTS_UD : PARTS_X;
        if (RIGHT) vertex_part_f32<R, true>(V, G, parts, true, 8 | 16 | 32, w, qn[j], ve, g, pass > 0);
        else vertex_part_f32<R, true>(V, G, parts, false, 8 | 16 | 32, w, ve, qn[j], g, pass > 0);
        if (dform && pass == 0) {
            // density record up-up + up-down = 2 up-down + exchanged term
#pragma unroll
            for (int c = 0; c < 16; ++c) g[c] = make_float2(2.f * g[c].x, 2.f * g[c].y);
            continue;
        }
        const bool uu = pass > 0;
        const int s = (NS == 1 || dform) ? 0 : (RIGHT ? (uu ? 1 : 0) : (uu ? 0 : 1));
        if (MODE != 1) {
            float* base = tile + (size_t)(wt0 + wl) * 4 * planeL;
            size_t col = ((size_t)s * J.nq + j) * 4;
#pragma unroll
            for (int A = 0; A < 4; ++A) {
                float2 v[4] = {g[cmap<R>(A, 0)], g[cmap<R>(A, 1)], g[cmap<R>(A, 2)], g[cmap<R>(A, 3)]};
                write_planes(base, planeL, (size_t)(vi - vh) * 4 + A, K, col, v);
            }
        }
        if (MODE != 0) {
            float2 h[16];
            int sr = s;
            if (MODE == 2) {
                // right record Gamma2^c(w, v'', v' = v) = sign(c) conj(Gamma1^{pi(c)}(w, v, v''))
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    int pc = (R == KB_CH_T) ? perm_x(perm_c(c)) : perm_c(c);
                    float sg = sign_c(c);
                    h[c] = make_float2(sg * g[pc].x, -sg * g[pc].y);
                }
                if (R == KB_CH_T && !dform) sr = 1 - s;      // left up-up (0) <-> right up-up (1)
            } else {
#pragma unroll
                for (int c = 0; c < 16; ++c) h[c] = g[c];
            }
            float* base = (MODE == 2 ? tileR : tile) + (size_t)(wt0 + wl) * 4 * planeR;
            size_t col = ((size_t)sr * J.nq + j) * 4;
#pragma unroll
            for (int C = 0; C < 4; ++C) {
                float2 v[4];
#pragma unroll
                for (int B = 0; B < 4; ++B) {
                    float2 a = make_float2(0, 0);
#pragma unroll
                    for (int D = 0; D < 4; ++D) {
                        float2 p = P[4 * B + D], x = h[cmap<R>(D, C)];
                        a.x = fmaf(p.x, x.x, fmaf(-p.y, x.y, a.x));
                        a.y = fmaf(p.x, x.y, fmaf(p.y, x.x, a.y));
                    }
                    v[B] = a;
                }
                write_planes(base, planeR, (size_t)vi * 4 + C, K, col, v);
            }
            if (mirror) {
                // crossing image: component c of the mirrored record is component perm_x(c)
                size_t colm = ((size_t)sr * J.nq + jm) * 4;
#pragma unroll
                for (int C = 0; C < 4; ++C) {
                    float2 v[4];
#pragma unroll
                    for (int B = 0; B < 4; ++B) {
                        float2 a = make_float2(0, 0);
#pragma unroll
                        for (int D = 0; D < 4; ++D) {
                            float2 p = Pm[4 * B + D], x = h[perm_x(cmap<R>(D, C))];
                            a.x = fmaf(p.x, x.x, fmaf(-p.y, x.y, a.x));
                            a.y = fmaf(p.x, x.y, fmaf(p.y, x.x, a.y));
                        }
                        v[B] = a;
                    }
                    write_planes(base, planeR, (size_t)vm * 4 + C, K, colm, v);
                }
            }
        }
    }
}


// Symmetry fill: out[dst] = image of out[src] for the output classes of a bubble of a
// symmetric vertex with itself (see kb_set_vertex_symmetric).  kind: 0 conjugation after
// crossing (a: w -> -w), 1 conjugation (t: w -> -w), 2 crossing (p: v -> -v), 3 conjugation
// with v <-> v' (a, p: K2' from K2), 4 conjugation after crossing at the same w (t: K2'
// from K2).  Elements: class layout [w][v][v'][16] with nv2/nv3 = 1 where absent.
__global__ void k_mx_symfill(void* outp, const void* srcp, int dt, int kind, int nw, int nv, int nvp, int w_cnt,
                             int v_cnt) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)w_cnt * v_cnt * nvp * 16;
    if (idx >= total) return;
    int c = idx % 16;
    size_t rest = idx / 16;
    int ip = rest % nvp;
    rest /= nvp;
    int iv = rest % v_cnt;
    int iw = (int)(rest / v_cnt);
    // destination indices and source indices
    int dw = iw, dv = iv, dp = ip, sw = iw, sv = iv, sp = ip;
    int pc;
    bool cj;
    float sg = 1.f;
    if (kind == 0 || kind == 1) { sw = nw - 1 - iw; }
    if (kind == 2) { sv = nv - 1 - iv; sp = nvp - 1 - ip; }
    if (kind == 0) { pc = perm_x(perm_c(c)); cj = true; }
    else if (kind == 1) { pc = perm_c(c); cj = true; }
    else if (kind == 2) { pc = perm_x(c); cj = false; }
    else if (kind == 3) { pc = perm_c(c); cj = true; }
    else { pc = perm_x(perm_c(c)); cj = true; }
    if (cj) sg = sign_c(c);
    size_t de = (((size_t)dw * nv + dv) * nvp + dp) * 16 + c;
    size_t se = (((size_t)sw * nv + sv) * nvp + sp) * 16 + pc;
    if (dt == KB_DT_C128) {
        double2 v = reinterpret_cast<const double2*>(srcp)[se];
        reinterpret_cast<double2*>(outp)[de] = make_double2(sg * v.x, cj ? -sg * v.y : sg * v.y);
    } else {
        float2 v = reinterpret_cast<const float2*>(srcp)[se];
        reinterpret_cast<float2*>(outp)[de] = make_float2(sg * v.x, cj ? -sg * v.y : sg * v.y);
    }
}

// SIMT reference contraction of the K3 tiles (hi + lo recombined, FP32 products, FP32
// partial sums over chunks of 64 k, FP64 across chunks).  C[b][m][n] (double2).
__global__ void __launch_bounds__(256) k_mx_cgemm(const float* __restrict__ At, const float* __restrict__ Bt,
                                                  double2* __restrict__ Cm, int M, int N, int K) {
    __shared__ float2 sA[16][65], sB[16][65];
    int b = blockIdx.z, m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    size_t pa = (size_t)M * K, pb = (size_t)N * K;
    const float* A = At + (size_t)b * 4 * pa;
    const float* B = Bt + (size_t)b * 4 * pb;
    int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float2 acc[4][4];
    double2 tot[4][4];
    for (int i = 0; i < 4; ++i)
        for (int jj = 0; jj < 4; ++jj) { acc[i][jj] = make_float2(0, 0); tot[i][jj] = make_double2(0, 0); }
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = threadIdx.x; i < 64 * 16; i += 256) {
            int row = i / 16, kk = i % 16, gk = k0 + kk;
            int gm = m0 + row, gn = n0 + row;
            float2 a = make_float2(0, 0), bb = make_float2(0, 0);
            if (gm < M && gk < K) {
                size_t o = (size_t)gm * K + gk;
                a = make_float2(A[o] + A[pa + o], A[2 * pa + o] + A[3 * pa + o]);
            }
            if (gn < N && gk < K) {
                size_t o = (size_t)gn * K + gk;
                bb = make_float2(B[o] + B[pb + o], B[2 * pb + o] + B[3 * pb + o]);
            }
            sA[kk][row] = a;
            sB[kk][row] = bb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float2 av[4], bv[4];
            for (int i = 0; i < 4; ++i) { av[i] = sA[kk][ty + 16 * i]; bv[i] = sB[kk][tx + 16 * i]; }
            for (int i = 0; i < 4; ++i)
                for (int jj = 0; jj < 4; ++jj) {
                    float2& c = acc[i][jj];
                    c.x = fmaf(av[i].x, bv[jj].x, fmaf(-av[i].y, bv[jj].y, c.x));
                    c.y = fmaf(av[i].x, bv[jj].y, fmaf(av[i].y, bv[jj].x, c.y));
                }
        }
        __syncthreads();
        if (((k0 / 16) & 3) == 3 || k0 + 16 >= K)
            for (int i = 0; i < 4; ++i)
                for (int jj = 0; jj < 4; ++jj) {
                    tot[i][jj].x += acc[i][jj].x; tot[i][jj].y += acc[i][jj].y;
                    acc[i][jj] = make_float2(0, 0);
                }
    }
    for (int i = 0; i < 4; ++i)
        for (int jj = 0; jj < 4; ++jj) {
            int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * jj;
            if (gm < M && gn < N) Cm[((size_t)b * M + gm) * N + gn] = tot[i][jj];
        }
}

// out K3 <- alpha C + beta out, C[wl][(v - vh, A)][(v', C)] for v = vh .. nv-1; with tri only
// the points v <= v' (the rest is filled by k_mx_trifill).
__global__ void k_mx_scatter3(MixedJob J, int w0, int nwc, int nv, int vh, const double2* __restrict__ Cm, void* out,
                              int odt, int tri) {
    const int nvL = nv - vh;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)nwc * nvL * nv * 16;
    if (idx >= total) return;
    int o = idx % 16;
    size_t rest = idx / 16;
    int vR = rest % nv;
    rest /= nv;
    int vL = rest % nvL;
    int wl = (int)(rest / nvL);
    if (tri && vh + vL > vR) return;
    int A = 0, C = 0;
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 4; ++c)
            if (J.M.cO[a][c] == o) { A = a; C = c; }
    int Mr = 4 * nvL, Nc = 4 * nv;
    double2 gv = Cm[((size_t)wl * Mr + 4 * vL + A) * Nc + 4 * vR + C];
    store_out(out, odt, (((size_t)(w0 + wl) * nv + vh + vL) * nv + vR) * 16 + o, gv, J.alpha, J.beta);
}

// K3 points v > v' of the bosonic frequencies w0 .. nw-1 of a symmetric bubble as images of
// the computed points (w, v', v) at the same w: conjugation with v <-> v' (a; kind 0) or
// conjugation after crossing (t; kind 1), component c from component perm(c) with the sign
// of the conjugation.  Class layout [w][v][v'][16]; reads and writes are disjoint (v' < v
// read, v > v' written).
__global__ void k_mx_trifill(void* outp, int dt, int kind, int w0, int nw, int nv) {
    const size_t npair = (size_t)nv * (nv - 1) / 2;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)(nw - w0) * npair * 16) return;
    const int c = idx % 16;
    size_t rest = idx / 16;
    const size_t pr = rest % npair;
    const int iw = w0 + (int)(rest / npair);
    // pair index pr -> (v, v') with v > v': v(v-1)/2 <= pr < v(v+1)/2
    int v = (int)((1.0 + sqrt(1.0 + 8.0 * (double)pr)) * 0.5);
    while ((size_t)v * (v - 1) / 2 > pr) --v;
    while ((size_t)(v + 1) * v / 2 <= pr) ++v;
    const int vp = (int)(pr - (size_t)v * (v - 1) / 2);
    const int pc = kind == 0 ? perm_c(c) : perm_x(perm_c(c));
    const float sg = sign_c(c);
    const size_t de = (((size_t)iw * nv + v) * nv + vp) * 16 + c;
    const size_t se = (((size_t)iw * nv + vp) * nv + v) * 16 + pc;
    if (dt == KB_DT_C128) {
        const double2 x = reinterpret_cast<const double2*>(outp)[se];
        reinterpret_cast<double2*>(outp)[de] = make_double2(sg * x.x, -sg * x.y);
    } else {
        const float2 x = reinterpret_cast<const float2*>(outp)[se];
        reinterpret_cast<float2*>(outp)[de] = make_float2(sg * x.x, -sg * x.y);
    }
}

}  // namespace kb

using namespace kb;

// tcgen05 contraction of the K3 tiles (kb_tc.cu); returns false if not launched.  tri: the
// output blocks whose points all have v > v' are not computed (filled by k_mx_trifill).
bool kb_tc_k3(kb_ctx* ctx, const float* At, const float* Bt, double2* Cm, int M, int N, int K, int batch,
              void* scratch, size_t scratch_bytes, bool tri, cudaStream_t st);

static VertexF to_vf(const VertexDev& V, kb_ctx* ctx, bool& ok) {
    VertexF F;
    ok = true;
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 4; ++k) {
            F.cls[c][k] = reinterpret_cast<const float2*>(V.cls[c][k]);
            if (V.cls[c][k] && V.dt[c][k] != KB_DT_C64) ok = false;
            if (V.cls[c][k] && (reinterpret_cast<uintptr_t>(V.cls[c][k]) & 15)) ok = false;
        }
    F.has_R = V.has_R;
    F.mask = V.mask;
    F.bare = (float)V.bare;
    if (!ok) ctx->err = "mixed precision needs complex64 classes aligned to 16 bytes";
    return F;
}

// The record cache of `slot` for channel r and side (0 left, 1 right), if it was built from
// the slot's current state.
static const float2* valid_cache(const kb_ctx* ctx, int slot, int r, int side) {
    const kb_ctx::RecCache& c = ctx->rc[slot];
    if (!c.ptr[side] || !((c.sides >> side) & 1) || c.channel != r || c.gen != ctx->slot_gen[slot]) return nullptr;
    return static_cast<const float2*>(c.ptr[side]);
}

static size_t cache_side_bytes(const Grids& g, int r, int side) {
    const size_t ns = (r == KB_CH_T) ? 2 : 1;
    if (side < 2) return (size_t)g.n2w * g.n2v * (size_t)rc_blocks(g.nq) * 32 * ns * 16 * sizeof(float2);
    // K3 tile of every bosonic frequency: 4 planes x (4 n3v rows) x (4 ns nq columns), FP32
    return (size_t)g.n3w * 4 * (4 * (size_t)g.n3v) * (4 * ns * (size_t)g.nq) * sizeof(float);
}

// Workspace layout of one mixed-precision bubble of channel r (byte offsets into the
// context's workspace) and the bytes it needs.
struct MixedLayout {
    size_t off_tab, off_N, off_M, off_S, off_P3, off_K1, off_NT, off_BS, off_NS, off_T, rows, K, per_w, tc_scratch,
        need;
    int chunk;
};

static MixedLayout mixed_layout(const kb_ctx* ctx, int r, unsigned mask) {
    const Grids& g = ctx->g;
    int ns = (r == KB_CH_T) ? 2 : 1;
    MixedLayout L;
    size_t ntab = (size_t)g.n1 + g.n2w + g.n2v + g.n3w + g.n3v + g.nq;
    L.off_tab = 0;
    L.off_N = (ntab * sizeof(df) + 255) / 256 * 256;
    size_t szNM = (size_t)g.n2w * ns * g.nq * 16 * sizeof(float2);
    L.off_M = L.off_N + szNM;
    L.off_S = L.off_M + szNM;
    size_t szS = (size_t)2 * g.n2w * ns * 16 * sizeof(double2);
    L.off_P3 = (L.off_S + szS + 255) / 256 * 256;
    size_t szP3 = (size_t)g.n3w * g.nq * 16 * sizeof(float2);
    L.off_K1 = (L.off_P3 + szP3 + 255) / 256 * 256;
    size_t szK1 = (size_t)g.n1 * K1_SLICES * 16 * sizeof(double2);
    L.off_NT = (L.off_K1 + szK1 + 255) / 256 * 256;
    size_t szNT = (size_t)2 * g.n2w * ns * g.n3v * 16 * sizeof(double2);
    // bosonic stencils of the K2 gather's lookup groups (one side at a time)
    L.off_BS = (L.off_NT + szNT + 255) / 256 * 256;
    size_t szBS = (size_t)2 * ns * g.n2v * g.nq * sizeof(float4);
    // the nodes' stencils on the K3 fermionic grid (k_mx_nstencil)
    L.off_NS = (L.off_BS + szBS + 255) / 256 * 256;
    size_t szNS = (size_t)g.nq * sizeof(int2);
    L.off_T = (L.off_NS + szNS + 1023) / 1024 * 1024;
    L.rows = (size_t)4 * g.n3v;
    L.K = (size_t)4 * ns * g.nq;
    L.per_w = 2 * 4 * L.rows * L.K * sizeof(float) + L.rows * L.rows * sizeof(double2) + 1024;
    size_t budget = ctx->ws_limit > L.off_T ? ctx->ws_limit - L.off_T : 0;
    L.chunk = (int)std::max<size_t>(1, std::min<size_t>(g.n3w, budget / L.per_w));
    L.tc_scratch = std::min<size_t>(2ull << 30, std::max<size_t>(64ull << 20, (size_t)24 * L.chunk * L.rows * L.rows * 16));
    L.need = ((mask >> KB_K3) & 1) ? L.off_T + L.per_w * L.chunk + L.tc_scratch : L.off_T;
    return L;
}

size_t kb_mixed_workspace_need(const kb_ctx* ctx, int r, unsigned mask) { return mixed_layout(ctx, r, mask).need; }

// One-time per device (not a stream operation, so done before any capture): the dynamic
// shared memory of the K2 gather beyond the default 48 KB.
static bool mixed_prepare(int device) {
    static bool done[64] = {};
    if (device < 0 || device >= 64) return false;
    if (done[device]) return true;
    bool ok = true;
    ok = ok && cudaFuncSetAttribute(k_mx_k2<false, KB_CH_T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)k2_smem_bytes<KB_CH_T>()) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_mx_k2<true, KB_CH_T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)k2_smem_bytes<KB_CH_T>()) == cudaSuccess;
    done[device] = ok;
    return ok;
}

bool kb_mixed_prepare(int device) { return mixed_prepare(device); }

bool kb::kb_slot_f32(kb_ctx* ctx, int slot, VertexF& F) {
    bool ok;
    F = to_vf(ctx->slots[slot], ctx, ok);
    return ok;
}

void kb::kb_mixed_tables(kb_ctx* ctx, df* tab, DfGrids& G, cudaStream_t st) {
    const Grids& g = ctx->g;
    const size_t ntab = (size_t)g.n1 + g.n2w + g.n2v + g.n3w + g.n3v + g.nq;
    G.n1 = tab; G.n2w = G.n1 + g.n1; G.n2v = G.n2w + g.n2w; G.n3w = G.n2v + g.n2v; G.n3v = G.n3w + g.n3w;
    G.N1 = g.n1; G.N2w = g.n2w; G.N2v = g.n2v; G.N3w = g.n3w; G.N3v = g.n3v; G.A = (float)g.A;
    KB_LAUNCH(ctx, st, "k_mx_tables");
    k_mx_tables<<<(unsigned)((ntab + 255) / 256), 256, 0, st>>>(g.n1, g.n2w, g.n2v, g.n3w, g.n3v, g.nq, g.A, ctx->d_xq,
                                                                tab);
}

template <int r>
static kb_status mixed_impl(kb_ctx* ctx, int sl, int sr, int so, int pi_kind, unsigned mask, double alpha, double beta,
                            cudaStream_t st, bool tsu2 = false) {
    const Grids& g = ctx->g;
    bool ok1, ok2;
    VertexF VL = to_vf(ctx->slots[sl], ctx, ok1), VR = to_vf(ctx->slots[sr], ctx, ok2);
    if (!ok1 || !ok2) return KB_ERR_ARG;
    const VertexDev& VO = ctx->slots[so];
    // classes that vanish identically (a side without bare part and without channel r)
    {
        const unsigned zero = kb_zero_classes(ctx, r, sl, sr, mask);
        kb_status zs = kb_scale_classes(ctx, r, so, zero, beta, st);
        if (zs != KB_OK) return zs;
        mask &= ~zero;
    }
    // a bubble of a declared-symmetric vertex with itself: compute the independent part only
    const bool sym = (sl == sr) && ctx->slots[sl].symmetric && beta == 0.0 &&
                     (!((mask >> KB_K2P) & 1) || ((mask >> KB_K2) & 1)) && std::getenv("KB_NO_SYMMETRY") == nullptr;
    MixedJob J;
    J.r = r; J.pi_kind = pi_kind; J.ns = (r == KB_CH_T) ? 2 : 1; J.nq = g.nq;
    J.M = channel_maps(r); J.alpha = alpha; J.beta = beta;
    int ns = J.ns;
    const MixedLayout Lo = mixed_layout(ctx, r, mask);
    const size_t off_tab = Lo.off_tab, off_N = Lo.off_N, off_M = Lo.off_M, off_S = Lo.off_S, off_P3 = Lo.off_P3,
                 off_T = Lo.off_T, rows = Lo.rows, K = Lo.K, tc_scratch = Lo.tc_scratch;
    const int chunk = Lo.chunk;
    const size_t ntab = (size_t)g.n1 + g.n2w + g.n2v + g.n3w + g.n3v + g.nq;
    kb_status s = kb_ensure_workspace(ctx, Lo.need, st);
    if (s != KB_OK) return s;
    if (!mixed_prepare(ctx->device)) {
        ctx->err = "mixed path: cannot set the K2 gather's shared-memory size";
        return KB_ERR_CUDA;
    }
    char* ws = static_cast<char*>(ctx->ws.ptr);
    df* tab = reinterpret_cast<df*>(ws + off_tab);
    float2* Nt = reinterpret_cast<float2*>(ws + off_N);
    float2* Mt = reinterpret_cast<float2*>(ws + off_M);
    double2* Ss = reinterpret_cast<double2*>(ws + off_S);
    double2* Ntl = reinterpret_cast<double2*>(ws + Lo.off_NT);
    float2* P3 = reinterpret_cast<float2*>(ws + off_P3);
    DfGrids G;
    G.n1 = tab; G.n2w = G.n1 + g.n1; G.n2v = G.n2w + g.n2w; G.n3w = G.n2v + g.n2v; G.n3v = G.n3w + g.n3w;
    G.N1 = g.n1; G.N2w = g.n2w; G.N2v = g.n2v; G.N3w = g.n3w; G.N3v = g.n3v; G.A = (float)g.A;
    {
        KB_LAUNCH(ctx, st, "k_mx_tables");
        k_mx_tables<<<(unsigned)((ntab + 255) / 256), 256, 0, st>>>(g.n1, g.n2w, g.n2v, g.n3w, g.n3v, g.nq, g.A, ctx->d_xq,
                                                                    tab);
    }
    if ((mask >> KB_K1) & 1) {
        int w_off = (sym && r != KB_CH_P) ? g.n1 / 2 : 0;
        const int half = (sym && r == KB_CH_P) ? 1 : 0;
        double2* part = reinterpret_cast<double2*>(ws + Lo.off_K1);
        {
            KB_LAUNCH(ctx, st, "k_mx_k1");
            k_mx_k1<r><<<dim3(g.n1 - w_off, K1_SLICES), 128, 0, st>>>(VL, VR, G, ctx->m, J, ctx->d_xq, ctx->d_wq,
                                                                     part, w_off, half);
        }
        {
            KB_LAUNCH(ctx, st, "k_mx_k1_fin");
            int tot = (g.n1 - w_off) * 16;
            k_mx_k1_fin<<<(tot + 127) / 128, 128, 0, st>>>(J, part, const_cast<void*>(VO.cls[r][KB_K1]),
                                                          VO.dt[r][KB_K1], w_off, g.n1 - w_off, half);
        }
    }
    if (mask & ((1u << KB_K2) | (1u << KB_K2P))) {
        {
            KB_LAUNCH(ctx, st, "k_mx_prep_k2");
            k_mx_prep_k2<r><<<dim3((g.nq + 127) / 128, g.n2w), 128, 0, st>>>(VL, VR, G, ctx->m, J, ctx->d_xq, ctx->d_wq,
                                                                          G.n2w, Nt, Mt);
        }
        {
            KB_LAUNCH(ctx, st, "k_mx_sumj");
            k_mx_sumj<<<dim3(g.n2w, ns, 2), 128, 0, st>>>(Nt, Mt, g.nq, ns, Ss);
        }
        {
            // left (N) table for K2; the right (M) table only when K2' is gathered
            int2* nst = reinterpret_cast<int2*>(ws + Lo.off_NS);
            {
                KB_LAUNCH(ctx, st, "k_mx_nstencil");
                k_mx_nstencil<<<(g.nq + 127) / 128, 128, 0, st>>>(G, g.nq, nst);
            }
            KB_LAUNCH(ctx, st, "k_mx_ntilde");
            const int nt = (!sym && ((mask >> KB_K2P) & 1)) ? 2 : 1;
            const int t0 = ((mask >> KB_K2) & 1) ? 0 : 1;
            k_mx_ntilde<<<dim3((g.n3v * 64 + 127) / 128, g.n2w, ns * (t0 == 1 ? 1 : nt)), 128, 0, st>>>(
                Nt, Mt, G, g.nq, ns, t0, nst, Ntl);
        }
        const float2* cacheL = valid_cache(ctx, sl, r, 0);
        const float2* cacheR = valid_cache(ctx, sr, r, 1);
        // bosonic stencils of the gather's lookup groups, tabulated per (group, v, node)
        // before each gather side (grids within the packing limits; else found in the gather)
        float4* bst = (g.n1 <= BSTEN_MAX_N1 && g.n2w <= BSTEN_MAX_NW && g.n3w <= BSTEN_MAX_NW)
                          ? reinterpret_cast<float4*>(ws + Lo.off_BS)
                          : nullptr;
        auto bsten = [&](bool right) {
            if (!bst) return;
            KB_LAUNCH(ctx, st, "k_mx_bsten");
            const dim3 grid((g.nq + 127) / 128, g.n2v, 2 * ns);
            if (right) k_mx_bsten<true, r><<<grid, 128, 0, st>>>(G, g.nq, bst);
            else k_mx_bsten<false, r><<<grid, 128, 0, st>>>(G, g.nq, bst);
        };
        if ((mask >> KB_K2) & 1) {
            int w_off = (sym && r != KB_CH_P) ? g.n2w / 2 : 0, v_off = (sym && r == KB_CH_P) ? g.n2v / 2 : 0;
            void* o = const_cast<void*>(VO.cls[r][KB_K2]);
            const dim3 grid(g.n2v - v_off, g.n2w - w_off);
            if (cacheL) {
                KB_LAUNCH(ctx, st, "k_mx_k2c");
                k_mx_k2_rc<false, r><<<grid, 128, 0, st>>>(VL, G, J, Nt, Ss, Ntl, o, VO.dt[r][KB_K2], w_off, v_off,
                                                           cacheL);
            } else {
                bsten(false);
                KB_LAUNCH(ctx, st, "k_mx_k2");
                k_mx_k2<false, r><<<grid, K2_THREADS, k2_smem_bytes<r>(), st>>>(VL, G, J, Nt, Ss, Ntl, o, VO.dt[r][KB_K2],
                                                                         w_off, v_off, bst);
            }
        }
        if (!sym && ((mask >> KB_K2P) & 1)) {
            void* o = const_cast<void*>(VO.cls[r][KB_K2P]);
            if (cacheR) {
                KB_LAUNCH(ctx, st, "k_mx_k2pc");
                k_mx_k2_rc<true, r><<<dim3(g.n2v, g.n2w), 128, 0, st>>>(VR, G, J, Mt, Ss, Ntl, o, VO.dt[r][KB_K2P], 0,
                                                                        0, cacheR);
            } else {
                bsten(true);
                KB_LAUNCH(ctx, st, "k_mx_k2p");
                k_mx_k2<true, r><<<dim3(g.n2v, g.n2w), K2_THREADS, k2_smem_bytes<r>(), st>>>(VR, G, J, Mt, Ss, Ntl, o,
                                                                                      VO.dt[r][KB_K2P], 0, 0, bst);
            }
        }
    }
    if ((mask >> KB_K3) & 1) {
        {
            KB_LAUNCH(ctx, st, "k_mx_pi3");
            k_mx_pi3<<<dim3((g.nq + 127) / 128, g.n3w), 128, 0, st>>>(G, ctx->m, J, ctx->d_xq, ctx->d_wq, P3);
        }
        float* TA = reinterpret_cast<float*>(ws + off_T);
        float* TB = TA + (size_t)chunk * 4 * rows * K;
        double2* Cm = reinterpret_cast<double2*>(TB + (size_t)chunk * 4 * rows * K);
        void* scratch = reinterpret_cast<char*>(Cm) + (size_t)chunk * rows * rows * sizeof(double2);
        bool use_tc = std::getenv("KB_K3_SIMT") == nullptr;
        const float* cacheL3 = reinterpret_cast<const float*>(valid_cache(ctx, sl, r, 2));
        const float* cacheR3 =
            pi_kind == KB_PI_GG ? reinterpret_cast<const float*>(valid_cache(ctx, sr, r, 3)) : nullptr;
        int w3_lo = (sym && r != KB_CH_P) ? g.n3w / 2 : 0;
        // p (symmetric): rows v >= 0 only, the rest by crossing (k_mx_tile3, symmetry fill)
        const int vh3 = (sym && r == KB_CH_P) ? g.n3v / 2 : 0;
        const int rowsL = 4 * (g.n3v - vh3), rowsR = (int)rows;
        // a, t (symmetric): the points v > v' of each w are the images of (w, v', v) at the
        // same w, so the contraction skips the blocks that hold only such points
        const bool tri3 = sym && r != KB_CH_P;
        // t in its SU(2) form (tsu2, symmetric only): the density contraction with K = 4 Nq,
        // scattered with alpha / 2; kb_t_su2_finish adds the crossed a bubble and the images
        const bool td = tsu2 && r == KB_CH_T && sym;
        const size_t K3K = td ? (size_t)4 * g.nq : K;
        MixedJob J3 = J;
        if (td) J3.alpha = 0.5 * J.alpha;
        for (int w0 = w3_lo; w0 < g.n3w; w0 += chunk) {
            int nwc = std::min(chunk, g.n3w - w0);
            float* TAc = TA;
            float* TBc = TB;
            if (sym) {
                KB_LAUNCH(ctx, st, "k_mx_tile3_both");
                k_mx_tile3<2, r><<<dim3((g.nq + 127) / 128, g.n3v - vh3, nwc), 128, 0, st>>>(VL, G, J, w0, 0, vh3, rowsL,
                                                                                           rowsR, P3, TA, TB, td ? 1 : 0);
            } else {
                if (cacheL3) {
                    TAc = const_cast<float*>(cacheL3) + (size_t)w0 * 4 * rowsL * K;      // cached left tile
                } else {
                    KB_LAUNCH(ctx, st, "k_mx_tile3_left");
                    k_mx_tile3<0, r><<<dim3((g.nq + 127) / 128, g.n3v, nwc), 128, 0, st>>>(VL, G, J, w0, 0, 0, rowsL,
                                                                                           rowsR, P3, TA, nullptr);
                }
                if (cacheR3) {
                    TBc = const_cast<float*>(cacheR3) + (size_t)w0 * 4 * rowsR * K;      // cached right tile
                } else {
                    KB_LAUNCH(ctx, st, "k_mx_tile3_right");
                    k_mx_tile3<1, r><<<dim3((g.nq + 127) / 128, g.n3v, nwc), 128, 0, st>>>(VR, G, J, w0, 0, 0, rowsL,
                                                                                           rowsR, P3, TB, nullptr);
                }
            }
            bool done = false;
            if (use_tc) done = kb_tc_k3(ctx, TAc, TBc, Cm, rowsL, rowsR, (int)K3K, nwc, scratch, tc_scratch, tri3, st);
            if (!done) {
                KB_LAUNCH(ctx, st, "k_mx_cgemm");
                k_mx_cgemm<<<dim3((unsigned)((rowsR + 63) / 64), (unsigned)((rowsL + 63) / 64), nwc), 256, 0, st>>>(
                    TAc, TBc, Cm, rowsL, rowsR, (int)K3K);
            }
            {
                KB_LAUNCH(ctx, st, "k_mx_scatter3");
                size_t tot = (size_t)nwc * (g.n3v - vh3) * g.n3v * 16;
                k_mx_scatter3<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(J3, w0, nwc, g.n3v, vh3, Cm,
                                                                            const_cast<void*>(VO.cls[r][KB_K3]),
                                                                            VO.dt[r][KB_K3], tri3 ? 1 : 0);
            }
        }
        if (tri3 && g.n3v > 1 && !td) {
            KB_LAUNCH(ctx, st, "k_mx_trifill");
            const size_t tot = (size_t)(g.n3w - w3_lo) * g.n3v * (g.n3v - 1) / 2 * 16;
            k_mx_trifill<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(const_cast<void*>(VO.cls[r][KB_K3]),
                                                                       VO.dt[r][KB_K3], r == KB_CH_A ? 0 : 1, w3_lo,
                                                                       g.n3w, g.n3v);
        }
    }
    if (sym) {
        auto fill = [&](int dst_cls, int src_cls, int kind, int nw, int nv, int nvp, int wc, int vc) {
            KB_LAUNCH(ctx, st, "k_mx_symfill");
            size_t tot = (size_t)wc * vc * nvp * 16;
            if (tot == 0) return;
            k_mx_symfill<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(const_cast<void*>(VO.cls[r][dst_cls]),
                                                                        VO.cls[r][src_cls], VO.dt[r][dst_cls], kind, nw,
                                                                        nv, nvp, wc, vc);
        };
        int kw = (r == KB_CH_A) ? 0 : 1;                 // w -> -w image: a conj-after-crossing, t conj
        if (r != KB_CH_P) {
            if ((mask >> KB_K1) & 1) fill(KB_K1, KB_K1, kw, g.n1, 1, 1, g.n1 / 2, 1);
            if (((mask >> KB_K3) & 1) && !(tsu2 && r == KB_CH_T)) fill(KB_K3, KB_K3, kw, g.n3w, g.n3v, g.n3v, g.n3w / 2, g.n3v);
        }
        if (r == KB_CH_P && ((mask >> KB_K3) & 1)) fill(KB_K3, KB_K3, 2, g.n3w, g.n3v, g.n3v, g.n3w, g.n3v / 2);
        if ((mask >> KB_K2) & 1) {
            if (r != KB_CH_P) fill(KB_K2, KB_K2, kw, g.n2w, g.n2v, 1, g.n2w / 2, g.n2v);
            else fill(KB_K2, KB_K2, 2, g.n2w, g.n2v, 1, g.n2w, g.n2v / 2);
            if ((mask >> KB_K2P) & 1) fill(KB_K2P, KB_K2, r == KB_CH_T ? 4 : 3, g.n2w, g.n2v, 1, g.n2w, g.n2v);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("mixed launch: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}

// The t bubble of a symmetric slot with itself in its SU(2) form (kb_bubble_t_su2): K1, K2
// and K2' as kb_bubble computes them, K3 = alpha/2 times the density contraction for the
// independent points (w >= 0, v <= v'), completed by kb_t_su2_finish_impl.
kb_status kb_bubble_mixed_t_su2(kb_ctx* ctx, int sl, int so, int pi_kind, unsigned mask, double alpha,
                                cudaStream_t st) {
    if (!ctx->slots[sl].symmetric) {
        ctx->err = "kb_bubble_t_su2: the slot must be declared symmetric";
        return KB_ERR_ARG;
    }
    // the identity needs the density contraction itself: K3 must not be one of the classes
    // the ordinary bubble skips as identically zero
    if ((mask >> KB_K3) & 1 & (kb_zero_classes(ctx, KB_CH_T, sl, sl, mask) >> KB_K3)) {
        ctx->err = "kb_bubble_t_su2: the slot needs its bare part or channel t";
        return KB_ERR_ARG;
    }
    return mixed_impl<KB_CH_T>(ctx, sl, sl, so, pi_kind, mask, alpha, 0.0, st, true);
}

// K3 of the t output += alpha/2 X[B_a]: the crossed a bubble at t-variables (w, v, v') is
// B_a(-w, v, v') with the Keldysh indices a1, a2 exchanged (component kswap12(c)); for the
// independent points w >= 0 (index >= n3w / 2), v <= v'.
__global__ void k_mx_t_su2_add(void* outp, int odt, const void* ap, int adt, double half_alpha, int nw, int nv) {
    const int w0 = nw / 2;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)(nw - w0) * nv * nv * 16;
    if (idx >= total) return;
    const int c = idx % 16;
    size_t rest = idx / 16;
    const int vp = rest % nv;
    rest /= nv;
    const int v = rest % nv;
    const int w = w0 + (int)(rest / nv);
    if (v > vp) return;
    const size_t de = (((size_t)w * nv + v) * nv + vp) * 16 + c;
    const size_t se = (((size_t)(nw - 1 - w) * nv + v) * nv + vp) * 16 + kswap12(c);
    double2 x;
    if (adt == KB_DT_C128) x = reinterpret_cast<const double2*>(ap)[se];
    else {
        const float2 y = reinterpret_cast<const float2*>(ap)[se];
        x = make_double2(y.x, y.y);
    }
    if (odt == KB_DT_C128) {
        double2* o = reinterpret_cast<double2*>(outp) + de;
        *o = make_double2(o->x + half_alpha * x.x, o->y + half_alpha * x.y);
    } else {
        float2* o = reinterpret_cast<float2*>(outp) + de;
        *o = make_float2((float)(o->x + half_alpha * x.x), (float)(o->y + half_alpha * x.y));
    }
}

kb_status kb_t_su2_finish_impl(kb_ctx* ctx, int so, const void* a_k3, int a_dt, double alpha, cudaStream_t st) {
    const Grids& g = ctx->g;
    void* out = const_cast<void*>(ctx->slots[so].cls[KB_CH_T][KB_K3]);
    const int odt = ctx->slots[so].dt[KB_CH_T][KB_K3];
    {
        KB_LAUNCH(ctx, st, "k_mx_t_su2_add");
        const size_t tot = (size_t)(g.n3w - g.n3w / 2) * g.n3v * g.n3v * 16;
        k_mx_t_su2_add<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(out, odt, a_k3, a_dt, 0.5 * alpha, g.n3w, g.n3v);
    }
    if (g.n3v > 1) {
        KB_LAUNCH(ctx, st, "k_mx_trifill");
        const size_t tot = (size_t)(g.n3w - g.n3w / 2) * g.n3v * (g.n3v - 1) / 2 * 16;
        k_mx_trifill<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(out, odt, 1, g.n3w / 2, g.n3w, g.n3v);
    }
    {
        // w < 0 through conjugation (the t channel's image)
        KB_LAUNCH(ctx, st, "k_mx_symfill");
        const size_t tot = (size_t)(g.n3w / 2) * g.n3v * g.n3v * 16;
        if (tot)
            k_mx_symfill<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(out, out, odt, 1, g.n3w, g.n3v, g.n3v,
                                                                        g.n3w / 2, g.n3v);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("kb_t_su2_finish launch: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}

kb_status kb_bubble_mixed(kb_ctx* ctx, int r, int sl, int sr, int so, int pi_kind, unsigned mask, double alpha,
                          double beta, cudaStream_t st) {
    if (r == KB_CH_A) return mixed_impl<KB_CH_A>(ctx, sl, sr, so, pi_kind, mask, alpha, beta, st);
    if (r == KB_CH_P) return mixed_impl<KB_CH_P>(ctx, sl, sr, so, pi_kind, mask, alpha, beta, st);
    return mixed_impl<KB_CH_T>(ctx, sl, sr, so, pi_kind, mask, alpha, beta, st);
}

void kb_vertex_cache_free(kb_ctx* ctx, int slot) {
    kb_ctx::RecCache& c = ctx->rc[slot];
    if (c.ptr[0] || c.ptr[1] || c.ptr[2] || c.ptr[3]) ++ctx->mem_gen;
    for (int side = 0; side < 4; ++side) {
        if (c.ptr[side]) cudaFree(c.ptr[side]);
        c.ptr[side] = nullptr;
        c.bytes[side] = 0;
    }
    c.channel = -1;
    c.sides = 0;
    c.gen = ~0ull;
}

kb_status kb_vertex_cache_prepare(kb_ctx* ctx, int slot, int channel, unsigned sides) {
    if (!ctx) return KB_ERR_ARG;
    if (slot < 0 || slot >= KB_MAX_SLOTS || channel < 0 || channel > 2 || sides < 1 || sides > 15) {
        ctx->err = "kb_vertex_cache: bad slot, channel or sides";
        return KB_ERR_ARG;
    }
    if (!ctx->grids_set || !ctx->slot_set[slot]) {
        ctx->err = "kb_vertex_cache: set the grids and the vertex first";
        return KB_ERR_STATE;
    }
    bool ok;
    to_vf(ctx->slots[slot], ctx, ok);
    if (!ok) return KB_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return KB_ERR_CUDA;
    kb_ctx::RecCache& c = ctx->rc[slot];
    for (int side = 0; side < 4; ++side) {
        if (!((sides >> side) & 1)) continue;
        const size_t need = cache_side_bytes(ctx->g, channel, side);
        if (c.ptr[side] && c.bytes[side] == need) continue;
        if (c.ptr[side]) {
            cudaFree(c.ptr[side]);
            ++ctx->mem_gen;
        }
        c.ptr[side] = nullptr;
        c.bytes[side] = 0;
        cudaError_t e = cudaMalloc(&c.ptr[side], need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c.ptr[side] = nullptr;
            ctx->err = "kb_vertex_cache: cannot allocate the record cache";
            return e == cudaErrorMemoryAllocation ? KB_ERR_OOM : KB_ERR_CUDA;
        }
        c.bytes[side] = need;
    }
    c.channel = channel;
    c.sides = sides;
    c.gen = ctx->slot_gen[slot];
    // the frequency tables (and, for the right K3 tile, the Π table) of the build
    return kb_ensure_workspace(ctx, mixed_layout(ctx, channel, 0).off_T, nullptr, true);
}

template <int r>
static void cache_launch(kb_ctx* ctx, int slot, const VertexF& V, unsigned sides, cudaStream_t st) {
    const Grids& g = ctx->g;
    const size_t ntab = (size_t)g.n1 + g.n2w + g.n2v + g.n3w + g.n3v + g.nq;
    df* tab = reinterpret_cast<df*>(static_cast<char*>(ctx->ws.ptr) + mixed_layout(ctx, r, 0).off_tab);
    DfGrids G;
    G.n1 = tab; G.n2w = G.n1 + g.n1; G.n2v = G.n2w + g.n2w; G.n3w = G.n2v + g.n2v; G.n3v = G.n3w + g.n3w;
    G.N1 = g.n1; G.N2w = g.n2w; G.N2v = g.n2v; G.N3w = g.n3w; G.N3v = g.n3v; G.A = (float)g.A;
    {
        KB_LAUNCH(ctx, st, "k_mx_tables");
        k_mx_tables<<<(unsigned)((ntab + 255) / 256), 256, 0, st>>>(g.n1, g.n2w, g.n2v, g.n3w, g.n3v, g.nq, g.A, ctx->d_xq,
                                                                    tab);
    }
    const dim3 grid((unsigned)((g.nq - 2 + 127) / 128), g.n2v, g.n2w);
    for (int side = 0; side < 2; ++side) {
        if (!((sides >> side) & 1)) continue;
        KB_LAUNCH(ctx, st, "k_mx_cache_k2");
        float2* dst = static_cast<float2*>(ctx->rc[slot].ptr[side]);
        if (side == 0) k_mx_cache_k2<false, r><<<grid, 128, 0, st>>>(V, G, g.nq, dst);
        else k_mx_cache_k2<true, r><<<grid, 128, 0, st>>>(V, G, g.nq, dst);
    }
    if (sides & 12) {
        // K3 tiles of all bosonic frequencies, as the non-symmetric bubble builds them
        // chunk by chunk; the right tile with Π = G G folded in
        MixedJob J;
        J.r = r; J.pi_kind = KB_PI_GG; J.ns = (r == KB_CH_T) ? 2 : 1; J.nq = g.nq;
        J.M = channel_maps(r); J.alpha = 1.0; J.beta = 0.0;
        const MixedLayout Lo = mixed_layout(ctx, r, 1u << KB_K3);
        float2* P3 = reinterpret_cast<float2*>(static_cast<char*>(ctx->ws.ptr) + Lo.off_P3);
        const int rows = (int)Lo.rows;
        const dim3 g3((g.nq + 127) / 128, g.n3v, g.n3w);
        if (sides & 4) {
            KB_LAUNCH(ctx, st, "k_mx_cache_tile3");
            k_mx_tile3<0, r><<<g3, 128, 0, st>>>(V, G, J, 0, 0, 0, rows, rows, P3,
                                                 static_cast<float*>(ctx->rc[slot].ptr[2]), nullptr);
        }
        if (sides & 8) {
            {
                KB_LAUNCH(ctx, st, "k_mx_pi3");
                k_mx_pi3<<<dim3((g.nq + 127) / 128, g.n3w), 128, 0, st>>>(G, ctx->m, J, ctx->d_xq, ctx->d_wq, P3);
            }
            KB_LAUNCH(ctx, st, "k_mx_cache_tile3");
            k_mx_tile3<1, r><<<g3, 128, 0, st>>>(V, G, J, 0, 0, 0, rows, rows, P3,
                                                 static_cast<float*>(ctx->rc[slot].ptr[3]), nullptr);
        }
    }
}

kb_status kb_vertex_cache_launch(kb_ctx* ctx, int slot, int channel, unsigned sides, cudaStream_t st) {
    const kb_ctx::RecCache& c = ctx->rc[slot];
    if (c.channel != channel || (c.sides & sides) != sides || c.gen != ctx->slot_gen[slot]) {
        ctx->err = "kb_vertex_cache: cache not prepared for this slot state";
        return KB_ERR_STATE;
    }
    bool ok;
    VertexF V = to_vf(ctx->slots[slot], ctx, ok);
    if (!ok) return KB_ERR_ARG;
    if (channel == KB_CH_A) cache_launch<KB_CH_A>(ctx, slot, V, sides, st);
    else if (channel == KB_CH_P) cache_launch<KB_CH_P>(ctx, slot, V, sides, st);
    else cache_launch<KB_CH_T>(ctx, slot, V, sides, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("kb_vertex_cache: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}

extern "C" kb_status kb_vertex_cache(kb_ctx* ctx, int slot, int channel, unsigned sides, void* stream) {
    kb_status s = kb_vertex_cache_prepare(ctx, slot, channel, sides);
    if (s != KB_OK) return s;
    return kb_vertex_cache_launch(ctx, slot, channel, sides, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" kb_status kb_vertex_uncache(kb_ctx* ctx, int slot) {
    if (!ctx) return KB_ERR_ARG;
    if (slot < 0 || slot >= KB_MAX_SLOTS) { ctx->err = "kb_vertex_uncache: bad slot"; return KB_ERR_ARG; }
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    kb_vertex_cache_free(ctx, slot);
    return KB_OK;
}

// Tune the split-K factor of the tensor-core contraction for the K3 shapes this bubble will
// use (the full chunks of bosonic frequencies and the last partial one), on the context's
// workspace as operands (any values do for timing); for step graphs, before the capture.
kb_status kb_mixed_tune(kb_ctx* ctx, int r, int sl, int sr, unsigned mask, double beta, cudaStream_t st, bool tsu2) {
    mask &= ~kb_zero_classes(ctx, r, sl, sr, mask);
    if (!((mask >> KB_K3) & 1) || std::getenv("KB_K3_SIMT")) return KB_OK;
    const Grids& g = ctx->g;
    const bool sym = (sl == sr) && ctx->slots[sl].symmetric && beta == 0.0 &&
                     (!((mask >> KB_K2P) & 1) || ((mask >> KB_K2) & 1)) && std::getenv("KB_NO_SYMMETRY") == nullptr;
    const MixedLayout Lo = mixed_layout(ctx, r, mask);
    kb_status s = kb_ensure_workspace(ctx, Lo.need, st);
    if (s != KB_OK) return s;
    char* ws = static_cast<char*>(ctx->ws.ptr);
    float* TA = reinterpret_cast<float*>(ws + Lo.off_T);
    float* TB = TA + (size_t)Lo.chunk * 4 * Lo.rows * Lo.K;
    double2* Cm = reinterpret_cast<double2*>(TB + (size_t)Lo.chunk * 4 * Lo.rows * Lo.K);
    void* scratch = reinterpret_cast<char*>(Cm) + (size_t)Lo.chunk * Lo.rows * Lo.rows * sizeof(double2);
    const int w3_lo = (sym && r != KB_CH_P) ? g.n3w / 2 : 0;
    const int vh3 = (sym && r == KB_CH_P) ? g.n3v / 2 : 0;
    const int rowsL = 4 * (g.n3v - vh3), rowsR = (int)Lo.rows, nw = g.n3w - w3_lo;
    const bool tri3 = sym && r != KB_CH_P;
    const int K3K = (tsu2 && sym && r == KB_CH_T) ? 4 * g.nq : (int)Lo.K;
    const int full = std::min(Lo.chunk, nw), last = nw % Lo.chunk;
    kb_tc_tune(ctx, TA, TB, Cm, rowsL, rowsR, K3K, full, scratch, Lo.tc_scratch, tri3, st);
    if (last && last != full) kb_tc_tune(ctx, TA, TB, Cm, rowsL, rowsR, K3K, last, scratch, Lo.tc_scratch, tri3, st);
    return cudaGetLastError() == cudaSuccess ? KB_OK : KB_ERR_CUDA;
}
