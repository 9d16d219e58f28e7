// Plain FP64 path: every step (propagators, Pi, vertex gather, contraction, scatter) in
// double precision.  Structure per output class and chunk of bosonic frequencies:
//   k_pi_table      Pi_r(w, v''_j) 4x4, times c_r w_j J_j / (2 pi i)
//   k_gather_f64    left tile  L[w][(v, A)][(s, j, B)]
//                   right tile R'[w][(v', C)][(s, j, B)] = sum_D Pi[B][D] R[D][C]
//   k_zgemm_f64     G[w][(v, A)][(v', C)] = sum_k L[..][k] R'[..][k]
//   k_scatter       out[w][v][v'][c(A, C)] = alpha G + beta out
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "kb_fp64.cuh"

namespace kb {

// Batched complex GEMM G[b][m][n] = sum_k A[b][m][k] * B[b][n][k] (both K-contiguous).
// 32x32 output tile, 256 threads, each 2x2 outputs; K chunks of 16 through shared memory.
__global__ void __launch_bounds__(256) k_zgemm_f64(const double2* __restrict__ Am, const double2* __restrict__ Bm,
                                                   double2* __restrict__ Cm, int M, int N, int K) {
    __shared__ double2 sA[16][33], sB[16][33];
    int b = blockIdx.z;
    int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    const double2* A = Am + (size_t)b * M * K;
    const double2* B = Bm + (size_t)b * N * K;
    int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double2 acc[2][2] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = threadIdx.x; i < 32 * 16; i += 256) {
            int row = i / 16, kk = i % 16;
            int gm = m0 + row, gn = n0 + row, gk = k0 + kk;
            sA[kk][row] = (gm < M && gk < K) ? A[(size_t)gm * K + gk] : make_double2(0, 0);
            sB[kk][row] = (gn < N && gk < K) ? B[(size_t)gn * K + gk] : make_double2(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double2 a0 = sA[kk][ty], a1 = sA[kk][ty + 16];
            double2 b0 = sB[kk][tx], b1 = sB[kk][tx + 16];
            cfma(acc[0][0], a0, b0);
            cfma(acc[0][1], a0, b1);
            cfma(acc[1][0], a1, b0);
            cfma(acc[1][1], a1, b1);
        }
        __syncthreads();
    }
    for (int i = 0; i < 2; ++i)
        for (int jj = 0; jj < 2; ++jj) {
            int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * jj;
            if (gm < M && gn < N) Cm[((size_t)b * M + gm) * N + gn] = acc[i][jj];
        }
}

// Skinny GEMM for N <= 4 (zero-part right tile): one warp per row m.
__global__ void k_zgemm_skinny_f64(const double2* __restrict__ Am, const double2* __restrict__ Bm,
                                   double2* __restrict__ Cm, int M, int N, int K, int batch) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= M * batch) return;
    int b = warp / M, m = warp % M;
    const double2* a = Am + ((size_t)b * M + m) * K;
    const double2* B = Bm + (size_t)b * N * K;
    double2 acc[4] = {};
    for (int k = lane; k < K; k += 32) {
        double2 av = a[k];
        for (int n = 0; n < N; ++n) cfma(acc[n], av, B[(size_t)n * K + k]);
    }
    for (int n = 0; n < N; ++n)
        for (int o = 16; o > 0; o >>= 1) {
            acc[n].x += __shfl_xor_sync(0xffffffffu, acc[n].x, o);
            acc[n].y += __shfl_xor_sync(0xffffffffu, acc[n].y, o);
        }
    if (lane == 0)
        for (int n = 0; n < N; ++n) Cm[((size_t)b * M + m) * N + n] = acc[n];
}

// out class array <- alpha * G + beta * out; G[wl][(vL, A)][(vR, C)]
__global__ void k_scatter(ClassJob J, int cls, const double2* __restrict__ Gm, void* out, int dt, double alpha,
                          double beta) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)J.nw_chunk * J.nL * J.nR * 16;
    if (idx >= total) return;
    int o = idx % 16;
    size_t rest = idx / 16;
    int vR = rest % J.nR;
    rest /= J.nR;
    int vL = rest % J.nL;
    int wl = rest / J.nL;
    // find (A, C) with cO[A][C] == o
    const ChannelMaps& M = c_maps[J.r];
    int A = 0, C = 0;
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 4; ++c)
            if (M.cO[a][c] == o) { A = a; C = c; }
    int Mrows = 4 * J.nL, Ncols = 4 * J.nR;
    double2 gv = Gm[((size_t)wl * Mrows + 4 * vL + A) * Ncols + 4 * vR + C];
    // output element index in the class layout
    size_t w = J.w0 + wl, e;
    if (cls == KB_K1) e = w * 16 + o;
    else if (cls == KB_K2) e = (w * J.nL + vL) * 16 + o;
    else if (cls == KB_K2P) e = (w * J.nR + vR) * 16 + o;
    else e = ((w * J.nL + vL) * J.nR + vR) * 16 + o;
    if (dt == KB_DT_C128) {
        double2* p = reinterpret_cast<double2*>(out) + e;
        double2 old = beta != 0.0 ? *p : make_double2(0, 0);
        *p = make_double2(alpha * gv.x + beta * old.x, alpha * gv.y + beta * old.y);
    } else {
        float2* p = reinterpret_cast<float2*>(out) + e;
        float2 old = beta != 0.0 ? *p : make_float2(0, 0);
        *p = make_float2((float)(alpha * gv.x + beta * old.x), (float)(alpha * gv.y + beta * old.y));
    }
}

}  // namespace kb

using namespace kb;

static bool g_maps_uploaded[64] = {};

static kb_status upload_maps(kb_ctx* ctx) {
    if (g_maps_uploaded[ctx->device]) return KB_OK;
    ChannelMaps h[3] = {channel_maps(0), channel_maps(1), channel_maps(2)};
    KB_CUDA_TRY(ctx, cudaMemcpyToSymbol(c_maps, h, sizeof(h)));
    g_maps_uploaded[ctx->device] = true;
    return KB_OK;
}

// Shapes of one output class: rows of the left tile, rows of the right tile, grids.
void class_shape(const Grids& g, int cls, int& nw, int& nL, int& nR, int& nvg) {
    if (cls == KB_K1) { nw = g.n1; nL = 1; nR = 1; nvg = 1; }
    else if (cls == KB_K2) { nw = g.n2w; nL = g.n2v; nR = 1; nvg = g.n2v; }
    else if (cls == KB_K2P) { nw = g.n2w; nL = 1; nR = g.n2v; nvg = g.n2v; }
    else { nw = g.n3w; nL = g.n3v; nR = g.n3v; nvg = g.n3v; }
}

// Bytes per bosonic frequency of the FP64 class pipeline (Pi table, both tiles, product)
// and the frequencies processed per chunk within the context's workspace limit.
static void fp64_chunking(const kb_ctx* ctx, int r, int cls, size_t& per_w, int& chunk) {
    const Grids& g = ctx->g;
    size_t K = (size_t)4 * ((r == KB_CH_T) ? 2 : 1) * g.nq;
    int nw, nL, nR, nvg;
    class_shape(g, cls, nw, nL, nR, nvg);
    per_w = (size_t)g.nq * 16 * sizeof(double2) + (size_t)4 * nL * K * sizeof(double2) +
            (size_t)4 * nR * K * sizeof(double2) + (size_t)16 * nL * nR * sizeof(double2);
    chunk = (int)std::max<size_t>(1, std::min<size_t>(nw, ctx->ws_limit / per_w));
}

size_t kb_fp64_workspace_need(const kb_ctx* ctx, int r, unsigned mask) {
    size_t need = 0;
    for (int cls = 0; cls < 4; ++cls)
        if ((mask >> cls) & 1) {
            size_t per_w;
            int chunk;
            fp64_chunking(ctx, r, cls, per_w, chunk);
            need = std::max(need, per_w * chunk);
        }
    return need;
}

kb_status kb_fp64_prepare(kb_ctx* ctx) { return upload_maps(ctx); }

kb_status kb_bubble_fp64(kb_ctx* ctx, int r, int sl, int sr, int so, int pi_kind, unsigned mask, double alpha,
                         double beta, cudaStream_t st) {
    kb_status s = upload_maps(ctx);
    if (s != KB_OK) return s;
    const Grids& g = ctx->g;
    int ns = (r == KB_CH_T) ? 2 : 1;
    size_t K = (size_t)4 * ns * g.nq;
    // classes that vanish identically (a side without bare part and without channel r)
    const unsigned zero = kb_zero_classes(ctx, r, sl, sr, mask);
    s = kb_scale_classes(ctx, r, so, zero, beta, st);
    if (s != KB_OK) return s;
    mask &= ~zero;
    for (int cls = 0; cls < 4; ++cls) {
        if (!((mask >> cls) & 1)) continue;
        int nw, nL, nR, nvg;
        class_shape(g, cls, nw, nL, nR, nvg);
        size_t per_w;
        int chunk;
        fp64_chunking(ctx, r, cls, per_w, chunk);
        s = kb_ensure_workspace(ctx, per_w * chunk, st);
        if (s != KB_OK) return s;
        char* base = static_cast<char*>(ctx->ws.ptr);
        double2* Pi = reinterpret_cast<double2*>(base);
        double2* Lt = Pi + (size_t)chunk * g.nq * 16;
        double2* Rt = Lt + (size_t)chunk * 4 * nL * K;
        double2* Gm = Rt + (size_t)chunk * 4 * nR * K;
        for (int w0 = 0; w0 < nw; w0 += chunk) {
            ClassJob J;
            J.r = r; J.pi_kind = pi_kind; J.ns = ns; J.nq = g.nq;
            J.nw_chunk = std::min(chunk, nw - w0); J.w0 = w0; J.nw_grid = nw;
            J.nL = nL; J.nR = nR; J.nvL_grid = nvg; J.nvR_grid = nvg;
            J.L_nu = (cls == KB_K2 || cls == KB_K3);
            J.R_nu = (cls == KB_K2P || cls == KB_K3);
            {
                KB_LAUNCH(ctx, st, "k_pi_table");
                dim3 bp((g.nq + 127) / 128, J.nw_chunk);
                k_pi_table<<<bp, 128, 0, st>>>(ctx->m, J, g.A, ctx->d_xq, ctx->d_wq, Pi);
            }
            {
                KB_LAUNCH(ctx, st, "k_gather_f64_left");
                dim3 bl((g.nq + 127) / 128, nL * ns, J.nw_chunk);
                k_gather_f64<false><<<bl, 128, 0, st>>>(ctx->slots[sl], g, J, ctx->d_xq, Pi, Lt);
            }
            {
                KB_LAUNCH(ctx, st, "k_gather_f64_right");
                dim3 br((g.nq + 127) / 128, nR * ns, J.nw_chunk);
                k_gather_f64<true><<<br, 128, 0, st>>>(ctx->slots[sr], g, J, ctx->d_xq, Pi, Rt);
            }
            int Mr = 4 * nL, Nc = 4 * nR;
            if (Nc <= 4) {
                KB_LAUNCH(ctx, st, "k_zgemm_skinny_f64");
                int warps = Mr * J.nw_chunk;
                k_zgemm_skinny_f64<<<(warps * 32 + 255) / 256, 256, 0, st>>>(Lt, Rt, Gm, Mr, Nc, (int)K, J.nw_chunk);
            } else {
                KB_LAUNCH(ctx, st, "k_zgemm_f64");
                dim3 bg((Nc + 31) / 32, (Mr + 31) / 32, J.nw_chunk);
                k_zgemm_f64<<<bg, 256, 0, st>>>(Lt, Rt, Gm, Mr, Nc, (int)K);
            }
            {
                KB_LAUNCH(ctx, st, "k_scatter");
                size_t tot = (size_t)J.nw_chunk * nL * nR * 16;
                k_scatter<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
                    J, cls, Gm, const_cast<void*>(ctx->slots[so].cls[r][cls]), ctx->slots[so].dt[r][cls], alpha, beta);
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { ctx->err = std::string("fp64 launch: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
        }
    }
    return KB_OK;
}

// ---------------------------------------------------------------------------------------
// Allocation-free entry point (kb_bubble_fp64_noalloc in include/kb.h).  The scratch of the
// FP64 class pipeline lives in this fixed device array instead of a cudaMalloc'ed
// workspace.  Host code must not pass the array's name to a kernel (on the host it is only
// a stand-in); its device address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_kb_noalloc_scratch[KB_NOALLOC_SCRATCH_BYTES];

namespace kb {
// Composite 5-point Gauss-Lobatto nodes and weights on [-1, 1] (same rule as kb_set_grids).
__global__ void k_gl5_table(int nq, double* __restrict__ x, double* __restrict__ w) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq) return;
    int P = (nq - 1) / 4, p = j / 4, q = j % 4;
    double h = 2.0 / P;
    const double t[4] = {-1.0, -0.65465367070797714380, 0.0, 0.65465367070797714380};   // sqrt(3/7)
    const double u[4] = {0.1, 49.0 / 90.0, 32.0 / 45.0, 49.0 / 90.0};
    if (j == nq - 1) { x[j] = 1.0; w[j] = 0.05 * h; return; }
    x[j] = (j == 0) ? -1.0 : -1.0 + p * h + (t[q] + 1.0) * 0.5 * h;
    w[j] = u[q] * 0.5 * h * ((q == 0 && p > 0) ? 2.0 : 1.0);
}
}  // namespace kb

static void* g_noalloc_ptr[64] = {};
static bool g_noalloc_ready[64] = {};

static kb_status noalloc_setup(int dev) {
    if (dev < 0 || dev >= 64) return KB_ERR_ARG;
    if (g_noalloc_ready[dev]) return KB_OK;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_kb_noalloc_scratch) != cudaSuccess || !p) return KB_ERR_CUDA;
    ChannelMaps h[3] = {channel_maps(0), channel_maps(1), channel_maps(2)};
    if (cudaMemcpyToSymbol(c_maps, h, sizeof(h)) != cudaSuccess) return KB_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
    g_noalloc_ready[dev] = true;
    return KB_OK;
}

extern "C" kb_status kb_bubble_fp64_noalloc(const kb_grid_desc* gd, double Delta, double T, double eps,
                                            const kb_vertex_desc* left, const kb_vertex_desc* right, int r,
                                            int pi_kind, int cls, void* out, int out_dtype, double alpha,
                                            double beta, void* stream) {
    if (!gd || !left || !right || !out || r < 0 || r > 2 || cls < 0 || cls > 3 ||
        (pi_kind != KB_PI_GG && pi_kind != KB_PI_GS_SG) || (out_dtype != KB_DT_C128 && out_dtype != KB_DT_C64) ||
        !(Delta > 0) || !(T >= 0) || !std::isfinite(eps) || !std::isfinite(alpha) || !std::isfinite(beta) ||
        gd->n1 < 1 || gd->n2w < 1 || gd->n2v < 1 || gd->n3w < 1 || gd->n3v < 1 || gd->nq < 5 ||
        (gd->nq - 1) % 4 || !(gd->A > 0) || left->channels > 7 || right->channels > 7)
        return KB_ERR_ARG;
    // a launch error left pending by earlier work is not this call's to report or clear
    if (cudaPeekAtLastError() != cudaSuccess) return KB_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return KB_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    {
        // the scratch address is per device: the stream must belong to the current device
        int sdev = -1;
        if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) return KB_ERR_CUDA;
        if (sdev != dev) return KB_ERR_ARG;
    }
    kb_status s = noalloc_setup(dev);
    if (s != KB_OK) return s;
    Grids g{gd->n1, gd->n2w, gd->n2v, gd->n3w, gd->n3v, gd->nq, gd->A};
    Model m{Delta, T, eps, 0, 1.0, nullptr, nullptr};
    VertexDev V[2]{};
    const kb_vertex_desc* D[2] = {left, right};
    for (int i = 0; i < 2; ++i) {
        V[i].has_R = D[i]->has_R ? 1 : 0;
        V[i].mask = (int)D[i]->channels;
        V[i].bare = -0.5 * D[i]->U;
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 4; ++k) {
                V[i].cls[c][k] = D[i]->cls[c][k];
                V[i].dt[c][k] = D[i]->dtype[c][k];
                if (V[i].dt[c][k] != KB_DT_C128 && V[i].dt[c][k] != KB_DT_C64) return KB_ERR_ARG;
            }
    }
    int ns = (r == KB_CH_T) ? 2 : 1;
    size_t K = (size_t)4 * ns * g.nq;
    int nw, nL, nR, nvg;
    class_shape(g, cls, nw, nL, nR, nvg);
    size_t table = 2 * sizeof(double) * ((g.nq + 31) / 32 * 32);
    size_t per_w = (size_t)g.nq * 16 * sizeof(double2) + (size_t)4 * nL * K * sizeof(double2) +
                   (size_t)4 * nR * K * sizeof(double2) + (size_t)16 * nL * nR * sizeof(double2);
    if (table + per_w > KB_NOALLOC_SCRATCH_BYTES) return KB_ERR_TOO_LARGE;
    int chunk = (int)std::min<size_t>(nw, (KB_NOALLOC_SCRATCH_BYTES - table) / per_w);
    char* base = static_cast<char*>(g_noalloc_ptr[dev]);
    double* xq = reinterpret_cast<double*>(base);
    double* wq = xq + (g.nq + 31) / 32 * 32;
    double2* Pi = reinterpret_cast<double2*>(base + table);
    double2* Lt = Pi + (size_t)chunk * g.nq * 16;
    double2* Rt = Lt + (size_t)chunk * 4 * nL * K;
    double2* Gm = Rt + (size_t)chunk * 4 * nR * K;
    k_gl5_table<<<(g.nq + 127) / 128, 128, 0, st>>>(g.nq, xq, wq);
    if (cudaGetLastError() != cudaSuccess) return KB_ERR_CUDA;
    for (int w0 = 0; w0 < nw; w0 += chunk) {
        ClassJob J;
        J.r = r; J.pi_kind = pi_kind; J.ns = ns; J.nq = g.nq;
        J.nw_chunk = std::min(chunk, nw - w0); J.w0 = w0; J.nw_grid = nw;
        J.nL = nL; J.nR = nR; J.nvL_grid = nvg; J.nvR_grid = nvg;
        J.L_nu = (cls == KB_K2 || cls == KB_K3);
        J.R_nu = (cls == KB_K2P || cls == KB_K3);
        k_pi_table<<<dim3((g.nq + 127) / 128, J.nw_chunk), 128, 0, st>>>(m, J, g.A, xq, wq, Pi);
        k_gather_f64<false><<<dim3((g.nq + 127) / 128, nL * ns, J.nw_chunk), 128, 0, st>>>(V[0], g, J, xq, Pi, Lt);
        k_gather_f64<true><<<dim3((g.nq + 127) / 128, nR * ns, J.nw_chunk), 128, 0, st>>>(V[1], g, J, xq, Pi, Rt);
        int Mr = 4 * nL, Nc = 4 * nR;
        if (Nc <= 4)
            k_zgemm_skinny_f64<<<(Mr * J.nw_chunk * 32 + 255) / 256, 256, 0, st>>>(Lt, Rt, Gm, Mr, Nc, (int)K,
                                                                                    J.nw_chunk);
        else
            k_zgemm_f64<<<dim3((Nc + 31) / 32, (Mr + 31) / 32, J.nw_chunk), 256, 0, st>>>(Lt, Rt, Gm, Mr, Nc, (int)K);
        size_t tot = (size_t)J.nw_chunk * nL * nR * 16;
        k_scatter<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(J, cls, Gm, out, out_dtype, alpha, beta);
        // stop at the first chunk whose launches failed (the entry check above guarantees
        // that the error, if any, comes from this call's launches)
        if (cudaGetLastError() != cudaSuccess) return KB_ERR_CUDA;
    }
    return KB_OK;
}
