// Vertex arithmetic between slots: the sums the multiloop step needs between its bubbles
// (Sec. III.C: the l-loop derivative of channel r is the sum of its left, central and right
// parts, and the left part is also the right vertex of the next order's central part, so it
// is computed once into its own slot and added).
#include <algorithm>
#include <cstdio>
#include <string>

#include "kb_internal.h"

namespace kb {
namespace {

template <typename TS, typename TD>
__global__ void k_class_add(const TS* __restrict__ src, TD* __restrict__ dst, size_t n, double alpha) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double sx = (double)src[2 * i], sy = (double)src[2 * i + 1];
        dst[2 * i] = (TD)((double)dst[2 * i] + alpha * sx);
        dst[2 * i + 1] = (TD)((double)dst[2 * i + 1] + alpha * sy);
    }
}

size_t class_points(const Grids& g, int k) {
    switch (k) {
        case 0: return (size_t)g.n1;
        case 1:
        case 2: return (size_t)g.n2w * g.n2v;
        default: return (size_t)g.n3w * g.n3v * g.n3v;
    }
}

}  // namespace
}  // namespace kb

using namespace kb;

kb_status kb_vertex_add_impl(kb_ctx* ctx, int channel, int src, int dst, unsigned mask, double alpha,
                             cudaStream_t st) {
    if (!ctx) return KB_ERR_ARG;
    if (channel < 0 || channel > 2 || src < 0 || src >= KB_MAX_SLOTS || dst < 0 || dst >= KB_MAX_SLOTS ||
        (mask & ~KB_MASK_ALL)) {
        ctx->err = "kb_vertex_add: argument out of range";
        return KB_ERR_ARG;
    }
    if (!ctx->grids_set) {
        ctx->err = "kb_vertex_add: set grids first";
        return KB_ERR_STATE;
    }
    if (src == dst) {
        ctx->err = "kb_vertex_add: source and destination are the same slot";
        return KB_ERR_ARG;
    }
    const VertexDev& S = ctx->slots[src];
    const VertexDev& D = ctx->slots[dst];
    for (int k = 0; k < 4; ++k) {
        if (!((mask >> k) & 1) || !S.cls[channel][k]) continue;   // absent source classes read zero
        if (!D.cls[channel][k]) {
            ctx->err = "kb_vertex_add: destination class not attached";
            return KB_ERR_ARG;
        }
        if (S.cls[channel][k] == D.cls[channel][k]) {
            ctx->err = "kb_vertex_add: source and destination class alias";
            return KB_ERR_ARG;
        }
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return KB_ERR_CUDA;
    for (int k = 0; k < 4; ++k) {
        if (!((mask >> k) & 1) || !S.cls[channel][k]) continue;
        const size_t n = class_points(ctx->g, k) * 16;
        const int threads = 256;
        const int blocks = (int)std::min<size_t>((n + threads - 1) / threads, (size_t)152 * 8);
        KB_LAUNCH(ctx, st, "k_class_add");
        const bool s64 = S.dt[channel][k] == KB_DT_C64, d64 = D.dt[channel][k] == KB_DT_C64;
        const void* sp = S.cls[channel][k];
        void* dp = const_cast<void*>(D.cls[channel][k]);
        if (s64 && d64)
            k_class_add<float, float><<<blocks, threads, 0, st>>>((const float*)sp, (float*)dp, n, alpha);
        else if (s64)
            k_class_add<float, double><<<blocks, threads, 0, st>>>((const float*)sp, (double*)dp, n, alpha);
        else if (d64)
            k_class_add<double, float><<<blocks, threads, 0, st>>>((const double*)sp, (float*)dp, n, alpha);
        else
            k_class_add<double, double><<<blocks, threads, 0, st>>>((const double*)sp, (double*)dp, n, alpha);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            ctx->err = std::string("kb_vertex_add: ") + cudaGetErrorString(e);
            return KB_ERR_CUDA;
        }
    }
    return KB_OK;
}

extern "C" kb_status kb_vertex_add(kb_ctx* ctx, int channel, int slot_src, int slot_dst, unsigned class_mask,
                                   double alpha, void* stream) {
    return kb_vertex_add_impl(ctx, channel, slot_src, slot_dst, class_mask, alpha,
                              reinterpret_cast<cudaStream_t>(stream));
}

// Classes of a bubble that vanish identically: the r-independent parts L0 = R + K1_r + K2'_r
// of the left vertex and R0 = R + K1_r + K2_r of the right one are zero when a slot has no
// bare part and leaves channel r out of its channel mask (the vertex gamma_rbar of the
// multiloop parts, the directions of the parquet Jacobian); then K1 = L0 Pi R0 and
// K2' = L0 Pi R^v' (left) or K2 = L^v Pi R0 (right) are zero.
unsigned kb_zero_classes(const kb_ctx* ctx, int r, int sl, int sr, unsigned mask) {
    unsigned zero = 0;
    const VertexDev& L = ctx->slots[sl];
    const VertexDev& R = ctx->slots[sr];
    if (!L.has_R && !((L.mask >> r) & 1)) zero |= (1u << KB_K1) | (1u << KB_K2P);
    if (!R.has_R && !((R.mask >> r) & 1)) zero |= (1u << KB_K1) | (1u << KB_K2);
    return zero & mask;
}

namespace kb {
namespace {
// out <- beta * out over n complex elements (alpha * 0 + beta * out)
__global__ void k_class_scale(void* out, int dt, size_t n, double beta) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (dt == KB_DT_C128) {
            double2* p = reinterpret_cast<double2*>(out) + i;
            *p = beta != 0.0 ? make_double2(beta * p->x, beta * p->y) : make_double2(0.0, 0.0);
        } else {
            float2* p = reinterpret_cast<float2*>(out) + i;
            *p = beta != 0.0 ? make_float2((float)(beta * p->x), (float)(beta * p->y)) : make_float2(0.f, 0.f);
        }
    }
}
}  // namespace
}  // namespace kb

kb_status kb_scale_classes(kb_ctx* ctx, int r, int so, unsigned classes, double beta, cudaStream_t st) {
    if (!classes || beta == 1.0) return KB_OK;
    const VertexDev& O = ctx->slots[so];
    for (int k = 0; k < 4; ++k) {
        if (!((classes >> k) & 1)) continue;
        const size_t n = class_points(ctx->g, k) * 16;
        KB_LAUNCH(ctx, st, "k_class_scale");
        k_class_scale<<<(unsigned)std::min<size_t>((n + 255) / 256, (size_t)152 * 8), 256, 0, st>>>(
            const_cast<void*>(O.cls[r][k]), O.dt[r][k], n, beta);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("zero classes: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}

// ---------------------------------------------------------------------------------------
// Symmetry image of a channel's classes (Sec. II.G.3): for a conjugation- and
// crossing-symmetric pair of vertices the right multiloop part B_r(Γ, X) is the image of the
// left one B_r(X, Γ) — the conjugation in a and p ((w, v, v') -> (w, v', v), Keldysh
// (a1'a2'|a1a2) -> (a1a2|a1'a2'), complex conjugate, sign (-1)^(1+Σa)), the conjugation after
// crossing in t (the same w, v <-> v', both Keldysh permutations).  K2 and K2' trade places.
namespace kb {
namespace {

__host__ __device__ constexpr int img_perm_c(int c) { return ((c & 3) << 2) | (c >> 2); }
__host__ __device__ constexpr int img_perm_x(int c) {
    return (((c >> 2) & 1) << 3) | (((c >> 3) & 1) << 2) | ((c & 1) << 1) | ((c >> 1) & 1);
}
__host__ __device__ constexpr double img_sign(int c) {
    return (((c & 1) + ((c >> 1) & 1) + ((c >> 2) & 1) + ((c >> 3) & 1)) & 1) ? 1.0 : -1.0;
}

// dst class of layout [nw][nv][nvp][16] from the src class; swap: K3 (v, v') -> (v', v)
template <typename T>
__global__ void k_class_image(T* __restrict__ dst, const T* __restrict__ src, int t_channel, int swap, int nw, int nv,
                              int nvp) {
    const size_t total = (size_t)nw * nv * nvp * 16;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % 16);
        size_t rest = i / 16;
        const int ip = (int)(rest % nvp);
        rest /= nvp;
        const int iv = (int)(rest % nv);
        const int iw = (int)(rest / nv);
        const int pc = t_channel ? img_perm_x(img_perm_c(c)) : img_perm_c(c);
        const size_t se = swap ? ((((size_t)iw * nv + ip) * nvp + iv) * 16 + pc) : ((i / 16) * 16 + pc);
        const double sg = img_sign(c);
        const T v = src[se];
        dst[i] = T{(decltype(v.x))(sg * v.x), (decltype(v.x))(-sg * v.y)};
    }
}

}  // namespace
}  // namespace kb

kb_status kb_vertex_image_impl(kb_ctx* ctx, int channel, int src, int dst, unsigned mask, cudaStream_t st) {
    if (!ctx) return KB_ERR_ARG;
    if (channel < 0 || channel > 2 || src < 0 || src >= KB_MAX_SLOTS || dst < 0 || dst >= KB_MAX_SLOTS ||
        src == dst || (mask & ~KB_MASK_ALL)) {
        ctx->err = "kb_vertex_image: argument out of range";
        return KB_ERR_ARG;
    }
    if (!ctx->grids_set) { ctx->err = "kb_vertex_image: set grids first"; return KB_ERR_STATE; }
    const VertexDev& S = ctx->slots[src];
    const VertexDev& D = ctx->slots[dst];
    const Grids& g = ctx->g;
    // destination class k is the image of source class from[k]
    const int from[4] = {KB_K1, KB_K2P, KB_K2, KB_K3};
    for (int k = 0; k < 4; ++k) {
        if (!((mask >> k) & 1)) continue;
        const int ks = from[k];
        if (!D.cls[channel][k] || !S.cls[channel][ks] || D.dt[channel][k] != S.dt[channel][ks] ||
            D.cls[channel][k] == S.cls[channel][ks]) {
            ctx->err = "kb_vertex_image: classes must be attached, of one dtype and distinct";
            return KB_ERR_ARG;
        }
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return KB_ERR_CUDA;
    for (int k = 0; k < 4; ++k) {
        if (!((mask >> k) & 1)) continue;
        const int ks = from[k];
        int nw = g.n1, nv = 1, nvp = 1;
        if (k == KB_K2 || k == KB_K2P) { nw = g.n2w; nv = g.n2v; }
        if (k == KB_K3) { nw = g.n3w; nv = g.n3v; nvp = g.n3v; }
        const size_t total = (size_t)nw * nv * nvp * 16;
        const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)152 * 8);
        const int tch = channel == KB_CH_T, swap = k == KB_K3;
        KB_LAUNCH(ctx, st, "k_class_image");
        if (D.dt[channel][k] == KB_DT_C64)
            k_class_image<float2><<<blocks, 256, 0, st>>>((float2*)D.cls[channel][k], (const float2*)S.cls[channel][ks],
                                                          tch, swap, nw, nv, nvp);
        else
            k_class_image<double2><<<blocks, 256, 0, st>>>((double2*)D.cls[channel][k],
                                                           (const double2*)S.cls[channel][ks], tch, swap, nw, nv, nvp);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("kb_vertex_image: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}

extern "C" kb_status kb_vertex_image(kb_ctx* ctx, int channel, int slot_src, int slot_dst, unsigned class_mask,
                                     void* stream) {
    return kb_vertex_image_impl(ctx, channel, slot_src, slot_dst, class_mask, reinterpret_cast<cudaStream_t>(stream));
}
