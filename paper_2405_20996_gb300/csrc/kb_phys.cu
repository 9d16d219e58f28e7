// Physical-only Keldysh structure of a vertex (Sec. II.E.2 FDRs, Sec. II.G.3 symmetries).
//
// In the parquet approximation every class of a channel keeps the structure of the bare
// vertex, which depends on the parity of the quantum indices only: writing a component
// c = (a1', a2', a1, a2) of channel r's 4x4 form as (left pair, right pair) — a: (a1', a2),
// (a1, a2'); p: (a1', a2'), (a1, a2); t: (a1', a1), (a2', a2) — K1 depends on the two
// pairs' parities alone (4 distinct numbers of 16), K2 on the left pair and the right
// parity (8), K2' on the left parity and the right pair (8), K3 on both pairs (16).  In
// thermal equilibrium K1 in addition has a vanishing all-even block (causality), an
// advanced block that is the conjugate of the retarded one, and a Keldysh block fixed by
// the bosonic FDR, tanh(w/2T) K1^K = K1^R - K1^A; the retarded block is the one of
// component 1 (a, t) or 8 (p), the advanced block its mirror, the Keldysh block odd-odd.
//
//   k_phys_check   residuals of these relations (max deviation / max |class|)
//   k_phys_pack    the distinct components of a class, in the compact order d(c)
//   k_phys_unpack  the class from its distinct components
// Compact index d(c): K1 2 pl + pr; K2 4 x + 2 y + pr (x, y the left pair's indices); K2'
// 4 pl + 2 x' + y' (x', y' the right pair's); K3 c.  The representative of d is the smallest
// component with that index.
#include <cmath>
#include <string>

#include "kb_internal.h"

namespace kb {
namespace {

__device__ __forceinline__ double2 ld_cc(const void* p, int dt, size_t i) {
    if (dt == KB_DT_C128) return reinterpret_cast<const double2*>(p)[i];
    const float2 v = reinterpret_cast<const float2*>(p)[i];
    return make_double2(v.x, v.y);
}

__host__ __device__ inline int pair_bits(int r, int c, int side, int which) {
    const int b[4] = {(c >> 3) & 1, (c >> 2) & 1, (c >> 1) & 1, c & 1};     // a1', a2', a1, a2
    // legs of the left / right pair of channel r, in the order (first, second)
    const int L[3][2] = {{0, 3}, {0, 1}, {0, 2}}, R[3][2] = {{2, 1}, {2, 3}, {1, 3}};
    return b[side ? R[r][which] : L[r][which]];
}

__host__ __device__ inline int compact_index(int r, int k, int c) {
    const int x = pair_bits(r, c, 0, 0), y = pair_bits(r, c, 0, 1);
    const int xp = pair_bits(r, c, 1, 0), yp = pair_bits(r, c, 1, 1);
    const int pl = x ^ y, pr = xp ^ yp;
    if (k == KB_K1) return 2 * pl + pr;
    if (k == KB_K2) return 4 * x + 2 * y + pr;
    if (k == KB_K2P) return 4 * pl + 2 * xp + yp;
    return c;
}

__host__ __device__ inline int compact_size(int k) { return k == KB_K1 ? 4 : (k == KB_K3 ? 16 : 8); }

__host__ __device__ inline int representative(int r, int k, int d) {
    for (int c = 0; c < 16; ++c)
        if (compact_index(r, k, c) == d) return c;
    return 0;
}

__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }

// res[2k] = max |X_c - X_rep(d(c))|, res[2k+1] = max |X| over the class's records.
__global__ void k_phys_check(const void* __restrict__ X, int dt, int r, int k, size_t nrec, double* __restrict__ res) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dev = 0.0, mag = 0.0;
    if (i < nrec * 16) {
        const int c = (int)(i % 16);
        const size_t rec = i / 16;
        const double2 v = ld_cc(X, dt, i), u = ld_cc(X, dt, rec * 16 + representative(r, k, compact_index(r, k, c)));
        dev = cabs2(make_double2(v.x - u.x, v.y - u.y));
        mag = cabs2(v);
    }
    for (int o = 16; o; o >>= 1) {
        dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
        mag = fmax(mag, __shfl_xor_sync(0xffffffffu, mag, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(res + 2 * k, dev);
        atomic_max_nonneg(res + 2 * k + 1, mag);
    }
}

// K1 equilibrium relations per bosonic frequency w_i (grid frequency of node i):
// res[8] causality max |X on the all-even block|, res[9] conjugation max |A - R*|,
// res[10] FDR max |tanh(w/2T) K - (R - A)|.
__global__ void k_phys_k1(const void* __restrict__ X, int dt, int r, int n1, double A, double T, double* __restrict__ res) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double caus = 0.0, conj = 0.0, fdr = 0.0;
    if (i < n1) {
        const double x = -1.0 + 2.0 * (i + 1) / (double)(n1 + 1);
        const double w = A * tan(0.5 * 3.14159265358979323846 * x);
        const int cR = (r == KB_CH_P) ? 8 : 1;
        const int dR = compact_index(r, KB_K1, cR);
        const int dA = 2 * (dR & 1) + (dR >> 1);               // mirrored parities
        const double2 R = ld_cc(X, dt, (size_t)i * 16 + cR);
        const double2 Av = ld_cc(X, dt, (size_t)i * 16 + representative(r, KB_K1, dA));
        const double2 K = ld_cc(X, dt, (size_t)i * 16 + representative(r, KB_K1, 3));
        const double2 Z = ld_cc(X, dt, (size_t)i * 16 + representative(r, KB_K1, 0));
        const double th = (T > 0.0) ? tanh(w / (2.0 * T)) : (w > 0.0 ? 1.0 : (w < 0.0 ? -1.0 : 0.0));
        caus = cabs2(Z);
        conj = cabs2(make_double2(Av.x - R.x, Av.y + R.y));
        fdr = cabs2(make_double2(th * K.x - (R.x - Av.x), th * K.y - (R.y - Av.y)));
    }
    for (int o = 16; o; o >>= 1) {
        caus = fmax(caus, __shfl_xor_sync(0xffffffffu, caus, o));
        conj = fmax(conj, __shfl_xor_sync(0xffffffffu, conj, o));
        fdr = fmax(fdr, __shfl_xor_sync(0xffffffffu, fdr, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(res + 8, caus);
        atomic_max_nonneg(res + 9, conj);
        atomic_max_nonneg(res + 10, fdr);
    }
}

template <typename T2>
__global__ void k_phys_pack(const T2* __restrict__ X, int r, int k, size_t nrec, T2* __restrict__ out) {
    const int nd = compact_size(k);
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrec * nd) return;
    const int d = (int)(i % nd);
    out[i] = X[(i / nd) * 16 + representative(r, k, d)];
}

template <typename T2>
__global__ void k_phys_unpack(const T2* __restrict__ src, int r, int k, size_t nrec, T2* __restrict__ X) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrec * 16) return;
    X[i] = src[(i / 16) * compact_size(k) + compact_index(r, k, (int)(i % 16))];
}

size_t class_records(const Grids& g, int k) {
    if (k == KB_K1) return (size_t)g.n1;
    if (k == KB_K3) return (size_t)g.n3w * g.n3v * g.n3v;
    return (size_t)g.n2w * g.n2v;
}

kb_status phys_args(kb_ctx* ctx, int slot, int channel, int cls, const char* who) {
    if (!ctx) return KB_ERR_ARG;
    if (slot < 0 || slot >= KB_MAX_SLOTS || channel < 0 || channel > 2 || cls < -1 || cls > 3) {
        ctx->err = std::string(who) + ": argument out of range";
        return KB_ERR_ARG;
    }
    if (!ctx->grids_set || !ctx->slot_set[slot]) {
        ctx->err = std::string(who) + ": set the grids and the slot first";
        return KB_ERR_STATE;
    }
    if (cls >= 0 && !ctx->slots[slot].cls[channel][cls]) {
        ctx->err = std::string(who) + ": class not attached";
        return KB_ERR_STATE;
    }
    return cudaSetDevice(ctx->device) == cudaSuccess ? KB_OK : KB_ERR_CUDA;
}

}  // namespace
}  // namespace kb

using namespace kb;

extern "C" kb_status kb_keldysh_check(kb_ctx* ctx, int slot, int channel, double T, double* out, void* stream) {
    kb_status s = phys_args(ctx, slot, channel, -1, "kb_keldysh_check");
    if (s != KB_OK) return s;
    if (!out || !(T >= 0.0) || !std::isfinite(T)) { ctx->err = "kb_keldysh_check: bad output or temperature"; return KB_ERR_ARG; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    s = kb_ensure_workspace(ctx, 16 * sizeof(double), st);
    if (s != KB_OK) return s;
    double* res = static_cast<double*>(ctx->ws.ptr);
    KB_CUDA_TRY(ctx, cudaMemsetAsync(res, 0, 16 * sizeof(double), st));
    const VertexDev& V = ctx->slots[slot];
    for (int k = 0; k < 4; ++k) {
        if (!V.cls[channel][k]) continue;
        const size_t nrec = class_records(ctx->g, k);
        KB_LAUNCH(ctx, st, "k_phys_check");
        k_phys_check<<<(unsigned)((nrec * 16 + 255) / 256), 256, 0, st>>>(V.cls[channel][k], V.dt[channel][k], channel,
                                                                          k, nrec, res);
    }
    if (V.cls[channel][KB_K1]) {
        KB_LAUNCH(ctx, st, "k_phys_k1");
        k_phys_k1<<<(ctx->g.n1 + 127) / 128, 128, 0, st>>>(V.cls[channel][KB_K1], V.dt[channel][KB_K1], channel,
                                                           ctx->g.n1, ctx->g.A, T, res);
    }
    double h[16];
    KB_CUDA_TRY(ctx, cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, st));
    KB_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    for (int k = 0; k < 4; ++k) out[k] = h[2 * k + 1] > 0.0 ? h[2 * k] / h[2 * k + 1] : 0.0;
    const double m1 = h[1];
    for (int q = 0; q < 3; ++q) out[4 + q] = m1 > 0.0 ? h[8 + q] / m1 : 0.0;
    out[7] = 0.0;
    return KB_OK;
}

extern "C" kb_status kb_vertex_pack(kb_ctx* ctx, int slot, int channel, int cls, void* dst, void* stream) {
    kb_status s = phys_args(ctx, slot, channel, cls, "kb_vertex_pack");
    if (s != KB_OK) return s;
    if (cls < 0 || !dst) { ctx->err = "kb_vertex_pack: bad class or destination"; return KB_ERR_ARG; }
    const VertexDev& V = ctx->slots[slot];
    const size_t nrec = class_records(ctx->g, cls), n = nrec * compact_size(cls);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    KB_LAUNCH(ctx, st, "k_phys_pack");
    if (V.dt[channel][cls] == KB_DT_C128)
        k_phys_pack<double2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            static_cast<const double2*>(V.cls[channel][cls]), channel, cls, nrec, static_cast<double2*>(dst));
    else
        k_phys_pack<float2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            static_cast<const float2*>(V.cls[channel][cls]), channel, cls, nrec, static_cast<float2*>(dst));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("k_phys_pack: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}

extern "C" kb_status kb_vertex_unpack(kb_ctx* ctx, int slot, int channel, int cls, const void* src, void* stream) {
    kb_status s = phys_args(ctx, slot, channel, cls, "kb_vertex_unpack");
    if (s != KB_OK) return s;
    if (cls < 0 || !src) { ctx->err = "kb_vertex_unpack: bad class or source"; return KB_ERR_ARG; }
    const VertexDev& V = ctx->slots[slot];
    const size_t nrec = class_records(ctx->g, cls), n = nrec * 16;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    KB_LAUNCH(ctx, st, "k_phys_unpack");
    if (V.dt[channel][cls] == KB_DT_C128)
        k_phys_unpack<double2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            static_cast<const double2*>(src), channel, cls, nrec,
            static_cast<double2*>(const_cast<void*>(V.cls[channel][cls])));
    else
        k_phys_unpack<float2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            static_cast<const float2*>(src), channel, cls, nrec, static_cast<float2*>(const_cast<void*>(V.cls[channel][cls])));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("k_phys_unpack: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}
