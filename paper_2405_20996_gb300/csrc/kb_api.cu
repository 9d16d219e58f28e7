// C ABI of libkb: context, grids, model, vertex slots, dispatch (include/kb.h).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "kb_internal.h"

namespace kb {

// Keldysh index maps per channel, from the bubble's leg routing (Sec. III.B diagrams with
// the channel parametrisations of Sec. II.C.1):
//   a: Gamma1^{a1' b4' | b3 a2} G^{b3|b3'}(v''+w/2) G^{b4|b4'}(v''-w/2) Gamma2^{b3' a2' | a1 b4}
//      A = (a1', a2), B = (b4', b3), D = (b3', b4), C = (a2', a1)
//   p: Gamma1^{a1' a2' | b3 b4} G^{b3|b3'}(w/2+v'') G^{b4|b4'}(w/2-v'') Gamma2^{b3' b4' | a1 a2}
//      A = (a1', a2'), B = (b3, b4), D = (b3', b4'), C = (a1, a2)
//   t: Gamma1^{a1' b3' | a1 b4} G^{b3|b3'}(v''+w/2) G^{b4|b4'}(v''-w/2) Gamma2^{b4' a2' | b3 a2}
//      A = (a1', a1), B = (b3', b4), D = (b4', b3), C = (a2', a2)
// A pair (x, y) is the index 2x + y with 0 = classical, 1 = quantum.
static inline int comp(int b1p, int b2p, int b1, int b2) { return 8 * b1p + 4 * b2p + 2 * b1 + b2; }

ChannelMaps channel_maps(int r) {
    ChannelMaps M;
    for (int X = 0; X < 4; ++X)
        for (int Y = 0; Y < 4; ++Y) {
            int xh = X >> 1, xl = X & 1, yh = Y >> 1, yl = Y & 1;
            if (r == KB_CH_A) {
                M.cL[X][Y] = comp(xh, yh, yl, xl);   // X=A=(a1',a2), Y=B=(b4',b3)
                M.cR[X][Y] = comp(xh, yh, yl, xl);   // X=D=(b3',b4), Y=C=(a2',a1)
                M.cO[X][Y] = comp(xh, yh, yl, xl);   // X=A, Y=C
            } else if (r == KB_CH_P) {
                M.cL[X][Y] = comp(xh, xl, yh, yl);
                M.cR[X][Y] = comp(xh, xl, yh, yl);
                M.cO[X][Y] = comp(xh, xl, yh, yl);
            } else {
                M.cL[X][Y] = comp(xh, yh, xl, yl);   // A=(a1',a1), B=(b3',b4)
                M.cR[X][Y] = comp(xh, yh, xl, yl);   // D=(b4',b3), C=(a2',a2)
                M.cO[X][Y] = comp(xh, yh, xl, yl);   // A=(a1',a1), C=(a2',a2)
            }
        }
    for (int b3 = 0; b3 < 2; ++b3)
        for (int b3p = 0; b3p < 2; ++b3p)
            for (int b4 = 0; b4 < 2; ++b4)
                for (int b4p = 0; b4p < 2; ++b4p) {
                    int B, D;
                    if (r == KB_CH_A) { B = 2 * b4p + b3; D = 2 * b3p + b4; }
                    else if (r == KB_CH_P) { B = 2 * b3 + b4; D = 2 * b3p + b4p; }
                    else { B = 2 * b3p + b4; D = 2 * b4p + b3; }
                    M.piq[B][D][0] = b3; M.piq[B][D][1] = b3p; M.piq[B][D][2] = b4; M.piq[B][D][3] = b4p;
                }
    return M;
}

// Composite 5-point Gauss-Lobatto rule on [-1, 1] (nodes 0, +-sqrt(3/7), +-1 per panel).
static void gl5_nodes(int nq, std::vector<double>& x, std::vector<double>& w) {
    int P = (nq - 1) / 4;
    double h = 2.0 / P;
    const double t[5] = {-1.0, -std::sqrt(3.0 / 7.0), 0.0, std::sqrt(3.0 / 7.0), 1.0};
    const double u[5] = {0.1, 49.0 / 90.0, 32.0 / 45.0, 49.0 / 90.0, 0.1};
    x.assign(nq, 0.0);
    w.assign(nq, 0.0);
    for (int p = 0; p < P; ++p)
        for (int q = 0; q < 5; ++q) {
            int j = 4 * p + q;
            x[j] = -1.0 + p * h + (t[q] + 1.0) * 0.5 * h;
            w[j] += u[q] * 0.5 * h;
        }
    x[0] = -1.0;
    x[nq - 1] = 1.0;
}

}  // namespace kb

kb_status kb_ensure_workspace(kb_ctx* ctx, size_t bytes, cudaStream_t st, bool sync) {
    if (ctx->ws.bytes >= bytes) return KB_OK;
    if (ctx->fail_allocs > 0) {
        --ctx->fail_allocs;
        ctx->err = "workspace allocation failed (injected by kb_inject_alloc_failures)";
        return KB_ERR_OOM;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!sync && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        ctx->err = "the workspace would have to grow inside a stream capture; size it before the capture";
        return KB_ERR_STATE;
    }
    if (sync) {
        KB_CUDA_TRY(ctx, cudaDeviceSynchronize());
        st = nullptr;
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->err = std::string("workspace allocation: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? KB_ERR_OOM : KB_ERR_CUDA;
    }
    if (ctx->ws.ptr) KB_CUDA_TRY(ctx, cudaFreeAsync(ctx->ws.ptr, st));
    if (sync) KB_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    ctx->ws.ptr = p;
    ctx->ws.bytes = bytes;
    ++ctx->mem_gen;
    return KB_OK;
}

static void prof_clear(kb_ctx* ctx) {
    for (auto& r : ctx->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    ctx->prof.clear();
}

int kb_tc_take_status();

static std::vector<unsigned (*)(unsigned long long*)>& oob_registry() {
    static std::vector<unsigned (*)(unsigned long long*)> r;
    return r;
}

bool kb_oob_register(unsigned (*take)(unsigned long long*)) {
    oob_registry().push_back(take);
    return true;
}

unsigned kb_oob_take_all(unsigned long long* first) {
    unsigned total = 0;
    for (auto f : oob_registry()) {
        unsigned long long fi = 0;
        const unsigned n = f(&fi);
        if (n && !total) *first = fi;
        total += n;
    }
    return total;
}

extern "C" {

kb_status kb_create(kb_ctx** out, int device) {
    if (!out) return KB_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= device || device < 0) return KB_ERR_CUDA;
    kb_ctx* ctx = new (std::nothrow) kb_ctx();
    if (!ctx) return KB_ERR_OOM;
    ctx->device = device;
    for (int s = 0; s < KB_MAX_SLOTS; ++s) {
        std::memset(&ctx->slots[s], 0, sizeof(kb::VertexDev));
        ctx->slot_set[s] = false;
    }
    const char* lim = std::getenv("KB_WORKSPACE_MB");
    ctx->ws_limit = (size_t)(lim ? std::atof(lim) : 4096.0) * (1ull << 20);
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return KB_ERR_CUDA; }
    *out = ctx;
    return KB_OK;
}

kb_status kb_destroy(kb_ctx* ctx) {
    if (!ctx) return KB_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    cudaFree(ctx->d_xq);
    cudaFree(ctx->d_wq);
    cudaFree(ctx->d_sig);
    cudaFree(ctx->d_dsig);
    cudaFree(ctx->d_gt);
    cudaFree(ctx->d_st);
    if (ctx->ws.ptr) {
        cudaFreeAsync(ctx->ws.ptr, nullptr);
        cudaDeviceSynchronize();
    }
    for (int s = 0; s < KB_MAX_SLOTS; ++s) kb_vertex_cache_free(ctx, s);
    prof_clear(ctx);
    delete ctx;
    return KB_OK;
}

kb_status kb_set_grids(kb_ctx* ctx, const kb_grid_desc* g) {
    if (!ctx || !g) return KB_ERR_ARG;
    if (g->n1 < 1 || g->n2w < 1 || g->n2v < 1 || g->n3w < 1 || g->n3v < 1 || g->nq < 5 || (g->nq - 1) % 4 ||
        !(g->A > 0)) {
        ctx->err = "kb_set_grids: sizes must be >= 1, nq = 4P+1 >= 5, A > 0";
        return KB_ERR_ARG;
    }
    cudaSetDevice(ctx->device);
    std::vector<double> x, w;
    kb::gl5_nodes(g->nq, x, w);
    cudaFree(ctx->d_xq);
    cudaFree(ctx->d_wq);
    ++ctx->mem_gen;
    ctx->d_xq = ctx->d_wq = nullptr;
    KB_CUDA_TRY(ctx, cudaMalloc(&ctx->d_xq, sizeof(double) * g->nq));
    KB_CUDA_TRY(ctx, cudaMalloc(&ctx->d_wq, sizeof(double) * g->nq));
    KB_CUDA_TRY(ctx, cudaMemcpy(ctx->d_xq, x.data(), sizeof(double) * g->nq, cudaMemcpyHostToDevice));
    KB_CUDA_TRY(ctx, cudaMemcpy(ctx->d_wq, w.data(), sizeof(double) * g->nq, cudaMemcpyHostToDevice));
    ctx->g = {g->n1, g->n2w, g->n2v, g->n3w, g->n3v, g->nq, g->A};
    ctx->grids_set = true;
    for (int s = 0; s < KB_MAX_SLOTS; ++s) ++ctx->slot_gen[s];
    return KB_OK;
}

kb_status kb_set_model(kb_ctx* ctx, double Delta, double T, double eps) {
    if (!ctx || !(Delta > 0) || !(T >= 0) || !std::isfinite(eps) || (ctx->m.reg == KB_REG_T && !(T > 0))) {
        if (ctx) ctx->err = "kb_set_model: need Delta > 0, T >= 0 (T > 0 in the temperature flow), finite eps";
        return KB_ERR_ARG;
    }
    ctx->m.Delta = Delta;
    ctx->m.T = T;
    ctx->m.eps = eps;
    ctx->model_set = true;
    for (int s = 0; s < KB_MAX_SLOTS; ++s) ++ctx->slot_gen[s];     // cached K3 right tiles hold Π
    return KB_OK;
}

kb_status kb_set_self_energy_derivative(kb_ctx* ctx, int n, double A, const double* dsigR, const double* dsigK) {
    if (!ctx) return KB_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (ctx->d_dsig) ++ctx->mem_gen;
    cudaFree(ctx->d_dsig);
    ctx->d_dsig = nullptr;
    ctx->m.n_dsig = 0;
    ctx->m.dsigR = ctx->m.dsigK = nullptr;
    for (int s = 0; s < KB_MAX_SLOTS; ++s) ++ctx->slot_gen[s];
    if (!dsigR) return KB_OK;
    if (n < 1 || !(A > 0)) { ctx->err = "kb_set_self_energy_derivative: n >= 1, A > 0"; return KB_ERR_ARG; }
    std::vector<double2> h(2 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        h[i] = make_double2(dsigR[2 * i], dsigR[2 * i + 1]);
        h[n + i] = dsigK ? make_double2(dsigK[2 * i], dsigK[2 * i + 1]) : make_double2(0, 0);
    }
    KB_CUDA_TRY(ctx, cudaMalloc(&ctx->d_dsig, sizeof(double2) * h.size()));
    KB_CUDA_TRY(ctx, cudaMemcpy(ctx->d_dsig, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice));
    ctx->m.n_dsig = n;
    ctx->m.A_dsig = A;
    ctx->m.dsigR = ctx->d_dsig;
    ctx->m.dsigK = ctx->d_dsig + n;
    return KB_OK;
}

kb_status kb_set_regulator(kb_ctx* ctx, int kind, double lambda) {
    if (!ctx) return KB_ERR_ARG;
    if ((kind != KB_REG_DELTA && kind != KB_REG_U && kind != KB_REG_T && kind != KB_REG_NONE) ||
        (kind == KB_REG_U && !(lambda > 0 && std::isfinite(lambda)))) {
        ctx->err = "kb_set_regulator: unknown scheme, or lambda <= 0 for the interaction flow";
        return KB_ERR_ARG;
    }
    if (kind == KB_REG_T && ctx->model_set && !(ctx->m.T > 0)) {
        ctx->err = "kb_set_regulator: the temperature flow needs T > 0";
        return KB_ERR_ARG;
    }
    ctx->m.reg = kind;
    ctx->m.lam = (kind == KB_REG_U) ? lambda : 1.0;
    for (int s = 0; s < KB_MAX_SLOTS; ++s) ++ctx->slot_gen[s];     // cached K3 right tiles hold Π
    return KB_OK;
}

kb_status kb_set_self_energy(kb_ctx* ctx, int n_sig, double A_sig, const double* sigR, const double* sigK) {
    if (!ctx) return KB_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (ctx->d_sig) ++ctx->mem_gen;
    cudaFree(ctx->d_sig);
    ctx->d_sig = nullptr;
    ctx->m.n_sig = 0;
    ctx->m.sigR = ctx->m.sigK = nullptr;
    for (int s = 0; s < KB_MAX_SLOTS; ++s) ++ctx->slot_gen[s];
    if (!sigR) return KB_OK;
    if (n_sig < 1 || !(A_sig > 0)) { ctx->err = "kb_set_self_energy: n_sig >= 1, A_sig > 0"; return KB_ERR_ARG; }
    std::vector<double2> h(2 * (size_t)n_sig);
    for (int i = 0; i < n_sig; ++i) {
        h[i] = make_double2(sigR[2 * i], sigR[2 * i + 1]);
        h[n_sig + i] = sigK ? make_double2(sigK[2 * i], sigK[2 * i + 1]) : make_double2(0, 0);
    }
    KB_CUDA_TRY(ctx, cudaMalloc(&ctx->d_sig, sizeof(double2) * h.size()));
    KB_CUDA_TRY(ctx, cudaMemcpy(ctx->d_sig, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice));
    ctx->m.n_sig = n_sig;
    ctx->m.A_sig = A_sig;
    ctx->m.sigR = ctx->d_sig;
    ctx->m.sigK = ctx->d_sig + n_sig;
    return KB_OK;
}

kb_status kb_set_propagator_table(kb_ctx* ctx, int which, int n, double A_tab, const double* tabR,
                                  const double* tabK) {
    if (!ctx) return KB_ERR_ARG;
    if (which != KB_PROP_G && which != KB_PROP_S) {
        ctx->err = "kb_set_propagator_table: which must be KB_PROP_G or KB_PROP_S";
        return KB_ERR_ARG;
    }
    if (tabR && (n < 1 || !(A_tab > 0) || !std::isfinite(A_tab))) {
        ctx->err = "kb_set_propagator_table: n >= 1, A_tab > 0";
        return KB_ERR_ARG;
    }
    if (tabR)
        for (int i = 0; i < 2 * n; ++i)
            if (!std::isfinite(tabR[i]) || (tabK && !std::isfinite(tabK[i]))) {
                ctx->err = "kb_set_propagator_table: table entries must be finite";
                return KB_ERR_ARG;
            }
    cudaSetDevice(ctx->device);
    double2*& buf = (which == KB_PROP_G) ? ctx->d_gt : ctx->d_st;
    if (buf) ++ctx->mem_gen;                   // step graphs that captured the old table
    cudaFree(buf);
    buf = nullptr;
    if (which == KB_PROP_G) { ctx->m.n_gt = 0; ctx->m.gtR = ctx->m.gtK = nullptr; }
    else { ctx->m.n_st = 0; ctx->m.stR = ctx->m.stK = nullptr; }
    for (int s = 0; s < KB_MAX_SLOTS; ++s) ++ctx->slot_gen[s];     // cached K3 right tiles hold Π
    if (!tabR) return KB_OK;
    std::vector<double2> h(2 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        h[i] = make_double2(tabR[2 * i], tabR[2 * i + 1]);
        h[n + i] = tabK ? make_double2(tabK[2 * i], tabK[2 * i + 1]) : make_double2(0, 0);
    }
    KB_CUDA_TRY(ctx, cudaMalloc(&buf, sizeof(double2) * h.size()));
    KB_CUDA_TRY(ctx, cudaMemcpy(buf, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice));
    if (which == KB_PROP_G) { ctx->m.n_gt = n; ctx->m.A_gt = A_tab; ctx->m.gtR = buf; ctx->m.gtK = buf + n; }
    else { ctx->m.n_st = n; ctx->m.A_st = A_tab; ctx->m.stR = buf; ctx->m.stK = buf + n; }
    return KB_OK;
}

// A tabulated G leaves the single-scale line S undefined unless S is tabulated too.
static bool s_line_defined(const kb_ctx* ctx) { return ctx->m.n_gt == 0 || ctx->m.n_st > 0; }

kb_status kb_set_vertex(kb_ctx* ctx, int slot, int has_R, double U) {
    if (!ctx || slot < 0 || slot >= KB_MAX_SLOTS || !std::isfinite(U)) {
        if (ctx) ctx->err = "kb_set_vertex: bad slot or U";
        return KB_ERR_ARG;
    }
    std::memset(&ctx->slots[slot], 0, sizeof(kb::VertexDev));
    ctx->slots[slot].has_R = has_R ? 1 : 0;
    ctx->slots[slot].mask = 7;
    ctx->slots[slot].bare = -0.5 * U;
    ctx->slot_set[slot] = true;
    ++ctx->slot_gen[slot];
    return KB_OK;
}

kb_status kb_set_vertex_channels(kb_ctx* ctx, int slot, unsigned mask) {
    if (!ctx || slot < 0 || slot >= KB_MAX_SLOTS || mask > 7) {
        if (ctx) ctx->err = "kb_set_vertex_channels: bad slot or mask";
        return KB_ERR_ARG;
    }
    if (!ctx->slot_set[slot]) { ctx->err = "kb_set_vertex_channels: call kb_set_vertex first"; return KB_ERR_STATE; }
    ctx->slots[slot].mask = (int)mask;
    ++ctx->slot_gen[slot];
    return KB_OK;
}

kb_status kb_set_vertex_symmetric(kb_ctx* ctx, int slot, int symmetric) {
    if (!ctx || slot < 0 || slot >= KB_MAX_SLOTS) {
        if (ctx) ctx->err = "kb_set_vertex_symmetric: bad slot";
        return KB_ERR_ARG;
    }
    if (!ctx->slot_set[slot]) { ctx->err = "kb_set_vertex_symmetric: call kb_set_vertex first"; return KB_ERR_STATE; }
    ctx->slots[slot].symmetric = symmetric ? 1 : 0;
    return KB_OK;
}

kb_status kb_set_vertex_class(kb_ctx* ctx, int slot, int channel, int cls, void* ptr, int dtype) {
    if (!ctx || slot < 0 || slot >= KB_MAX_SLOTS || channel < 0 || channel > 2 || cls < 0 || cls > 3 ||
        (dtype != KB_DT_C128 && dtype != KB_DT_C64)) {
        if (ctx) ctx->err = "kb_set_vertex_class: bad slot/channel/class/dtype";
        return KB_ERR_ARG;
    }
    if (!ctx->slot_set[slot]) { ctx->err = "kb_set_vertex_class: call kb_set_vertex first"; return KB_ERR_STATE; }
    if (ptr && (reinterpret_cast<uintptr_t>(ptr) % (dtype == KB_DT_C128 ? 16 : 8))) {
        ctx->err = "kb_set_vertex_class: pointer not aligned to the complex type";
        return KB_ERR_ARG;
    }
    ctx->slots[slot].cls[channel][cls] = ptr;
    ctx->slots[slot].dt[channel][cls] = dtype;
    ++ctx->slot_gen[slot];
    return KB_OK;
}

kb_status kb_bubble_t_su2(kb_ctx* ctx, int slot, int so, int pi_kind, unsigned mask, double alpha, void* stream) {
    if (!ctx) return KB_ERR_ARG;
    if (!ctx->grids_set || !ctx->model_set) {
        ctx->err = "kb_bubble_t_su2: set grids and model first";
        return KB_ERR_STATE;
    }
    if (slot < 0 || slot >= KB_MAX_SLOTS || so < 0 || so >= KB_MAX_SLOTS ||
        (pi_kind != KB_PI_GG && pi_kind != KB_PI_GS_SG) || (mask & ~KB_MASK_ALL) || !std::isfinite(alpha)) {
        ctx->err = "kb_bubble_t_su2: argument out of range";
        return KB_ERR_ARG;
    }
    if (!ctx->slot_set[slot] || !ctx->slot_set[so]) { ctx->err = "kb_bubble_t_su2: slot not set"; return KB_ERR_STATE; }
    if (pi_kind == KB_PI_GS_SG && !s_line_defined(ctx)) {
        ctx->err = "kb_bubble_t_su2: G is tabulated, so KB_PI_GS_SG needs an S table";
        return KB_ERR_STATE;
    }
    for (int k = 0; k < 4; ++k)
        if ((mask >> k) & 1) {
            const void* o = ctx->slots[so].cls[KB_CH_T][k];
            if (!o) { ctx->err = "kb_bubble_t_su2: output class not attached"; return KB_ERR_STATE; }
            for (int c = 0; c < 3; ++c)
                for (int q = 0; q < 4; ++q)
                    if (o == ctx->slots[slot].cls[c][q]) {
                        ctx->err = "kb_bubble_t_su2: output aliases an input class";
                        return KB_ERR_ARG;
                    }
        }
    if (mask == 0) return KB_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) { ctx->err = "cudaSetDevice failed"; return KB_ERR_CUDA; }
    return kb_bubble_mixed_t_su2(ctx, slot, so, pi_kind, mask, alpha, reinterpret_cast<cudaStream_t>(stream));
}

kb_status kb_t_su2_finish(kb_ctx* ctx, int so, const void* a_k3, int a_dtype, double alpha, void* stream) {
    if (!ctx) return KB_ERR_ARG;
    if (!ctx->grids_set) { ctx->err = "kb_t_su2_finish: set grids first"; return KB_ERR_STATE; }
    if (so < 0 || so >= KB_MAX_SLOTS || !a_k3 || (a_dtype != KB_DT_C64 && a_dtype != KB_DT_C128) ||
        !std::isfinite(alpha)) {
        ctx->err = "kb_t_su2_finish: argument out of range";
        return KB_ERR_ARG;
    }
    if (!ctx->slot_set[so] || !ctx->slots[so].cls[KB_CH_T][KB_K3]) {
        ctx->err = "kb_t_su2_finish: the output slot's t-channel K3 class is not attached";
        return KB_ERR_STATE;
    }
    if (ctx->slots[so].cls[KB_CH_T][KB_K3] == a_k3) {
        ctx->err = "kb_t_su2_finish: the a-channel K3 array aliases the output";
        return KB_ERR_ARG;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) { ctx->err = "cudaSetDevice failed"; return KB_ERR_CUDA; }
    return kb_t_su2_finish_impl(ctx, so, a_k3, a_dtype, alpha, reinterpret_cast<cudaStream_t>(stream));
}

kb_status kb_bubble(kb_ctx* ctx, int channel, int sl, int sr, int so, int pi_kind, unsigned mask, double alpha,
                    double beta, int precision, void* stream) {
    if (!ctx) return KB_ERR_ARG;
    if (!ctx->grids_set || !ctx->model_set) { ctx->err = "kb_bubble: set grids and model first"; return KB_ERR_STATE; }
    if (channel < 0 || channel > 2 || sl < 0 || sl >= KB_MAX_SLOTS || sr < 0 || sr >= KB_MAX_SLOTS || so < 0 ||
        so >= KB_MAX_SLOTS || (pi_kind != KB_PI_GG && pi_kind != KB_PI_GS_SG) || (mask & ~KB_MASK_ALL) ||
        !std::isfinite(alpha) || !std::isfinite(beta)) {
        ctx->err = "kb_bubble: argument out of range";
        return KB_ERR_ARG;
    }
    if (!ctx->slot_set[sl] || !ctx->slot_set[sr] || !ctx->slot_set[so]) {
        ctx->err = "kb_bubble: slot not set";
        return KB_ERR_STATE;
    }
    if (pi_kind == KB_PI_GS_SG && !s_line_defined(ctx)) {
        ctx->err = "kb_bubble: G is tabulated, so KB_PI_GS_SG needs an S table";
        return KB_ERR_STATE;
    }
    for (int k = 0; k < 4; ++k)
        if ((mask >> k) & 1) {
            const void* o = ctx->slots[so].cls[channel][k];
            if (!o) { ctx->err = "kb_bubble: output class not attached"; return KB_ERR_STATE; }
            for (int c = 0; c < 3; ++c)
                for (int q = 0; q < 4; ++q)
                    if (o == ctx->slots[sl].cls[c][q] || o == ctx->slots[sr].cls[c][q]) {
                        ctx->err = "kb_bubble: output aliases an input class";
                        return KB_ERR_ARG;
                    }
        }
    if (mask == 0) return KB_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) { ctx->err = "cudaSetDevice failed"; return KB_ERR_CUDA; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (precision == KB_PREC_FP64) return kb_bubble_fp64(ctx, channel, sl, sr, so, pi_kind, mask, alpha, beta, st);
    if (precision == KB_PREC_MIXED) return kb_bubble_mixed(ctx, channel, sl, sr, so, pi_kind, mask, alpha, beta, st);
    ctx->err = "kb_bubble: unknown precision";
    return KB_ERR_ARG;
}

kb_status kb_bubble_vjp(kb_ctx* ctx, int channel, int sl, int sr, int sgo, int pi_kind, unsigned mask, double alpha,
                        int sgl, int sgr, void* grad_GR_K1, void* grad_GR_K2, void* grad_GR_K3, int precision,
                        void* stream) {
    if (!ctx) return KB_ERR_ARG;
    if (!ctx->grids_set || !ctx->model_set) { ctx->err = "kb_bubble_vjp: set grids and model first"; return KB_ERR_STATE; }
    auto slot_ok = [](int s) { return s >= 0 && s < KB_MAX_SLOTS; };
    if (channel < 0 || channel > 2 || !slot_ok(sl) || !slot_ok(sr) || !slot_ok(sgo) || (sgl != -1 && !slot_ok(sgl)) ||
        (sgr != -1 && !slot_ok(sgr)) || (pi_kind != KB_PI_GG && pi_kind != KB_PI_GS_SG) || (mask & ~KB_MASK_ALL) ||
        !std::isfinite(alpha)) {
        ctx->err = "kb_bubble_vjp: argument out of range";
        return KB_ERR_ARG;
    }
    if (!ctx->slot_set[sl] || !ctx->slot_set[sr] || !ctx->slot_set[sgo] || (sgl >= 0 && !ctx->slot_set[sgl]) ||
        (sgr >= 0 && !ctx->slot_set[sgr])) {
        ctx->err = "kb_bubble_vjp: slot not set";
        return KB_ERR_STATE;
    }
    for (int k = 0; k < 4; ++k)
        if (((mask >> k) & 1) && !ctx->slots[sgo].cls[channel][k]) {
            ctx->err = "kb_bubble_vjp: output-gradient class not attached";
            return KB_ERR_STATE;
        }
    for (int gs : {sgl, sgr}) {
        if (gs < 0) continue;
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 4; ++k) {
                const void* p = ctx->slots[gs].cls[c][k];
                if (!p) continue;
                if (ctx->slots[gs].dt[c][k] != KB_DT_C128) {
                    ctx->err = "kb_bubble_vjp: gradient classes must be complex128";
                    return KB_ERR_ARG;
                }
                for (int q = 0; q < 4; ++q)
                    for (int cc = 0; cc < 3; ++cc)
                        if (p == ctx->slots[sl].cls[cc][q] || p == ctx->slots[sr].cls[cc][q] ||
                            p == ctx->slots[sgo].cls[cc][q]) {
                            ctx->err = "kb_bubble_vjp: a gradient class aliases an input";
                            return KB_ERR_ARG;
                        }
            }
    }
    void* tabs[3] = {grad_GR_K1, grad_GR_K2, grad_GR_K3};
    bool any_gr = grad_GR_K1 || grad_GR_K2 || grad_GR_K3;
    if (any_gr && (pi_kind != KB_PI_GG || ctx->m.n_sig > 0 || ctx->m.n_dsig > 0 || ctx->m.n_gt > 0 ||
                   ctx->m.n_st > 0)) {
        ctx->err = "kb_bubble_vjp: the G^R gradient needs pi_kind GG and no self-energy or line table (FDR form "
                   "of G^K)";
        return KB_ERR_UNSUPPORTED;
    }
    if (pi_kind == KB_PI_GS_SG && !s_line_defined(ctx)) {
        ctx->err = "kb_bubble_vjp: G is tabulated, so KB_PI_GS_SG needs an S table";
        return KB_ERR_STATE;
    }
    if (precision != KB_PREC_FP64 && precision != KB_PREC_MIXED) {
        ctx->err = "kb_bubble_vjp: precision must be KB_PREC_FP64 or KB_PREC_MIXED";
        return KB_ERR_ARG;
    }
    if (mask == 0 || (sgl < 0 && sgr < 0 && !any_gr)) return KB_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) { ctx->err = "cudaSetDevice failed"; return KB_ERR_CUDA; }
    if (precision == KB_PREC_MIXED)
        return kb_bubble_vjp_mixed(ctx, channel, sl, sr, sgo, pi_kind, mask, alpha, sgl, sgr, any_gr ? tabs : nullptr,
                                   reinterpret_cast<cudaStream_t>(stream));
    return kb_bubble_vjp_fp64(ctx, channel, sl, sr, sgo, pi_kind, mask, alpha, sgl, sgr, any_gr ? tabs : nullptr,
                              reinterpret_cast<cudaStream_t>(stream));
}

kb_status kb_set_autotune(kb_ctx* ctx, int on) {
    if (!ctx) return KB_ERR_ARG;
    ctx->autotune = on != 0;
    return KB_OK;
}

kb_status kb_set_workspace_limit(kb_ctx* ctx, unsigned long long bytes) {
    if (!ctx || bytes < (1ull << 20)) return KB_ERR_ARG;
    ctx->ws_limit = (size_t)bytes;
    return KB_OK;
}

kb_status kb_inject_alloc_failures(kb_ctx* ctx, int n) {
    if (!ctx || n < 0) return KB_ERR_ARG;
    ctx->fail_allocs = n;
    return KB_OK;
}

kb_status kb_set_wait_budget(kb_ctx* ctx, long long cycles) {
    if (!ctx || cycles < 0) return KB_ERR_ARG;
    ctx->wait_budget = cycles;
    return KB_OK;
}

kb_status kb_check_device(kb_ctx* ctx) {
    if (!ctx) return KB_ERR_ARG;
    cudaSetDevice(ctx->device);
    KB_CUDA_TRY(ctx, cudaDeviceSynchronize());
    int v = kb_tc_take_status();
    if (v < 0) { ctx->err = "kb_check_device: status read failed"; return KB_ERR_CUDA; }
    if (v) { ctx->err = "a bounded device-side wait gave up (tensor-core contraction)"; return KB_ERR_TIMEOUT; }
    unsigned long long first = 0;
    const unsigned oob = kb_oob_take_all(&first);
    if (oob) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "bounds-checked build: %u out-of-range record accesses skipped (first: site %llu, index %lld)",
                      oob, first >> 48, (long long)(first & 0xffffffffffffull));
        ctx->err = msg;
        return KB_ERR_STATE;
    }
    return KB_OK;
}

int kb_build_checked(void) {
#ifdef KB_CHECKED
    return 1;
#else
    return 0;
#endif
}

kb_status kb_workspace_bytes(kb_ctx* ctx, unsigned long long* bytes) {
    if (!ctx || !bytes) return KB_ERR_ARG;
    *bytes = ctx->ws.bytes;
    return KB_OK;
}

kb_status kb_launch_count(kb_ctx* ctx, unsigned long long* count) {
    if (!ctx || !count) return KB_ERR_ARG;
    *count = ctx->launches;
    return KB_OK;
}

kb_status kb_profile_enable(kb_ctx* ctx, int on) {
    if (!ctx) return KB_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    prof_clear(ctx);
    ctx->prof_on = on != 0;
    return KB_OK;
}

kb_status kb_profile_read(kb_ctx* ctx, int index, const char** name, double* ms, unsigned long long* launches,
                          int* count) {
    if (!ctx) return KB_ERR_ARG;
    cudaSetDevice(ctx->device);
    KB_CUDA_TRY(ctx, cudaDeviceSynchronize());
    std::vector<const char*> names;
    std::vector<double> tot;
    std::vector<unsigned long long> cnt;
    for (auto& r : ctx->prof) {
        float t = 0;
        cudaEventElapsedTime(&t, r.a, r.b);
        size_t i = 0;
        while (i < names.size() && std::strcmp(names[i], r.name)) ++i;
        if (i == names.size()) { names.push_back(r.name); tot.push_back(0); cnt.push_back(0); }
        tot[i] += t;
        cnt[i] += 1;
    }
    if (count) *count = (int)names.size();
    if (!name) return KB_OK;
    if (index < 0 || index >= (int)names.size()) { ctx->err = "kb_profile_read: index out of range"; return KB_ERR_ARG; }
    *name = names[index];
    if (ms) *ms = tot[index];
    if (launches) *launches = cnt[index];
    return KB_OK;
}

const char* kb_last_error(kb_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

}  // extern "C"
