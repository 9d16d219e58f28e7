// Internal types shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/kb.h"

namespace kb {

// Class grids and quadrature size; every axis uses v = A tan(pi x / 2) with
// x_i = -1 + 2 (i + 1) / (N + 1) (Sec. II.G.4).
struct Grids {
    int n1, n2w, n2v, n3w, n3v, nq;
    double A;
};

// One vertex slot as the kernels see it: bare part and per channel/class pointers.
struct VertexDev {
    const void* cls[3][4];   // [channel][K1, K2, K2', K3], nullptr = absent
    int dt[3][4];            // KB_DT_C128 / KB_DT_C64
    int has_R;
    int mask;                // channels included (bit c); excluded channels serve only as
                             // crossing partners of the up-up component
    double bare;             // bare vertex on the components with an odd number of
                             // quantum indices: -U/2
    int symmetric;           // declared conjugation + crossing symmetric
};

// Propagator model (Sec. III.A.1, III.C.2).
struct Model {
    double Delta, T, eps;
    int n_sig;
    double A_sig;
    const double2* sigR;     // device, n_sig entries or nullptr
    const double2* sigK;
    int reg = KB_REG_DELTA;  // flow scheme of the single-scale propagator
    double lam = 1.0;        // interaction-flow parameter (G^R = lam / (v - eps + i Delta - lam Sigma^R))
    int n_dsig = 0;          // > 0: Katanin substitution S -> S + G dSigma G with these tables
    double A_dsig = 5.0;
    const double2* dsigR = nullptr;
    const double2* dsigK = nullptr;
    int n_gt = 0;            // > 0: G^R, G^K read from these tables (kb_set_propagator_table)
    double A_gt = 5.0;
    const double2* gtR = nullptr;
    const double2* gtK = nullptr;
    int n_st = 0;            // > 0: S^R, S^K read from these tables
    double A_st = 5.0;
    const double2* stR = nullptr;
    const double2* stK = nullptr;
};

// Keldysh index maps of channel r (matrix form of the 16-component contraction):
//   left tile  L[A][B] = Gamma1^{cL[A][B]},  right tile R[D][C] = Gamma2^{cR[D][C]},
//   output     B[A][C] -> component cO[A][C];
//   Pi[B][D] = P^{b3|b3'}(arg3) P^{b4|b4'}(arg4) with (b3, b3', b4, b4') = piq[B][D].
struct ChannelMaps {
    int cL[4][4], cR[4][4], cO[4][4];
    int piq[4][4][4];
};
ChannelMaps channel_maps(int r);

// Workspace / bookkeeping owned by a context.
struct Workspace {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace kb

struct kb_prof_rec {
    const char* name;
    cudaEvent_t a, b;
};

struct kb_ctx {
    int device = 0;
    bool grids_set = false, model_set = false;
    kb::Grids g{};
    kb::Model m{};
    double* d_xq = nullptr;   // quadrature nodes x_j (device, nq)
    double* d_wq = nullptr;   // weights w_j (device, nq)
    double2* d_sig = nullptr; // Sigma tables (2 * n_sig)
    double2* d_dsig = nullptr; // dSigma/dLambda tables (2 * n_dsig), Katanin substitution
    double2* d_gt = nullptr;   // tabulated G (2 * n_gt), kb_set_propagator_table
    double2* d_st = nullptr;   // tabulated S (2 * n_st)
    kb::VertexDev slots[KB_MAX_SLOTS];
    bool slot_set[KB_MAX_SLOTS];
    kb::Workspace ws;
    unsigned long long launches = 0;
    std::string err;
    size_t ws_limit = 0;
    bool autotune = false;    // time the tensor-core contraction's split-K candidates per shape
    // bumped whenever device memory that a captured step graph may reference (the workspace,
    // a record cache) is freed or replaced; a graph refuses to launch after a change
    unsigned long long mem_gen = 0;
    int fail_allocs = 0;      // test hook: the next n workspace allocations report out of memory
    long long wait_budget = 0; // clock cycles a bounded device wait may take (0: the default)
    bool prof_on = false;
    std::vector<kb_prof_rec> prof;
    // bumped by every change of a slot (and of the grids); a record cache is valid only for
    // the generation it was built from
    unsigned long long slot_gen[KB_MAX_SLOTS] = {};
    // record caches (kb_vertex_cache), for one channel: side 0 = the slot's records as left
    // vertex of the K2 contraction, 1 = as right vertex of the K2' contraction, 2 = its K3
    // left tile, 3 = its K3 right tile (with Π = G G folded in)
    struct RecCache {
        void* ptr[4] = {nullptr, nullptr, nullptr, nullptr};
        size_t bytes[4] = {0, 0, 0, 0};
        int channel = -1;
        unsigned sides = 0;
        unsigned long long gen = ~0ull;
    } rc[KB_MAX_SLOTS];
};

// Bracket a launch with timing events when profiling is on.
struct KbProfScope {
    kb_ctx* c;
    cudaStream_t s;
    kb_prof_rec rec{};
    KbProfScope(kb_ctx* ctx, cudaStream_t st, const char* name) : c(ctx), s(st) {
        ++c->launches;
        if (!c->prof_on) return;
        rec.name = name;
        cudaEventCreate(&rec.a);
        cudaEventCreate(&rec.b);
        cudaEventRecord(rec.a, s);
    }
    ~KbProfScope() {
        if (!c->prof_on) return;
        cudaEventRecord(rec.b, s);
        c->prof.push_back(rec);
    }
};
#define KB_LAUNCH(ctx, st, name) KbProfScope kb_prof_scope_##__LINE__(ctx, st, name)

// error helper
#define KB_CUDA_TRY(ctx, call)                                                              \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
            return e_ == cudaErrorMemoryAllocation ? KB_ERR_OOM : KB_ERR_CUDA;              \
        }                                                                                   \
    } while (0)

// launchers implemented in kb_fp64.cu / kb_mixed.cu
kb_status kb_bubble_fp64(kb_ctx* ctx, int r, int sl, int sr, int so, int pi_kind, unsigned mask, double alpha,
                         double beta, cudaStream_t st);
kb_status kb_bubble_mixed(kb_ctx* ctx, int r, int sl, int sr, int so, int pi_kind, unsigned mask, double alpha,
                          double beta, cudaStream_t st);
kb_status kb_bubble_vjp_fp64(kb_ctx* ctx, int r, int sl, int sr, int sgo, int pi_kind, unsigned mask, double alpha,
                             int sgl, int sgr, void* const gGR[3], cudaStream_t st);
kb_status kb_bubble_vjp_mixed(kb_ctx* ctx, int r, int sl, int sr, int sgo, int pi_kind, unsigned mask, double alpha,
                             int sgl, int sgr, void* const gGR[3], cudaStream_t st);
// Grow the context's workspace to at least `bytes`, stream-ordered on st (the old buffer is
// released after the work already queued on st); sync = true first waits for the whole
// device (used outside the bubble calls, where no stream orders the context's earlier work).
// Refuses (KB_ERR_STATE) to grow while st is being captured.
kb_status kb_ensure_workspace(kb_ctx* ctx, size_t bytes, cudaStream_t st, bool sync = false);
// record caches (kb_mixed.cu): allocation (no launch, may cudaMalloc) and the build launch
kb_status kb_vertex_cache_prepare(kb_ctx* ctx, int slot, int channel, unsigned sides);
kb_status kb_vertex_cache_launch(kb_ctx* ctx, int slot, int channel, unsigned sides, cudaStream_t st);
void kb_vertex_cache_free(kb_ctx* ctx, int slot);
// classes of a bubble that vanish identically, and out <- beta * out for them (kb_ops.cu)
unsigned kb_zero_classes(const kb_ctx* ctx, int r, int sl, int sr, unsigned mask);
kb_status kb_scale_classes(kb_ctx* ctx, int r, int so, unsigned classes, double beta, cudaStream_t st);
// split-K autotuning of the tensor-core contraction (kb_tc.cu) and the shapes of a mixed
// bubble's K3 contraction tuned ahead of a graph capture (kb_mixed.cu)
bool kb_tc_tune(kb_ctx* ctx, const float* At, const float* Bt, double2* Cm, int M, int N, int K, int batch,
                void* scratch, size_t scratch_bytes, bool tri, cudaStream_t st);
kb_status kb_mixed_tune(kb_ctx* ctx, int r, int sl, int sr, unsigned mask, double beta, cudaStream_t st,
                        bool tsu2 = false);
// the t bubble in its SU(2) form and its completion (kb_mixed.cu)
kb_status kb_bubble_mixed_t_su2(kb_ctx* ctx, int sl, int so, int pi_kind, unsigned mask, double alpha,
                                cudaStream_t st);
kb_status kb_t_su2_finish_impl(kb_ctx* ctx, int so, const void* a_k3, int a_dt, double alpha, cudaStream_t st);
// symmetry image of a channel's classes into another slot (kb_ops.cu)
kb_status kb_vertex_image_impl(kb_ctx* ctx, int channel, int src, int dst, unsigned mask, cudaStream_t st);
// slot arithmetic (kb_ops.cu)
kb_status kb_vertex_add_impl(kb_ctx* ctx, int channel, int src, int dst, unsigned mask, double alpha,
                             cudaStream_t st);
// workspace a bubble needs (so that a graph capture never grows it), and the one-time
// device setup of each unit (constant tables, kernel attributes) done before a capture
size_t kb_fp64_workspace_need(const kb_ctx* ctx, int r, unsigned mask);
size_t kb_mixed_workspace_need(const kb_ctx* ctx, int r, unsigned mask);
kb_status kb_fp64_prepare(kb_ctx* ctx);
bool kb_tc_prepare(int device);
bool kb_mixed_prepare(int device);
// Bounds-checked builds (KB_CHECKED): each translation unit registers a function that reads
// and clears its count of skipped out-of-range record accesses (and the first offender,
// site << 48 | index); kb_check_device polls them.
bool kb_oob_register(unsigned (*take)(unsigned long long* first));
unsigned kb_oob_take_all(unsigned long long* first);
