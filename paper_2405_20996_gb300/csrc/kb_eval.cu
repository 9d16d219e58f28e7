// Point evaluation of a stored vertex: the full vertex of a slot — the bare part and the
// asymptotic classes of its channels, each read at the point converted to its own channel
// variables (Sec. II.C.1) and interpolated linearly in x (Sec. II.G.7) — at arbitrary
// frequencies given in the variables of one channel.  The paper's post-processing reads
// such slices of the full vertex, e.g. the t-channel plane (w_t = 0, v_t, v'_t).
#include <cstdio>
#include <string>

#include "kb_fp64.cuh"

namespace kb {
namespace {

__global__ void k_vertex_eval(VertexDev V, Grids G, int r, int uu, int n, const double* __restrict__ f,
                              double2* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double w = f[3 * i], v = f[3 * i + 1], vp = f[3 * i + 2];
    double2 a[16], b[16];
    vertex_part_f64(V, G, r, uu != 0, false, false, w, v, vp, a);     // R + K1_r + K2'_r
    vertex_part_f64(V, G, r, uu != 0, false, true, w, v, vp, b);      // K2_r + K3_r + other channels
#pragma unroll
    for (int o = 0; o < 16; ++o) out[(size_t)16 * i + o] = make_double2(a[o].x + b[o].x, a[o].y + b[o].y);
}

}  // namespace
}  // namespace kb

using namespace kb;

extern "C" kb_status kb_vertex_eval(kb_ctx* ctx, int slot, int channel, int spin_uu, int n, const double* freqs,
                                    void* out, void* stream) {
    if (!ctx) return KB_ERR_ARG;
    if (slot < 0 || slot >= KB_MAX_SLOTS || channel < 0 || channel > 2 || n < 0 || (n > 0 && (!freqs || !out))) {
        ctx->err = "kb_vertex_eval: bad slot, channel, count or pointer";
        return KB_ERR_ARG;
    }
    if (!ctx->grids_set || !ctx->slot_set[slot]) {
        ctx->err = "kb_vertex_eval: set the grids and the vertex first";
        return KB_ERR_STATE;
    }
    if (n == 0) return KB_OK;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return KB_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    {
        KB_LAUNCH(ctx, st, "k_vertex_eval");
        k_vertex_eval<<<(n + 127) / 128, 128, 0, st>>>(ctx->slots[slot], ctx->g, channel, spin_uu, n, freqs,
                                                       static_cast<double2*>(out));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("kb_vertex_eval: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}
