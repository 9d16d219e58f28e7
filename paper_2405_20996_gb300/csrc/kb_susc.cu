// Susceptibilities from the K1 class of a vertex slot (the paper's post-processing, Sec.
// II.E.5: for a converged parquet solution they follow from K1, K1_r = R χ_r R with the bare
// vertex R = -U/2 on the Keldysh components with an odd number of quantum indices).  In a
// channel's 4x4 form the components of one parity block carry one number; read on the
// retarded and Keldysh blocks and normalised to the bare susceptibilities at second order:
//   a (transverse spin, up-down):  χ = -2 K1_a / U²      (components 1: R, 3: K)
//   p (pairing, up-down):          χ = +2 K1_p / U²      (components 8: R, 9: K)
//   t (charge, both spins of the pair): χ = 2 [K1_t(ω) + K1_t^uu(ω)] / U²,
//       K1_t^uu(ω) = K1_t(ω) - K1_a(-ω) with a1 <-> a2 swapped (crossing), components 1, 3.
// The same readout serves the leg contraction, whose bubble chain closed by a unit bare
// vertex has the same K1 normalisation at U = 1.
#include <cmath>
#include <string>

#include "kb_internal.h"

namespace kb {
namespace {

__device__ __forceinline__ double2 ld_c(const void* p, int dt, size_t i) {
    if (dt == KB_DT_C128) return reinterpret_cast<const double2*>(p)[i];
    const float2 v = reinterpret_cast<const float2*>(p)[i];
    return make_double2(v.x, v.y);
}

__host__ __device__ constexpr int swap12c(int c) { return (c & 12) | ((c & 1) << 1) | ((c >> 1) & 1); }

// out[w][0] = χ^R(ω_w), out[w][1] = χ^K(ω_w)
__global__ void k_chi_k1(const void* __restrict__ k1, int dt, const void* __restrict__ k1a, int dta, int channel,
                         int n1, double f, double2* __restrict__ out) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n1) return;
    const int cR = channel == KB_CH_P ? 8 : 1, cK = channel == KB_CH_P ? 9 : 3;
    double2 r = ld_c(k1, dt, (size_t)w * 16 + cR), k = ld_c(k1, dt, (size_t)w * 16 + cK);
    if (channel == KB_CH_T) {
        // K1_t + K1_t^uu = 2 K1_t(ω) - K1_a(-ω) at the swapped components (the K1 grid is
        // symmetric under ω -> -ω: node n1 - 1 - w)
        const double2 ar = ld_c(k1a, dta, (size_t)(n1 - 1 - w) * 16 + swap12c(cR));
        const double2 ak = ld_c(k1a, dta, (size_t)(n1 - 1 - w) * 16 + swap12c(cK));
        r = make_double2(2.0 * r.x - ar.x, 2.0 * r.y - ar.y);
        k = make_double2(2.0 * k.x - ak.x, 2.0 * k.y - ak.y);
    }
    out[2 * w] = make_double2(f * r.x, f * r.y);
    out[2 * w + 1] = make_double2(f * k.x, f * k.y);
}

}  // namespace
}  // namespace kb

extern "C" kb_status kb_susceptibility_k1(kb_ctx* ctx, int channel, int slot, double U, void* out, void* stream) {
    if (!ctx) return KB_ERR_ARG;
    if (channel < 0 || channel > 2 || slot < 0 || slot >= KB_MAX_SLOTS || !out || !(U != 0.0) || !std::isfinite(U)) {
        ctx->err = "kb_susceptibility_k1: argument out of range (U must be finite and nonzero)";
        return KB_ERR_ARG;
    }
    if (!ctx->grids_set || !ctx->slot_set[slot]) {
        ctx->err = "kb_susceptibility_k1: set the grids and the slot first";
        return KB_ERR_STATE;
    }
    const kb::VertexDev& V = ctx->slots[slot];
    const void* k1 = V.cls[channel][KB_K1];
    const void* k1a = V.cls[KB_CH_A][KB_K1];
    if (!k1 || (channel == KB_CH_T && !k1a)) {
        ctx->err = "kb_susceptibility_k1: the K1 class (for t also the a channel's) is not attached";
        return KB_ERR_STATE;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return KB_ERR_CUDA;
    const double f = (channel == KB_CH_A ? -2.0 : 2.0) / (U * U);
    const int n1 = ctx->g.n1;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    {
        KB_LAUNCH(ctx, st, "k_chi_k1");
        kb::k_chi_k1<<<(n1 + 127) / 128, 128, 0, st>>>(k1, V.dt[channel][KB_K1], k1a ? k1a : k1,
                                                      k1a ? V.dt[KB_CH_A][KB_K1] : KB_DT_C128, channel, n1, f,
                                                      static_cast<double2*>(out));
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("k_chi_k1: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}
