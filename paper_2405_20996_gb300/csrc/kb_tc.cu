// K3 contraction on the 5th-generation tensor cores (tcgen05, kind::tf32) with a 3xTF32
// split: each FP32 operand x = hi + lo (hi = TF32 rounding of x, lo = x - hi), and
//   Re C = Ar Br - Ai Bi,  Im C = Ar Bi + Ai Br,
// every real product X Y taken as Xhi Yhi + Xhi Ylo + Xlo Yhi (the lo*lo term, ~2^-22
// relative, is dropped).  Two tile shapes (see TcShape):
//   one CTA for the real or the imaginary part of a 128 x 128 complex tile: 6 MMAs of
//   N = 128 per k-step, the minus sign of Ai Bi through the negate-A bit of the instruction
//   descriptor;
//   one CTA for both parts of a 128 x 64 complex tile: the B planes of the real and the
//   imaginary part sit side by side in shared memory as one 128-row operand [Br | Bi], so
//   P = Ar [Br | Bi] and Q = Ai [Br | Bi] are 6 MMAs of N = 128 per k-step into two
//   accumulators, and the epilogue forms Re = P_r - Q_i, Im = P_i + Q_r column by column.
// Every CTA loads all of its operand planes itself (plain TMA into its own shared memory;
// no thread-block clusters).  Accumulation in FP32 in tensor memory restarted every 32
// elements of K; finished segments are added into compensated FP32 sums in registers, the
// K dimension is split over CTAs and the split partials are added in FP64.
//
// Operands (written by k_mx_tile3): A = [batch][plane][M][K], B = [batch][plane][N][K],
// planes (re hi, re lo, im hi, im lo), K-contiguous FP32.  One CTA = one (batch, 128-row
// M tile, N tile, part or both parts, K range).  Warp roles: warp 0 issues the TMA loads,
// warp 1 allocates tensor memory and issues the MMAs, warps 2-17 drain the accumulators.
// All waits are bounded; a wait that gives up sets a device flag (read by kb_check_device),
// the CTA drains its copies in flight and frees its tensor memory before returning.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include <string>

#include "kb_internal.h"

namespace kb {
namespace tc {

constexpr int SEGK = 32;          // K elements per accumulation segment
constexpr int MT = 128;           // rows per M tile
constexpr long long WAIT_BUDGET = 4000000000LL;   // clock cycles (~2 s) per wait

__device__ int g_tc_status;       // nonzero: a bounded wait gave up (bit 0 producer, 1 MMA, 2 epilogue)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget = WAIT_BUDGET) {
    if (mbar_try(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major operand with rows of ROWB bytes
// (64: 64-byte swizzle, 128: 128-byte swizzle), 8-row groups 8 * ROWB bytes apart.
template <int ROWB>
__device__ __forceinline__ uint64_t sdesc_kmajor(uint32_t saddr) {
    static_assert(ROWB == 64 || ROWB == 128, "row bytes");
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);     // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused here)
    d |= (uint64_t)((8 * ROWB) >> 4) << 32;         // stride byte offset
    d |= (uint64_t)1 << 46;                         // descriptor version
    d |= (uint64_t)(ROWB == 128 ? 2 : 4) << 61;     // 128- or 64-byte swizzle
    return d;
}

// Instruction descriptor, kind::tf32: D F32, A/B TF32, both K-major, optional negate A.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N, bool negA) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((negA ? 1u : 0u) << 13) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Four 4-column loads (this warp's 32 lanes) and one wait, in one statement.
__device__ __forceinline__ void tmem_ld4x4(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3, float a[4], float b[4],
                                           float c[4], float d[4]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%16];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%17];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%18];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12, %13, %14, %15}, [%19];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3)
        : "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        a[i] = __uint_as_float(r[i]);
        b[i] = __uint_as_float(r[4 + i]);
        c[i] = __uint_as_float(r[8 + i]);
        d[i] = __uint_as_float(r[12 + i]);
    }
}

struct TcJob {
    int M, N, K, batch, mtiles, ntiles, ksplit, chunks_per_split, nchunks;
    int tiles;   // output tiles per batch entry that are computed
    int tri;     // 1: M = N and the tiles whose rows all lie below their columns' diagonal are skipped
};

// Lowest N tile of M tile mt that is computed.  Rows are (v, A) = 4 v + A and columns
// (v', C) = 4 v' + C; with tri set, a tile whose smallest row frequency v exceeds its
// largest column frequency v' (MT mt >= cols (nt + 1)) holds only points with v > v', which
// the caller fills as the conjugation images of computed points (w, v', v).
__host__ __device__ inline int tc_nt_lo(int mt, int cols, int ntiles, bool tri) {
    if (!tri) return 0;
    const int lo = (MT * mt) / cols;
    return lo < ntiles ? lo : ntiles - 1;
}
__host__ __device__ inline int tc_tiles(int mtiles, int ntiles, int cols, bool tri) {
    int n = 0;
    for (int mt = 0; mt < mtiles; ++mt) n += ntiles - tc_nt_lo(mt, cols, ntiles, tri);
    return n;
}

// Segmented accumulation: tensor memory holds two buffers of the CTA's FP32 accumulators
// (128 x 128, or for both parts the two 128 x 128 products P and Q); the MMA warp restarts a
// buffer every SEGK = 32 elements of K and the epilogue warps add each finished segment
// into compensated (Kahan) FP32 running sums held in registers, so no plain FP32 accumulator
// ever sums more than 6 * SEGK products (one part per CTA; both parts: 3 * SEGK into each of
// P and Q).
// Two tile shapes (template BOTH):
//   BOTH = false  one CTA per real or imaginary part of a 128 x 128 complex tile, N = 128
//                 MMAs (6 per k-step); the Re and Im CTAs of a tile each load all 8 planes;
//                 stages of 16 K elements (64-byte plane rows, 64-byte swizzle);
//   BOTH = true   one CTA for both parts of a 128 x 64 complex tile: the B planes stored as
//                 [re hi, im hi, re lo, im lo], so that [Br | Bi] (hi or lo) is one 128-row
//                 operand, and 6 MMAs of N = 128 per k-step give P = Ar [Br | Bi] and
//                 Q = Ai [Br | Bi] (512 tensor-memory columns: two buffers of P and Q);
//                 every operand byte is loaded once per tile; stages of 32 K elements
//                 (128-byte plane rows, 128-byte swizzle), so that each TMA row read is a
//                 whole 128-byte line.
// Both hold 128 x 128 running sums per CTA (the register budget of the Kahan epilogue).
constexpr int EPI_WARPS = 16;                 // 4 per TMEM lane quarter, 32 columns each
constexpr int NTHREADS_S = 64 + 32 * EPI_WARPS;

template <bool BOTH>
struct TcShape {
    static constexpr int NT = BOTH ? 64 : 128;            // B rows (complex columns) per CTA
    static constexpr int KC = BOTH ? 32 : 16;             // K elements per stage (plane row)
    static constexpr int ROWB = KC * 4;                   // plane row bytes = swizzle width
    static constexpr int SEG = SEGK / KC;                 // stages per accumulation segment
    static constexpr int STAGES = BOTH ? 2 : 3;
    static constexpr uint32_t A_PLANE = MT * KC * 4;      // 16 or 8 KB
    static constexpr uint32_t B_PLANE = NT * KC * 4;      // 8 KB
    static constexpr uint32_t STAGE = 4 * A_PLANE + 4 * B_PLANE;
    static constexpr int PARTS = BOTH ? 1 : 2;            // CTAs per tile
    static constexpr size_t smem() { return (size_t)STAGES * STAGE + 128 + 1024; }
};

// Compensated (Kahan) summation of two columns at once with packed FP32 operations:
// s is the running sum, n the negated compensation (the rounding error still to be added).
// Each step: y = x + n, t = s + y, n = y - (t - s), s = t; the subtractions are FMAs with
// -1, so every operation is one correctly rounded FP32 result.  The sum is s + n.
__device__ __forceinline__ void kahan2(float2& s, float2& n, float2 x) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 y = __fadd2_rn(x, n);
    const float2 t = __fadd2_rn(s, y);
    const float2 d = __ffma2_rn(m1, s, t);
    n = __ffma2_rn(m1, d, y);
    s = t;
}

// partial sums P[ks][b][M][N] double2.  Register cap: the 18 warps of a CTA sit 5, 5, 4, 4
// on the SM's four sub-partitions of 16384 registers each, so at most 102 per thread.
template <bool BOTH>
__global__ void __maxnreg__(96)
    k_tc_k3(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcJob J,
            double2* __restrict__ P) {
    using S = TcShape<BOTH>;
    constexpr int NT = S::NT, STAGES_S = S::STAGES, KC = S::KC, ROWB = S::ROWB, SEG = S::SEG;
    constexpr uint32_t A_PLANE = S::A_PLANE, B_PLANE = S::B_PLANE, STAGE = S::STAGE;
    constexpr uint32_t BUF_COLS = BOTH ? 256 : 128;  // one accumulator buffer (BOTH: P, Q)
    constexpr uint32_t TMEM_COLS = 2 * BUF_COLS;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES_S * STAGE);
    uint64_t* empty = full + STAGES_S;
    uint64_t* segfull = empty + STAGES_S;       // [2]
    uint64_t* segempty = segfull + 2;           // [2]
    uint64_t* drain = segempty + 2;             // [1] every MMA of this CTA has completed
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
    __shared__ volatile int s_fail;

    // BOTH = false: neighbouring CTAs are the real and the imaginary part of one tile
    const int part = BOTH ? 0 : (blockIdx.x & 1);
    int unit = BOTH ? blockIdx.x : (blockIdx.x >> 1);
    int ks = unit % J.ksplit;
    int rest = unit / J.ksplit;
    int tile = rest % J.tiles;
    int b = rest / J.tiles;
    int mt = 0, nt = 0;
    for (mt = 0; mt < J.mtiles; ++mt) {
        const int lo = tc_nt_lo(mt, NT, J.ntiles, J.tri != 0), cnt = J.ntiles - lo;
        if (tile < cnt) { nt = lo + tile; break; }
        tile -= cnt;
    }
    int c0 = ks * J.chunks_per_split;
    int c1 = min(J.nchunks, c0 + J.chunks_per_split);
    int nck = max(0, c1 - c0);
    int nseg = (nck + SEG - 1) / SEG;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES_S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&segfull[i], 1); mbar_init(&segempty[i], 32 * EPI_WARPS); }
        mbar_init(drain, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    uint32_t tbase = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t issued = 0, phases = 0;     // bit s: stage s issued / parity of its last issue
            for (int i = 0; i < nck; ++i) {
                int s = i % STAGES_S;
                uint32_t ph = (uint32_t)((i / STAGES_S) & 1);
                if (s_fail) break;
                if (i >= STAGES_S && !mbar_wait(&empty[s], ph ^ 1)) { atomicOr(&g_tc_status, 1); s_fail = 1; break; }
                unsigned char* st = smem + s * STAGE;
                mbar_expect_tx(&full[s], STAGE);
                int kx = (c0 + i) * KC;
                for (int p = 0; p < 4; ++p) {
                    // B planes: BOTH stores them as re hi, im hi, re lo, im lo
                    const int bslot = BOTH ? ((p & 1) * 2 + (p >> 1)) : p;
                    tma_load_3d(st + p * A_PLANE, &tmA, &full[s], kx, mt * MT, 4 * b + p);
                    tma_load_3d(st + 4 * A_PLANE + bslot * B_PLANE, &tmB, &full[s], kx, nt * NT, 4 * b + p);
                }
                issued |= 1u << s;
                phases = (phases & ~(1u << s)) | (ph << s);
            }
            for (int s = 0; s < STAGES_S; ++s)
                if (((issued >> s) & 1) && !mbar_wait(&full[s], (phases >> s) & 1)) atomicOr(&g_tc_status, 1);
            // tail: the MMAs have released every stage, so no commit arrival is still on its
            // way to this CTA's barriers when it leaves
            if (!s_fail)
                for (int s = 0; s < STAGES_S; ++s)
                    if (((issued >> s) & 1) && !mbar_wait(&empty[s], (phases >> s) & 1)) atomicOr(&g_tc_status, 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id_pos = idesc_tf32(MT, NT, false), id_neg = idesc_tf32(MT, NT, true);
            const uint32_t id_cat = idesc_tf32(MT, 2 * NT, false);   // BOTH: B = [Br | Bi]
            for (int i = 0; i < nck; ++i) {
                int s = i % STAGES_S;
                uint32_t ph = (uint32_t)((i / STAGES_S) & 1);
                int g = i / SEG, buf = g & 1;
                bool seg_start = (i % SEG) == 0;
                if (s_fail) break;
                if (seg_start && g >= 2 && !mbar_wait(&segempty[buf], (uint32_t)(((g >> 1) - 1) & 1))) {
                    atomicOr(&g_tc_status, 2); s_fail = 1; break;
                }
                if (!mbar_wait(&full[s], ph)) { atomicOr(&g_tc_status, 2); s_fail = 1; break; }
                fence_after();
                const uint32_t dacc = tbase + buf * BUF_COLS;
                uint32_t sa = smem_u32(smem + s * STAGE);
                uint32_t sb = sa + 4 * A_PLANE;
#pragma unroll
                for (int kk = 0; kk < KC / 8; ++kk) {
                    uint32_t off = kk * 32;
                    uint64_t arh = sdesc_kmajor<ROWB>(sa + 0 * A_PLANE + off), arl = sdesc_kmajor<ROWB>(sa + 1 * A_PLANE + off);
                    uint64_t aih = sdesc_kmajor<ROWB>(sa + 2 * A_PLANE + off), ail = sdesc_kmajor<ROWB>(sa + 3 * A_PLANE + off);
                    uint32_t first = (seg_start && kk == 0) ? 0u : 1u;
                    if (BOTH) {
                        // P = Ar [Br | Bi] (columns 0-127), Q = Ai [Br | Bi] (128-255)
                        const uint64_t bch = sdesc_kmajor<ROWB>(sb + off), bcl = sdesc_kmajor<ROWB>(sb + 2 * B_PLANE + off);
                        mma_tf32(dacc, arh, bch, id_cat, first);
                        mma_tf32(dacc, arh, bcl, id_cat, 1);
                        mma_tf32(dacc, arl, bch, id_cat, 1);
                        mma_tf32(dacc + 128, aih, bch, id_cat, first);
                        mma_tf32(dacc + 128, aih, bcl, id_cat, 1);
                        mma_tf32(dacc + 128, ail, bch, id_cat, 1);
                        continue;
                    }
                    uint64_t brh = sdesc_kmajor<ROWB>(sb + 0 * B_PLANE + off), brl = sdesc_kmajor<ROWB>(sb + 1 * B_PLANE + off);
                    uint64_t bih = sdesc_kmajor<ROWB>(sb + 2 * B_PLANE + off), bil = sdesc_kmajor<ROWB>(sb + 3 * B_PLANE + off);
                    if (part == 0) {           // Re = Ar Br - Ai Bi
                        mma_tf32(dacc, arh, brh, id_pos, first);
                        mma_tf32(dacc, arh, brl, id_pos, 1);
                        mma_tf32(dacc, arl, brh, id_pos, 1);
                        mma_tf32(dacc, aih, bih, id_neg, 1);
                        mma_tf32(dacc, aih, bil, id_neg, 1);
                        mma_tf32(dacc, ail, bih, id_neg, 1);
                    }
                    if (part == 1) {           // Im = Ar Bi + Ai Br
                        mma_tf32(dacc, arh, bih, id_pos, first);
                        mma_tf32(dacc, arh, bil, id_pos, 1);
                        mma_tf32(dacc, arl, bih, id_pos, 1);
                        mma_tf32(dacc, aih, brh, id_pos, 1);
                        mma_tf32(dacc, aih, brl, id_pos, 1);
                        mma_tf32(dacc, ail, brh, id_pos, 1);
                    }
                }
                mma_commit(&empty[s]);                   // the stage is free once its MMAs are done
                if ((i % SEG) == SEG - 1 || i == nck - 1) mma_commit(&segfull[buf]);
            }
            // whether the loop finished or gave up: every MMA issued so far completes before
            // the tensor memory is released at the end
            mma_commit(drain);
            if (!mbar_wait(drain, 0)) atomicOr(&g_tc_status, 2);
        }
    } else {
        // epilogue warps 2 .. 2+EPI_WARPS-1: lane quarter q, column group cg: one part, 32
        // real columns 2i, 2i+1 per sm[i]; BOTH: 16 complex columns, the real and imaginary
        // part of column i in sm[i], each formed from the products P and Q
        int e = warp - 2;
        int q = warp & 3, cg = e >> 2;
        float2 sm[16], ng[16];       // running sums and negated compensations
#pragma unroll
        for (int i = 0; i < 16; ++i) { sm[i] = make_float2(0.f, 0.f); ng[i] = make_float2(0.f, 0.f); }
        bool ok = true;
        for (int g = 0; g < nseg; ++g) {
            int buf = g & 1;
            if (s_fail || !mbar_wait(&segfull[buf], (uint32_t)((g >> 1) & 1))) {
                atomicOr(&g_tc_status, 4); ok = false; break;
            }
            fence_after();
            const uint32_t lb = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BUF_COLS);
            if (BOTH) {
                // column c = 16 cg + i: Re = Ar Br - Ai Bi = P[c] - Q[64 + c],
                // Im = Ar Bi + Ai Br = P[64 + c] + Q[c]
                const uint32_t t0 = lb + (uint32_t)(16 * cg);
#pragma unroll
                for (int hh = 0; hh < 4; ++hh) {
                    float pr[4], qi[4], pim[4], qr[4];
                    tmem_ld4x4(t0 + 4 * hh, t0 + 192 + 4 * hh, t0 + 64 + 4 * hh, t0 + 128 + 4 * hh, pr, qi, pim, qr);
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        kahan2(sm[4 * hh + c], ng[4 * hh + c],
                               make_float2(__fsub_rn(pr[c], qi[c]), __fadd_rn(pim[c], qr[c])));
                }
            } else {
                // two 16-column loads, one wait each
                const uint32_t ta = lb + (uint32_t)(cg * 32);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float v[16];
                    tmem_ld16(ta + 16 * h, v);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        kahan2(sm[8 * h + c], ng[8 * h + c], make_float2(v[2 * c], v[2 * c + 1]));
                }
            }
            fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&segempty[buf])) : "memory");
        }
        int row = mt * MT + q * 32 + lane;
        if (ok && row < J.M && BOTH) {
            // the FP64 partial of 16 complex columns, one 16-byte store each
            double2* out = P + (((size_t)ks * J.batch + b) * J.M + row) * J.N;
            const int col0 = nt * NT + 16 * cg;
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (col0 + i < J.N)
                    out[col0 + i] = make_double2((double)sm[i].x + (double)ng[i].x, (double)sm[i].y + (double)ng[i].y);
        } else if (ok && row < J.M) {
            // the FP64 partial: .x real / .y imaginary part of this CTA's columns
            double* out = reinterpret_cast<double*>(P + (((size_t)ks * J.batch + b) * J.M + row) * J.N) + part;
            int col0 = nt * NT + cg * 32;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (col0 + 2 * i < J.N) out[2 * (col0 + 2 * i)] = (double)sm[i].x + (double)ng[i].x;
                if (col0 + 2 * i + 1 < J.N) out[2 * (col0 + 2 * i + 1)] = (double)sm[i].y + (double)ng[i].y;
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
}

// Bounded-wait probe: one thread waits, with the given budget, on a shared-memory barrier
// that nothing arrives on; the wait gives up, the device status records it (bit 3) and the
// kernel returns.  No copy or MMA is in flight, so giving up leaves nothing behind.
__global__ void k_wait_probe(long long budget) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0, budget)) atomicOr(&g_tc_status, 8);
}

// C[b][m][n] = sum over splits of P (FP64); with tri (M = N) only the points whose row
// frequency m / 4 does not exceed the column frequency n / 4 (the others are not read).
__global__ void k_tc_reduce(const double2* __restrict__ P, double2* __restrict__ C, size_t per_split, int ksplit,
                            int N, int tri) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= per_split) return;
    if (tri) {
        const int n = (int)(i % N), m = (int)((i / N) % N);
        if ((m >> 2) > (n >> 2)) return;
    }
    double re = 0, im = 0;
    for (int k = 0; k < ksplit; ++k) {
        double2 v = P[(size_t)k * per_split + i];
        re += v.x;
        im += v.y;
    }
    C[i] = make_double2(re, im);
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

static bool make_map(CUtensorMap* m, const float* base, int K, int rows, int planes, int box_rows, int kc) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)K * 4, (cuuint64_t)K * 4 * rows};
    cuuint32_t box[3] = {(cuuint32_t)kc, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, kc == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// One-time per device: opt both kernel shapes in to their dynamic shared memory (not a
// stream operation, so it is done before any capture) and resolve the tensor-map encoder.
static bool tc_prepare(int device) {
    static bool attr_set[64] = {};
    if (device < 0 || device >= 64) return false;
    if (!attr_set[device]) {
        if (cudaFuncSetAttribute(k_tc_k3<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TcShape<true>::smem()) != cudaSuccess ||
            cudaFuncSetAttribute(k_tc_k3<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TcShape<false>::smem()) != cudaSuccess)
            return false;
        attr_set[device] = true;
    }
    return encoder() != nullptr;
}

// A launch shape of the contraction: the tile shape (1: both parts per CTA, 128 x 64
// complex; 0: one part per CTA, 128 x 128) and the split-K factor.
struct TcPlan {
    int both, split;
};

static int tc_cols(int both) { return both ? TcShape<true>::NT : TcShape<false>::NT; }
static int tc_kc(int both) { return both ? TcShape<true>::KC : TcShape<false>::KC; }
static int tc_parts(int both) { return both ? TcShape<true>::PARTS : TcShape<false>::PARTS; }

// Split-K candidates for one contraction shape and tile shape, best first by the wave
// model: a split s gives base * s CTAs (base = batch x tiles x CTAs per tile) of at least 8
// segments of K each, whose partial sums must fit the scratch; the model rates the fraction
// of the last wave that is busy, with a small charge per split for the reduction.
static std::vector<std::pair<double, int>> split_candidates(int device, int both, int M, int N, int K, int batch,
                                                            size_t scratch_bytes, bool tri) {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int mtiles = (M + MT - 1) / MT, ntiles = (N + tc_cols(both) - 1) / tc_cols(both),
              nseg = (K + SEGK - 1) / SEGK;
    const long base = (long)batch * tc_tiles(mtiles, ntiles, tc_cols(both), tri) * tc_parts(both);
    std::vector<std::pair<double, int>> c;
    for (int s = 1; s <= 64; ++s) {
        if ((nseg + s - 1) / s < 8) break;
        if ((size_t)s * batch * M * N * sizeof(double2) > scratch_bytes) break;
        const long units = base * s, waves = (units + sms - 1) / sms;
        c.push_back({(double)units / (waves * sms) * (1.0 - 0.002 * s), s});
    }
    if (c.empty()) c.push_back({0.0, 1});
    std::stable_sort(c.begin(), c.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
        return a.first > b.first + 1e-9;
    });
    return c;
}

// Default plan without timing: the tile shape from KB_TC_SHAPE (developer override) or both
// parts per CTA, and the wave model's best split for it.
static TcPlan default_plan(int device, int M, int N, int K, int batch, size_t scratch_bytes, bool tri) {
    const char* sh = std::getenv("KB_TC_SHAPE");
    const int both = (sh && std::atoi(sh) == 0) ? 0 : 1;
    return {both, split_candidates(device, both, M, N, K, batch, scratch_bytes, tri)[0].second};
}

// Autotuned plans, per device and shape (M, N, K, batch, triangle); filled by tc_tune.
static std::mutex g_tune_mu;
static std::map<std::array<int, 6>, TcPlan> g_tuned;

static bool tuned_plan(int device, int M, int N, int K, int batch, bool tri, TcPlan& p) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find({device, M, N, K, batch, tri ? 1 : 0});
    if (it == g_tuned.end()) return false;
    p = it->second;
    return true;
}

static bool launch_plan(kb_ctx* ctx, const float* At, const float* Bt, double2* Cm, int M, int N, int K, int batch,
                        void* scratch, TcPlan plan, bool tri, cudaStream_t st);

static bool launch(kb_ctx* ctx, const float* At, const float* Bt, double2* Cm, int M, int N, int K, int batch,
                   void* scratch, size_t scratch_bytes, bool tri, cudaStream_t st) {
    TcPlan plan;
    if (!tuned_plan(ctx->device, M, N, K, batch, tri, plan) ||
        (size_t)plan.split * batch * M * N * sizeof(double2) > scratch_bytes)
        plan = default_plan(ctx->device, M, N, K, batch, scratch_bytes, tri);
    const char* cps_env = std::getenv("KB_TC_CPS");   // developer override: K chunks per split
    if (cps_env && std::atoi(cps_env) > 0) {
        const int nchunks = (K + tc_kc(plan.both) - 1) / tc_kc(plan.both);
        int cps = std::atoi(cps_env);
        int s = (nchunks + cps - 1) / cps;
        if ((size_t)s * batch * M * N * sizeof(double2) <= scratch_bytes) plan.split = s;
    }
    return launch_plan(ctx, At, Bt, Cm, M, N, K, batch, scratch, plan, tri, st);
}

// Time the wave model's three best splits of each tile shape for this contraction shape
// (the kernel and its split-K reduction, two runs each, CUDA events on the stream) and
// remember the fastest plan.  Reads At/Bt and writes only the scratch and Cm, so any
// operands of the right shape do; not while the stream is being captured.
static bool tune(kb_ctx* ctx, const float* At, const float* Bt, double2* Cm, int M, int N, int K, int batch,
                 void* scratch, size_t scratch_bytes, bool tri, cudaStream_t st) {
    TcPlan have;
    if (tuned_plan(ctx->device, M, N, K, batch, tri, have)) return true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    std::vector<TcPlan> cand;
    for (int both = 1; both >= 0; --both) {
        auto c = split_candidates(ctx->device, both, M, N, K, batch, scratch_bytes, tri);
        for (size_t i = 0; i < c.size() && i < 3; ++i) cand.push_back({both, c[i].second});
    }
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return false;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return false; }
    TcPlan best = cand[0];
    float best_ms = 1e30f;
    for (const TcPlan& pl : cand) {
        float ms_min = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(a, st);
            if (!launch_plan(ctx, At, Bt, Cm, M, N, K, batch, scratch, pl, tri, st)) { ms_min = 1e30f; break; }
            cudaEventRecord(b, st);
            if (cudaEventSynchronize(b) != cudaSuccess) { ms_min = 1e30f; break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            ms_min = std::min(ms_min, ms);
        }
        if (ms_min < best_ms) { best_ms = ms_min; best = pl; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (std::getenv("KB_TC_VERBOSE"))
        std::fprintf(stderr, "k_tc_k3 autotune: M %d N %d K %d batch %d%s -> %s ksplit %d (%.3f ms)\n", M, N, K,
                     batch, tri ? " (triangle)" : "", best.both ? "re+im per CTA" : "one part per CTA", best.split,
                     best_ms);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[{ctx->device, M, N, K, batch, tri ? 1 : 0}] = best;
    return true;
}

static bool launch_plan(kb_ctx* ctx, const float* At, const float* Bt, double2* Cm, int M, int N, int K, int batch,
                        void* scratch, TcPlan plan, bool tri, cudaStream_t st) {
    TcJob J;
    J.M = M; J.N = N; J.K = K; J.batch = batch;
    const int cols = tc_cols(plan.both);
    J.mtiles = (M + MT - 1) / MT;
    J.ntiles = (N + cols - 1) / cols;
    J.nchunks = (K + tc_kc(plan.both) - 1) / tc_kc(plan.both);
    J.tri = (tri && M == N) ? 1 : 0;
    J.tiles = tc_tiles(J.mtiles, J.ntiles, cols, J.tri != 0);
    const int base = batch * J.tiles * tc_parts(plan.both);
    J.ksplit = plan.split;
    J.chunks_per_split = (J.nchunks + plan.split - 1) / plan.split;
    if (std::getenv("KB_TC_VERBOSE"))
        std::fprintf(stderr, "k_tc_k3: M %d N %d K %d batch %d tiles %dx%d, %d computed (%s) ksplit %d chunks/split %d\n",
                     M, N, K, batch, J.mtiles, J.ntiles, J.tiles, plan.both ? "re+im" : "part", J.ksplit,
                     J.chunks_per_split);
    CUtensorMap ma, mb;
    if (!make_map(&ma, At, K, M, 4 * batch, MT, tc_kc(plan.both)) ||
        !make_map(&mb, Bt, K, N, 4 * batch, cols, tc_kc(plan.both)))
        return false;
    if (!tc_prepare(ctx->device)) return false;
    double2* P = reinterpret_cast<double2*>(scratch);
    {
        KB_LAUNCH(ctx, st, "k_tc_k3");
        if (plan.both)
            k_tc_k3<true><<<(unsigned)(base * J.ksplit), NTHREADS_S, TcShape<true>::smem(), st>>>(ma, mb, J, P);
        else
            k_tc_k3<false><<<(unsigned)(base * J.ksplit), NTHREADS_S, TcShape<false>::smem(), st>>>(ma, mb, J, P);
    }
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
        ctx->err = std::string("k_tc_k3 launch: ") + cudaGetErrorString(le);
        if (std::getenv("KB_TC_VERBOSE")) std::fprintf(stderr, "%s\n", ctx->err.c_str());
        return false;
    }
    {
        KB_LAUNCH(ctx, st, "k_tc_reduce");
        size_t per = (size_t)batch * M * N;
        k_tc_reduce<<<(unsigned)((per + 255) / 256), 256, 0, st>>>(P, Cm, per, J.ksplit, N, J.tri);
    }
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace tc
}  // namespace kb

bool kb_tc_k3(kb_ctx* ctx, const float* At, const float* Bt, double2* Cm, int M, int N, int K, int batch, void* scratch,
              size_t scratch_bytes, bool tri, cudaStream_t st) {
    using namespace kb::tc;
    if ((K % 4) != 0 || (reinterpret_cast<uintptr_t>(At) & 15) || (reinterpret_cast<uintptr_t>(Bt) & 15))
        return false;
    if (tri && M != N) return false;
    if (ctx->autotune) tune(ctx, At, Bt, Cm, M, N, K, batch, scratch, scratch_bytes, tri, st);
    return launch(ctx, At, Bt, Cm, M, N, K, batch, scratch, scratch_bytes, tri, st);
}

bool kb_tc_tune(kb_ctx* ctx, const float* At, const float* Bt, double2* Cm, int M, int N, int K, int batch,
                void* scratch, size_t scratch_bytes, bool tri, cudaStream_t st) {
    using namespace kb::tc;
    if ((K % 4) != 0 || (reinterpret_cast<uintptr_t>(At) & 15) || (reinterpret_cast<uintptr_t>(Bt) & 15))
        return false;
    if (tri && M != N) return false;
    return tune(ctx, At, Bt, Cm, M, N, K, batch, scratch, scratch_bytes, tri, st);
}

bool kb_tc_prepare(int device) { return kb::tc::tc_prepare(device); }

extern "C" kb_status kb_check_wait(kb_ctx* ctx, void* stream) {
    if (!ctx) return KB_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return KB_ERR_CUDA;
    const long long budget = ctx->wait_budget > 0 ? ctx->wait_budget : kb::tc::WAIT_BUDGET;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    {
        KB_LAUNCH(ctx, st, "k_wait_probe");
        kb::tc::k_wait_probe<<<1, 32, 0, st>>>(budget);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { ctx->err = std::string("k_wait_probe launch: ") + cudaGetErrorString(e); return KB_ERR_CUDA; }
    return KB_OK;
}

int kb_tc_take_status() {
    int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, kb::tc::g_tc_status, sizeof(int)) != cudaSuccess) return -1;
    if (v) cudaMemcpyToSymbol(kb::tc::g_tc_status, &z, sizeof(int));
    return v;
}
