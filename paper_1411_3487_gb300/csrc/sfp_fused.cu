// sfp_fused.cu -- mode-space steps (Sec. 4) for tiles of 42 chains of the
// SFP_FP32 path, M = 64, 128 or 256 beads, n_steps per launch.
//
// A tile's chain-axis rows j = 3c + alpha (up to 42 chains, 126 rows; the
// rest padding) are the 128 TMEM lanes; bead / mode indices are TMEM
// columns.  Fewer chains per tile give more CTAs on small batches: the MMA
// time of a tile is fixed by its 128 rows, the noise and force work is not.  Per step and tile:
//   inverse  (Eq. e5)   D_u[j][n]   = sum_p R[j][p] chi[n][p]            (bonds)
//   force    (Eq. e11)  v_n = u_n (1/|u_n| - (1 - 2 nu)),  v_0 = 0
//   noise    (Eq. b5)   z_n ~ N(0,1), Philox keyed by (seed, job, step, n)
//   forward  (Eqs. c4, e11, d6, f2)
//            D_inc[j][p] = sum_n v[j][n] h_p chi[n][p] + sum_n z[j][n] w_p phi[n][p]
//                        = h_p DeltaH_p + w_p Z_p
//   update   (Eqs. d3, btum)  R_p += -(1 - e^{-zeta_p dtau}) R_p + D_inc_p
//                             (+ shear g_p R^y_p on the x rows); p = 0 feeds the
//                             FP64 centre of mass.
// ΔH is never formed on its own: Eq. e11 makes it chi^T v, so the bead-space
// stencil of the staged path is not needed, and h_p, w_p are folded into one
// stacked table so a single accumulator holds the whole increment.
//
// Both contractions run on the tcgen05 tensor cores as three TF32 passes
// (A_hi B_lo + A_lo B_hi + A_hi B_hi, FP32 accumulate in TMEM), which keeps
// FP32 accuracy.  Roles (576 threads):
//   warp 0      TMA producer: R tiles and chi hi/lo (inverse), F hi/lo (forward)
//   warp 1      TMEM allocation; one thread issues every MMA and commit
//   warps 2..17 split R tiles into TF32 hi/lo; read D_u (warps 2..5) into a
//               swizzled staging buffer; write v and z blocks (hi/lo) as the
//               A operand of the forward MMAs; epilogue from D_inc.  Sixteen
//               warps keep enough Philox / Box-Muller chains in flight to
//               hide their latency behind the MMAs.
// Block order (K blocks of 32): inverse block nb and noise block nb alternate
// (inv 0, z 0, inv 1, z 1, ...), then the force blocks v 0 .. v KB-1.  The
// noise half of the forward contraction does not depend on the state, so its
// Philox / Box-Muller work overlaps the inverse MMAs; only the force blocks
// wait for the bond vectors.
// Chains never interact, so a CTA runs all n_steps of its tile without any
// grid-wide synchronisation: TMEM stays allocated, the tables stream again
// from L2, and the state goes through global memory (L2) between steps.
// Every mbarrier wait is bounded (1 s); after a timeout the CTA raises bit 1
// of the error word, skips all further work but still passes every barrier,
// frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/sfp.h"
#include "sfp_device.cuh"
#include "sfp_fused.h"
#include "sfp_ptx.cuh"

namespace sfp {
namespace {

using namespace ptx;

constexpr int kRows = 128;                   // UMMA M = TMEM lanes
constexpr int kChains = 42;                  // most chains per tile (126 of 128 rows)
constexpr int kKB = 32;                      // K block: 32 FP32 = one 128-byte swizzle row
constexpr int kComputeWarps = 16;
constexpr int kCompute = 32 * kComputeWarps;  // 512 threads
constexpr int kThreads = 64 + kCompute;

// Shared memory of one CTA.  A stage holds [R (FP32, BF16 operands only)]
// [A hi][A lo][B hi][B lo] for one K block of 32: TF32 operands are FP32-sized
// with a 128-byte swizzle (the R tile is split in place in A hi); BF16
// operands are 2 bytes with a 64-byte swizzle, the FP32 R tile converted from
// its own staging tile.
template <int NB, bool BF>
struct FSmem {
    static constexpr int kEl = BF ? 2 : 4;
    static constexpr int kA = kRows * kKB * kEl;          // 16 KB (TF32) / 8 KB (BF16)
    static constexpr int kB = NB * kKB * kEl;             // NB x 128 B / NB x 64 B
    static constexpr int kR = BF ? kRows * kKB * 4 : 0;   // FP32 R staging (BF16)
    static constexpr int kStage = kR + 2 * kA + 2 * kB;
    static constexpr int kStages = BF ? (192 * 1024) / kStage : (NB == 256 ? 2 : NB == 128 ? 3 : 4);
    static constexpr int kRT = kRows * kKB * 4;           // an FP32 R block of the epilogue, 16 KB
    static constexpr int kU = kRows * kKB * 4;            // bond-vector staging
    static constexpr int kMisc = 4096;
    static constexpr int kBytes = kStages * kStage + kU + kMisc + 1024;
    static_assert(kStages <= 4, "stage barriers");
    static_assert(kStages * kStage >= NB / kKB * kRT, "the epilogue reloads the R tile into the stages");
};

// Byte offset of element (r, k), k < 32, in a 128-byte-swizzled K-major tile.
__device__ __forceinline__ uint32_t swz(int r, int k)
{
    return (uint32_t)(r * 128 + ((((k >> 2) ^ (r & 7)) << 4)) + ((k & 3) << 2));
}

// Byte offset of element (r, k), k < 32, in a 64-byte-swizzled K-major BF16 tile.
__device__ __forceinline__ uint32_t swz_bf(int r, int k)
{
    return (uint32_t)(r * 64 + ((((k >> 3) ^ ((r >> 1) & 3)) << 4)) + ((k & 7) << 1));
}

__device__ __forceinline__ uint16_t bf16_rn(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_f(uint16_t h) { return __bfloat162float(__ushort_as_bfloat16(h)); }

// Operand element (r, k) as hi / lo parts: TF32 (rna) or BF16 (round to nearest even).
template <bool BF>
__device__ __forceinline__ void put_hi_lo(uint8_t* hi, uint8_t* lo, int r, int k, float x)
{
    if constexpr (BF) {
        const uint16_t h = bf16_rn(x);
        const uint32_t o = swz_bf(r, k);
        *reinterpret_cast<uint16_t*>(hi + o) = h;
        *reinterpret_cast<uint16_t*>(lo + o) = bf16_rn(x - bf16_f(h));
    } else {
        const float h = tf32_rna(x);
        const uint32_t o = swz(r, k);
        *reinterpret_cast<float*>(hi + o) = h;
        *reinterpret_cast<float*>(lo + o) = tf32_rna(x - h);
    }
}

template <int NB, bool BF>
__global__ void __launch_bounds__(kThreads, 1)
k_fused_step(const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmRst,
             const __grid_constant__ CUtensorMap tmChiH, const __grid_constant__ CUtensorMap tmChiL,
             const __grid_constant__ CUtensorMap tmFH, const __grid_constant__ CUtensorMap tmFL, const FusedArgs a)
{
    using S = FSmem<NB, BF>;
    constexpr int ST = S::kStages;
    constexpr int KB = NB / kKB;        // inverse K blocks = forward bead blocks
    constexpr int NBLK = 3 * KB;        // inverse / noise blocks interleaved, then force blocks
    constexpr uint32_t kCols = 2 * NB;  // D_u in [0, NB), D_inc in [NB, 2 NB)

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* stage0 = smem;
    float* U = (float*)(smem + ST * S::kStage);
    uint8_t* misc = smem + ST * S::kStage + S::kU;
    uint32_t* s_job = (uint32_t*)misc;
    int64_t* s_step = (int64_t*)(misc + 256);
    double* s_shear = (double*)(misc + 640);
    float* s_dm = (float*)(misc + 1024);
    float* s_g = (float*)(misc + 2048);
    uint64_t* bars = (uint64_t*)(misc + 3072);
    int64_t* s_stop = (int64_t*)(misc + 3328);
    uint64_t* full = bars;              // TMA bytes landed                 (1 + tx)
    uint64_t* ready = bars + 4;         // A operand prepared by threads    (256)
    uint64_t* empty = bars + 8;         // MMAs done with the stage         (commit)
    uint64_t* u_done = bars + 12;       // all inverse MMAs done            (commit)
    uint64_t* inc_done = bars + 13;     // all forward MMAs done            (commit)
    uint64_t* r_full = bars + 14;       // R tile reloaded for the epilogue (1 + tx)
    uint64_t* epi_done = bars + 15;     // epilogue stored R, stages free   (1)
    uint32_t* tmem_slot = (uint32_t*)(bars + 16);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = blockIdx.x * a.cpt;
    const int Ct = min(a.cpt, a.C - c0);
    const int row0 = 3 * c0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&ready[s], kCompute);
            mbar_init(&empty[s], 1);
        }
        mbar_init(u_done, 1);
        mbar_init(inc_done, 1);
        mbar_init(r_full, 1);
        mbar_init(epi_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmR)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmRst)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmChiH)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmChiL)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmFH)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmFL)) : "memory");
    }
    for (int i = threadIdx.x; i < kChains; i += kThreads) {
        const bool live = i < Ct;
        s_job[i] = live ? a.job[c0 + i] : 0u;
        s_step[i] = live ? a.step[c0 + i] : 0;
        s_stop[i] = (live && a.stop) ? a.stop[c0 + i] : INT64_MAX;
        s_shear[i] = live ? a.shear[c0 + i] : 0.0;
    }
    for (int p = threadIdx.x; p < NB; p += kThreads) {
        s_dm[p] = a.dm[p];
        s_g[p] = a.g[p];
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(kCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t t_u = tmem, t_inc = tmem + NB;
    const bool has_shear = __syncthreads_or(threadIdx.x < Ct && s_shear[threadIdx.x] != 0.0) != 0;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
          bool ok = true;
          for (int sp = 0; sp < a.n_steps && ok; ++sp) {
            // the previous step's epilogue used the stage memory and stored R
            if (sp > 0 && !mbar_wait(epi_done, (sp - 1) & 1, a.err, abort_flag)) break;
            for (int blk = 0; blk < NBLK; ++blk) {
                const int gb = sp * NBLK + blk;
                const int s = gb % ST;
                const uint32_t ph = (gb / ST) & 1;
                if (!mbar_wait(&empty[s], ph ^ 1, a.err, abort_flag)) { ok = false; break; }
                uint8_t* st = stage0 + s * S::kStage;
                uint8_t* bh = st + S::kR + 2 * S::kA;
                uint8_t* bl = bh + S::kB;
                if (blk < 2 * KB && (blk & 1) == 0) {
                    const int nb = blk >> 1;          // inverse: R tile (FP32) and chi
                    mbar_expect_tx(&full[s], S::kRT + 2 * S::kB);
                    tma_load_2d(st, &tmR, &full[s], nb * kKB, row0);
                    tma_load_2d(bh, &tmChiH, &full[s], nb * kKB, 0);
                    tma_load_2d(bl, &tmChiL, &full[s], nb * kKB, 0);
                } else {
                    // noise block nb: rows w_p phi (t = 1); force block nb: rows h_p chi (t = 0)
                    const bool noise = blk < 2 * KB;
                    const int nb = noise ? blk >> 1 : blk - 2 * KB;
                    mbar_expect_tx(&full[s], 2 * S::kB);
                    tma_load_2d(bh, &tmFH, &full[s], nb * kKB, noise ? NB : 0);
                    tma_load_2d(bl, &tmFL, &full[s], nb * kKB, noise ? NB : 0);
                }
            }
            // every stage is free once the forward MMAs are done: reload the R tile
            // (KB column blocks of 128 rows x 32) there for the epilogue
            if (ok && mbar_wait(inc_done, sp & 1, a.err, abort_flag)) {
                mbar_expect_tx(r_full, KB * S::kRT);
                for (int k = 0; k < KB; ++k) tma_load_2d(stage0 + k * S::kRT, &tmR, r_full, k * kKB, row0);
            } else {
                ok = false;
            }
          }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = BF ? idesc_bf16(kRows, NB) : idesc_tf32(kRows, NB);
            bool ok = true;
            for (int sp = 0; sp < a.n_steps; ++sp) {
            for (int blk = 0; blk < NBLK; ++blk) {
                const int gb = sp * NBLK + blk;
                const int s = gb % ST;
                const uint32_t ph = (gb / ST) & 1;
                ok = ok && mbar_wait(&full[s], ph, a.err, abort_flag);
                ok = ok && mbar_wait(&ready[s], ph, a.err, abort_flag);
                if (ok) {
                    fence_after();
                    const uint32_t st = smem_u32(stage0 + s * S::kStage);
                    const uint32_t a_hi = st + S::kR, a_lo = a_hi + S::kA, b_hi = a_lo + S::kA, b_lo = b_hi + S::kB;
                    const bool inv = blk < 2 * KB && (blk & 1) == 0;
                    const uint32_t d = inv ? t_u : t_inc;
                    const bool first = blk <= 1;       // first inverse block, first noise block
                    if constexpr (BF) {
#pragma unroll
                        for (int kk = 0; kk < kKB / 16; ++kk) {
                            const uint32_t off = kk * 32;   // 16 BF16 = 32 bytes along K
                            mma_bf16(d, sdesc64(a_hi + off), sdesc64(b_lo + off), idesc, (first && kk == 0) ? 0u : 1u);
                            mma_bf16(d, sdesc64(a_lo + off), sdesc64(b_hi + off), idesc, 1u);
                            mma_bf16(d, sdesc64(a_hi + off), sdesc64(b_hi + off), idesc, 1u);
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < kKB / 8; ++kk) {
                            const uint32_t off = kk * 32;   // 8 TF32 = 32 bytes along K
                            mma_tf32(d, sdesc(a_hi + off), sdesc(b_lo + off), idesc, (first && kk == 0) ? 0u : 1u);
                            mma_tf32(d, sdesc(a_lo + off), sdesc(b_hi + off), idesc, 1u);
                            mma_tf32(d, sdesc(a_hi + off), sdesc(b_hi + off), idesc, 1u);
                        }
                    }
                }
                mma_commit(&empty[s]);
                if (blk == 2 * KB - 2) mma_commit(u_done);
            }
            mma_commit(inc_done);
            }
        }
    } else {
        // ---------------- compute warps 2..17
        const int cw = warp - 2;            // 0..15
        const int ct = threadIdx.x - 64;    // 0..511
        const int q = warp & 3;             // TMEM lane quarter this warp may access
        bool ok = true;

        constexpr int kPer = (kChains + kComputeWarps - 1) / kComputeWarps;   // 3
        // Each warp owns chains c = cw + 16 i (i < 3) and bead n = 32 nb + lane of
        // every force / noise block; values are computed into registers first and
        // written once the stage is free, so the arithmetic overlaps earlier MMAs.

        const int grp = cw >> 2;                      // 4 groups of 4 warps (one per lane quarter)
        const int row = 32 * q + lane;
        const int crow = row / 3, ax = row - 3 * (row / 3);
        const bool live = row < 3 * Ct;
        float* col0 = U;                              // D_inc[j][0] per row (epilogue)
        bool finite = true;
#pragma unroll 1
        for (int sp = 0; sp < a.n_steps; ++sp) {
        const int g0 = sp * NBLK;                     // global index of this step's first block
        // (1) per bead block nb: split the R tile of inverse block nb into TF32
        //     hi / lo (in place), and write noise block nb (Eq. b5)
#pragma unroll 1
        for (int nb = 0; nb < KB; ++nb) {
            const int n = nb * kKB + lane;
            float zz[kPer][3];
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int c = cw + kComputeWarps * i;
                zz[i][0] = zz[i][1] = zz[i][2] = 0.f;
                if (c < Ct) Normals<float>::draw(a.seed, s_job[c], s_step[c] + sp, (uint32_t)n, 0u, zz[i]);
            }
            {
                const int blk = g0 + 2 * nb, s = blk % ST;
                const uint32_t ph = (blk / ST) & 1;
                ok = ok && mbar_wait(&full[s], ph, a.err, abort_flag);
                if (ok && BF) {
                    // row ct/4, BF16 chunk ct%4 (8 values) from the FP32 staging tile
                    const uint8_t* r32 = stage0 + s * S::kStage;
                    uint8_t* ah = stage0 + s * S::kStage + S::kR;
                    uint8_t* al = ah + S::kA;
                    const int r = ct >> 2, c = ct & 3;
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const float4 x = *reinterpret_cast<const float4*>(r32 + swz(r, 8 * c + 4 * h2));
                        const float xs[4] = {x.x, x.y, x.z, x.w};
                        uint16_t hh[4], ll[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            hh[i] = bf16_rn(xs[i]);
                            ll[i] = bf16_rn(xs[i] - bf16_f(hh[i]));
                        }
                        hw[2 * h2] = (uint32_t)hh[0] | ((uint32_t)hh[1] << 16);
                        hw[2 * h2 + 1] = (uint32_t)hh[2] | ((uint32_t)hh[3] << 16);
                        lw[2 * h2] = (uint32_t)ll[0] | ((uint32_t)ll[1] << 16);
                        lw[2 * h2 + 1] = (uint32_t)ll[2] | ((uint32_t)ll[3] << 16);
                    }
                    const uint32_t o = swz_bf(r, 8 * c);
                    *reinterpret_cast<uint4*>(ah + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4*>(al + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    fence_proxy_async();
                } else if (ok) {
                    float4* ah = (float4*)(stage0 + s * S::kStage);
                    float4* al = (float4*)(stage0 + s * S::kStage + S::kA);
#pragma unroll
                    for (int i = 0; i < S::kA / 16 / kCompute; ++i) {
                        const int e = ct + kCompute * i;
                        const float4 x = ah[e];
                        float4 h, l;
                        h.x = tf32_rna(x.x); l.x = tf32_rna(x.x - h.x);
                        h.y = tf32_rna(x.y); l.y = tf32_rna(x.y - h.y);
                        h.z = tf32_rna(x.z); l.z = tf32_rna(x.z - h.z);
                        h.w = tf32_rna(x.w); l.w = tf32_rna(x.w - h.w);
                        ah[e] = h;
                        al[e] = l;
                    }
                    fence_proxy_async();
                }
                mbar_arrive(&ready[s]);
            }
            {
                const int blk = g0 + 2 * nb + 1, s = blk % ST;
                const uint32_t ph = (blk / ST) & 1;
                ok = ok && mbar_wait(&empty[s], ph ^ 1, a.err, abort_flag);
                if (ok) {
                    uint8_t* ah = stage0 + s * S::kStage + S::kR;
                    uint8_t* al = ah + S::kA;
#pragma unroll
                    for (int i = 0; i < kPer; ++i) {
                        const int c = cw + kComputeWarps * i;
                        if (c < a.cpt) {
#pragma unroll
                            for (int x = 0; x < 3; ++x) put_hi_lo<BF>(ah, al, 3 * c + x, lane, zz[i][x]);
                        }
                    }
                    fence_proxy_async();
                }
                mbar_arrive(&ready[s]);
            }
        }

        // (2) per bead block nb: bond vectors from D_u -> residual force v (Eq. e11)
        ok = ok && mbar_wait(u_done, sp & 1, a.err, abort_flag);
        fence_after();
#pragma unroll 1
        for (int nb = 0; nb < KB; ++nb) {
            const int n = nb * kKB + lane;
            if (cw < 4) {
                // rows 32q..32q+31 of D_u, columns 32nb..32nb+31 -> U (swizzled rows)
                const int r = 32 * q + lane;
                float v[16];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    tmem_ld16(t_u + ((uint32_t)(32 * q) << 16) + (uint32_t)(nb * kKB + 16 * h), v);
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4)
                        *reinterpret_cast<float4*>((uint8_t*)U + swz(r, 16 * h + 4 * k4)) =
                            make_float4(v[4 * k4], v[4 * k4 + 1], v[4 * k4 + 2], v[4 * k4 + 3]);
                }
            }
            named_bar(1, kCompute);
            float vv[kPer][3];
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int c = cw + kComputeWarps * i;
                float u[3] = {0.f, 0.f, 0.f};
                if (c < a.cpt) {
#pragma unroll
                    for (int x = 0; x < 3; ++x)
                        u[x] = *reinterpret_cast<const float*>((const uint8_t*)U + swz(3 * c + x, lane));
                }
                const bool live = c < Ct && n >= 1;
                const float s2 = live ? rsqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) - a.c12nu : 0.f;
#pragma unroll
                for (int x = 0; x < 3; ++x) vv[i][x] = live ? u[x] * s2 : 0.f;
            }
            named_bar(1, kCompute);   // U is free for the next bead block
            {
                const int blk = g0 + 2 * KB + nb, s = blk % ST;
                const uint32_t ph = (blk / ST) & 1;
                ok = ok && mbar_wait(&empty[s], ph ^ 1, a.err, abort_flag);
                if (ok) {
                    uint8_t* ah = stage0 + s * S::kStage + S::kR;
                    uint8_t* al = ah + S::kA;
#pragma unroll
                    for (int i = 0; i < kPer; ++i) {
                        const int c = cw + kComputeWarps * i;
                        if (c < a.cpt) {
#pragma unroll
                            for (int x = 0; x < 3; ++x) put_hi_lo<BF>(ah, al, 3 * c + x, lane, vv[i][x]);
                        }
                    }
                    fence_proxy_async();
                }
                mbar_arrive(&ready[s]);
            }
        }

        // (3) epilogue: R += -dm R + D_inc (+ shear) on the R tile that the producer
        // reloaded into the stage memory (KB blocks of [128 rows][32], swizzled),
        // in place, 16 columns at a time; then TMA-stored back (126 rows).
        ok = ok && mbar_wait(inc_done, sp & 1, a.err, abort_flag);
        ok = ok && mbar_wait(r_full, sp & 1, a.err, abort_flag);
        fence_after();
#pragma unroll 1
        for (int k = grp; k < NB / 16; k += kComputeWarps / 4) {
            const int p0 = 16 * k;
            uint8_t* blk = stage0 + (p0 / kKB) * S::kRT;
            const int kin = p0 % kKB;
            float d[16], r[16];
            tmem_ld16(t_inc + ((uint32_t)(32 * q) << 16) + (uint32_t)p0, d);
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
                const float4 x = *reinterpret_cast<const float4*>(blk + swz(row, kin + 4 * k4));
                r[4 * k4] = x.x; r[4 * k4 + 1] = x.y; r[4 * k4 + 2] = x.z; r[4 * k4 + 3] = x.w;
            }
            float ry[16];
            if (has_shear) {
                // start-of-step R^y of this chain (row 3c+1), read before anyone writes
                const int ry_row = min(3 * crow + 1, kRows - 1);
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    const float4 x = *reinterpret_cast<const float4*>(blk + swz(ry_row, kin + 4 * k4));
                    ry[4 * k4] = x.x; ry[4 * k4 + 1] = x.y; ry[4 * k4 + 2] = x.z; ry[4 * k4 + 3] = x.w;
                }
                named_bar(2 + grp, 128);
            }
            // a chain whose step counter has reached its stop step stays as it is
            const bool adv = live && s_step[crow] + sp < s_stop[crow];
            float o[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) o[i] = adv ? r[i] + fmaf(-s_dm[p0 + i], r[i], d[i]) : r[i];
            if (has_shear && adv && ax == 0) {
                const float sh = (float)s_shear[crow];
#pragma unroll
                for (int i = 0; i < 16; ++i) o[i] += sh * s_g[p0 + i] * ry[i];
            }
            if (p0 == 0) {
                col0[row] = d[0];
                o[0] = 0.f;
            }
            if (live) {
#pragma unroll
                for (int i = 0; i < 16; ++i) finite = finite && isfinite(o[i]);
            }
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4)
                *reinterpret_cast<float4*>(blk + swz(row, kin + 4 * k4)) =
                    make_float4(o[4 * k4], o[4 * k4 + 1], o[4 * k4 + 2], o[4 * k4 + 3]);
            if (has_shear) named_bar(2 + grp, 128);
        }
        fence_proxy_async();
        named_bar(1, kCompute);   // tile and col0 complete
        if (ct == 0) {
            if (ok) {
                for (int k = 0; k < KB; ++k) tma_store_2d(&tmRst, stage0 + k * S::kRT, k * kKB, row0);
                tma_store_commit();
                tma_store_wait();   // R is in global memory and the stages are free again
            }
            mbar_arrive(epi_done);
        }
        if (ok && grp == 0 && live && ax == 0 && s_step[crow] + sp < s_stop[crow]) {
            // centre of mass in FP64 (p = 0 of Eq. d3 with zeta_0 = 0)
            double* cm = a.com + 3 * (size_t)(c0 + crow);
            const double ycm = cm[1];
            cm[0] += (double)col0[row] * a.inv_sqrtM + s_shear[crow] * a.dtau * ycm;
            cm[1] += (double)col0[row + 1] * a.inv_sqrtM;
            cm[2] += (double)col0[row + 2] * a.inv_sqrtM;
        }
        named_bar(1, kCompute);   // col0 read before the next step reuses U
        }   // steps
        if (ok && grp == 0 && live && ax == 0)
            a.step[c0 + crow] = max(s_step[crow], min(s_step[crow] + (int64_t)a.n_steps, s_stop[crow]));
        if (!finite) atomicOr(a.err, 1);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

}  // namespace

struct FusedPlan {
    int M = 0, C = 0, cpt = kChains;
    bool bf16 = false;
    void* tab[4] = {nullptr, nullptr, nullptr, nullptr};    // chi_hi, chi_lo, F_hi, F_lo (TF32 or BF16)
    float* R = nullptr;
    CUtensorMap tmR, tmRst, tmChiH, tmChiL, tmFH, tmFL;
};

bool fused_supported(int M) { return M == 64 || M == 128 || M == 256; }

template <int NB, bool BF>
static cudaError_t set_smem()
{
    return cudaFuncSetAttribute(k_fused_step<NB, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, FSmem<NB, BF>::kBytes);
}

// 2-D BF16 table [rows][cols], box 32 cols x box_rows, 64-byte swizzle.
static int make_map_bf16(CUtensorMap* m, const void* base, int rows, int cols, int box_rows)
{
    auto fn = encode_fn();
    if (!fn) return report(SFP_ECUDA, "cuTensorMapEncodeTiled unavailable");
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kKB, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return report(SFP_ECUDA, "cuTensorMapEncodeTiled (bf16) failed");
    return SFP_OK;
}

static uint16_t bf16_host(double x)
{
    const float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);   // round to nearest even
    return (uint16_t)(u >> 16);
}

static double bf16_value(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

int fused_create(FusedPlan** out, int M, int C, const double* chi, const double* phi, const double* h,
                 const double* w, float* R, cudaStream_t stream, bool bf16)
{
    *out = nullptr;
    if (!fused_supported(M)) return report(SFP_ENOTSUP, "the fused step needs M in {64, 128, 256}");
    FusedPlan* p = new FusedPlan();
    p->M = M;
    p->C = C;
    p->R = R;
    p->bf16 = bf16;
    // one wave: chains per tile = ceil(C / SMs), at most 42 (fused_set_tile changes it)
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 148;
    p->cpt = std::max(1, std::min(kChains, (C + sms - 1) / sms));
    const size_t mm = (size_t)M * M;
    // chi [n][p] (row n = 0 and column p = 0 are zero) and F [2M][M]:
    // F[p][n] = h_p chi[n][p] (Eq. f2 weight on DeltaH = chi^T v, Eq. e11),
    // F[M + p][n] = w_p phi[n][p] (Eq. d6 weight on Z = phi^T z, Eq. c4).
    std::vector<double> F(2 * mm);
    for (int q = 0; q < M; ++q)
        for (int n = 0; n < M; ++n) {
            F[(size_t)q * M + n] = h[q] * chi[(size_t)n * M + q];
            F[mm + (size_t)q * M + n] = w[q] * phi[(size_t)n * M + q];
        }
    const double* src[2] = {chi, F.data()};
    const size_t cnt[2] = {mm, 2 * mm};
    const size_t el = bf16 ? 2 : 4;
    for (int t = 0; t < 2; ++t) {
        std::vector<float> hi(cnt[t]), lo(cnt[t]);
        std::vector<uint16_t> hb(bf16 ? cnt[t] : 0), lb(bf16 ? cnt[t] : 0);
        for (size_t i = 0; i < cnt[t]; ++i) {
            if (bf16) {
                hb[i] = bf16_host(src[t][i]);
                lb[i] = bf16_host(src[t][i] - bf16_value(hb[i]));
            } else {
                hi[i] = tf32_round_host(src[t][i]);
                lo[i] = tf32_round_host(src[t][i] - (double)hi[i]);
            }
        }
        for (int k = 0; k < 2; ++k) {
            void*& d = p->tab[2 * t + k];
            const void* hsrc = bf16 ? (const void*)(k == 0 ? hb.data() : lb.data())
                                    : (const void*)(k == 0 ? hi.data() : lo.data());
            if (cudaMalloc(&d, cnt[t] * el) != cudaSuccess) {
                fused_destroy(p);
                return report(SFP_ENOMEM, "fused-step table allocation failed");
            }
            if (cudaMemcpyAsync(d, hsrc, cnt[t] * el, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess) {
                fused_destroy(p);
                return report(SFP_ECUDA, "fused-step table upload failed");
            }
        }
    }
    int rc;
    // the store box is the tile's 3 cpt rows: a tile must not write the next tile's chains
    if ((rc = make_map_2d(&p->tmR, R, 3 * C, M, kRows)) || (rc = make_map_2d(&p->tmRst, R, 3 * C, M, 3 * p->cpt))) {
        fused_destroy(p);
        return rc;
    }
    if (bf16)
        rc = make_map_bf16(&p->tmChiH, p->tab[0], M, M, M) ? -1 : make_map_bf16(&p->tmChiL, p->tab[1], M, M, M) ? -1 :
             make_map_bf16(&p->tmFH, p->tab[2], 2 * M, M, M) ? -1 : make_map_bf16(&p->tmFL, p->tab[3], 2 * M, M, M);
    else
        rc = make_map_2d(&p->tmChiH, (const float*)p->tab[0], M, M, M) ? -1 :
             make_map_2d(&p->tmChiL, (const float*)p->tab[1], M, M, M) ? -1 :
             make_map_2d(&p->tmFH, (const float*)p->tab[2], 2 * M, M, M) ? -1 :
             make_map_2d(&p->tmFL, (const float*)p->tab[3], 2 * M, M, M);
    if (rc) {
        fused_destroy(p);
        return SFP_ECUDA;
    }
    cudaError_t e;
    if (bf16) e = M == 256 ? set_smem<256, true>() : M == 128 ? set_smem<128, true>() : set_smem<64, true>();
    else e = M == 256 ? set_smem<256, false>() : M == 128 ? set_smem<128, false>() : set_smem<64, false>();
    if (e != cudaSuccess) {
        fused_destroy(p);
        return report(SFP_ECUDA, "cudaFuncSetAttribute (fused step) failed");
    }
    *out = p;
    return SFP_OK;
}

int fused_step(FusedPlan* p, const FusedArgs& args, cudaStream_t stream)
{
    if (args.cpt != p->cpt) return report(SFP_EINVAL, "fused step: chains per tile differ from the plan's");
    const dim3 grid((unsigned)((p->C + p->cpt - 1) / p->cpt));
#define SFP_FUSED_LAUNCH(NBV, BFV)                                                                   \
    k_fused_step<NBV, BFV><<<grid, kThreads, FSmem<NBV, BFV>::kBytes, stream>>>(p->tmR, p->tmRst, p->tmChiH, \
                                                                            p->tmChiL, p->tmFH, p->tmFL, args)
    switch (p->M * 2 + (p->bf16 ? 1 : 0)) {
        case 512: SFP_FUSED_LAUNCH(256, false); break;
        case 513: SFP_FUSED_LAUNCH(256, true); break;
        case 256: SFP_FUSED_LAUNCH(128, false); break;
        case 257: SFP_FUSED_LAUNCH(128, true); break;
        case 128: SFP_FUSED_LAUNCH(64, false); break;
        case 129: SFP_FUSED_LAUNCH(64, true); break;
        default: return report(SFP_ENOTSUP, "unsupported fused-step length");
    }
#undef SFP_FUSED_LAUNCH
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report(SFP_ECUDA, cudaGetErrorString(e));
    return SFP_OK;
}

int fused_tile(const FusedPlan* p) { return p->cpt; }

size_t fused_bytes(const FusedPlan* p) { return p ? (size_t)6 * p->M * p->M * (p->bf16 ? 2 : 4) : 0; }

int fused_set_tile(FusedPlan* p, int cpt)
{
    if (cpt < 1 || cpt > kChains) return report(SFP_EINVAL, "chains per tile must be 1..42");
    CUtensorMap m;
    const int rc = make_map_2d(&m, p->R, 3 * p->C, p->M, 3 * cpt);
    if (rc) return rc;
    p->tmRst = m;
    p->cpt = cpt;
    return SFP_OK;
}

void fused_destroy(FusedPlan* p)
{
    if (!p) return;
    for (void* t : p->tab)
        if (t) cudaFree(t);
    delete p;
}

}  // namespace sfp
