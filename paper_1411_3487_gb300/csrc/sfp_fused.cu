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
#include <algorithm>
#include <cstdint>
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

template <int NB>
struct FSmem {
    static constexpr int kStages = NB == 256 ? 2 : NB == 128 ? 3 : 4;
    static constexpr int kA = kRows * kKB * 4;            // 16 KB
    static constexpr int kB = NB * kKB * 4;               // NB x 128 B
    static constexpr int kStage = 2 * kA + 2 * kB;        // A hi, A lo, B hi, B lo
    static constexpr int kU = kRows * kKB * 4;            // bond-vector staging
    static constexpr int kMisc = 4096;
    static constexpr int kBytes = kStages * kStage + kU + kMisc + 1024;
};

// Byte offset of element (r, k), k < 32, in a 128-byte-swizzled K-major tile.
__device__ __forceinline__ uint32_t swz(int r, int k)
{
    return (uint32_t)(r * 128 + ((((k >> 2) ^ (r & 7)) << 4)) + ((k & 3) << 2));
}

__device__ __forceinline__ void put_hi_lo(uint8_t* hi, uint8_t* lo, int r, int k, float x)
{
    const float h = tf32_rna(x);
    const uint32_t o = swz(r, k);
    *reinterpret_cast<float*>(hi + o) = h;
    *reinterpret_cast<float*>(lo + o) = tf32_rna(x - h);
}

template <int NB>
__global__ void __launch_bounds__(kThreads, 1)
k_fused_step(const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmRst,
             const __grid_constant__ CUtensorMap tmChiH, const __grid_constant__ CUtensorMap tmChiL,
             const __grid_constant__ CUtensorMap tmFH, const __grid_constant__ CUtensorMap tmFL, const FusedArgs a)
{
    using S = FSmem<NB>;
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
                uint8_t* bh = st + 2 * S::kA;
                uint8_t* bl = bh + S::kB;
                if (blk < 2 * KB && (blk & 1) == 0) {
                    const int nb = blk >> 1;          // inverse: R tile and chi
                    mbar_expect_tx(&full[s], S::kA + 2 * S::kB);
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
                mbar_expect_tx(r_full, KB * S::kA);
                for (int k = 0; k < KB; ++k) tma_load_2d(stage0 + k * S::kA, &tmR, r_full, k * kKB, row0);
            } else {
                ok = false;
            }
          }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32(kRows, NB);
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
                    const uint32_t a_hi = st, a_lo = st + S::kA, b_hi = st + 2 * S::kA, b_lo = b_hi + S::kB;
                    const bool inv = blk < 2 * KB && (blk & 1) == 0;
                    const uint32_t d = inv ? t_u : t_inc;
                    const bool first = blk <= 1;       // first inverse block, first noise block
#pragma unroll
                    for (int kk = 0; kk < kKB / 8; ++kk) {
                        const uint32_t off = kk * 32;   // 8 TF32 = 32 bytes along K
                        mma_tf32(d, sdesc(a_hi + off), sdesc(b_lo + off), idesc, (first && kk == 0) ? 0u : 1u);
                        mma_tf32(d, sdesc(a_lo + off), sdesc(b_hi + off), idesc, 1u);
                        mma_tf32(d, sdesc(a_hi + off), sdesc(b_hi + off), idesc, 1u);
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
                if (ok) {
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
                    uint8_t* ah = stage0 + s * S::kStage;
                    uint8_t* al = ah + S::kA;
#pragma unroll
                    for (int i = 0; i < kPer; ++i) {
                        const int c = cw + kComputeWarps * i;
                        if (c < a.cpt) {
#pragma unroll
                            for (int x = 0; x < 3; ++x) put_hi_lo(ah, al, 3 * c + x, lane, zz[i][x]);
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
                    uint8_t* ah = stage0 + s * S::kStage;
                    uint8_t* al = ah + S::kA;
#pragma unroll
                    for (int i = 0; i < kPer; ++i) {
                        const int c = cw + kComputeWarps * i;
                        if (c < a.cpt) {
#pragma unroll
                            for (int x = 0; x < 3; ++x) put_hi_lo(ah, al, 3 * c + x, lane, vv[i][x]);
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
            uint8_t* blk = stage0 + (p0 / kKB) * S::kA;
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
                for (int k = 0; k < KB; ++k) tma_store_2d(&tmRst, stage0 + k * S::kA, k * kKB, row0);
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
    float* tab[4] = {nullptr, nullptr, nullptr, nullptr};   // chi_hi, chi_lo, F_hi, F_lo
    float* R = nullptr;
    CUtensorMap tmR, tmRst, tmChiH, tmChiL, tmFH, tmFL;
};

bool fused_supported(int M) { return M == 64 || M == 128 || M == 256; }

template <int NB>
static cudaError_t set_smem()
{
    return cudaFuncSetAttribute(k_fused_step<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, FSmem<NB>::kBytes);
}

int fused_create(FusedPlan** out, int M, int C, const double* chi, const double* phi, const double* h,
                 const double* w, float* R, cudaStream_t stream)
{
    *out = nullptr;
    if (!fused_supported(M)) return report(SFP_ENOTSUP, "the fused step needs M in {64, 128, 256}");
    FusedPlan* p = new FusedPlan();
    p->M = M;
    p->C = C;
    p->R = R;
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
    for (int t = 0; t < 2; ++t) {
        std::vector<float> hi(cnt[t]), lo(cnt[t]);
        for (size_t i = 0; i < cnt[t]; ++i) {
            hi[i] = tf32_round_host(src[t][i]);
            lo[i] = tf32_round_host(src[t][i] - (double)hi[i]);
        }
        for (int k = 0; k < 2; ++k) {
            float*& d = p->tab[2 * t + k];
            if (cudaMalloc(&d, cnt[t] * sizeof(float)) != cudaSuccess) {
                fused_destroy(p);
                return report(SFP_ENOMEM, "fused-step table allocation failed");
            }
            if (cudaMemcpyAsync(d, k == 0 ? hi.data() : lo.data(), cnt[t] * sizeof(float), cudaMemcpyHostToDevice,
                                stream) != cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess) {
                fused_destroy(p);
                return report(SFP_ECUDA, "fused-step table upload failed");
            }
        }
    }
    int rc;
    // the store box is the tile's 3 cpt rows: a tile must not write the next tile's chains
    if ((rc = make_map_2d(&p->tmR, R, 3 * C, M, kRows)) || (rc = make_map_2d(&p->tmRst, R, 3 * C, M, 3 * p->cpt)) ||
        (rc = make_map_2d(&p->tmChiH, p->tab[0], M, M, M)) ||
        (rc = make_map_2d(&p->tmChiL, p->tab[1], M, M, M)) || (rc = make_map_2d(&p->tmFH, p->tab[2], 2 * M, M, M)) ||
        (rc = make_map_2d(&p->tmFL, p->tab[3], 2 * M, M, M))) {
        fused_destroy(p);
        return rc;
    }
    const cudaError_t e = M == 256 ? set_smem<256>() : M == 128 ? set_smem<128>() : set_smem<64>();
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
    switch (p->M) {
        case 256:
            k_fused_step<256><<<grid, kThreads, FSmem<256>::kBytes, stream>>>(p->tmR, p->tmRst, p->tmChiH, p->tmChiL, p->tmFH, p->tmFL, args);
            break;
        case 128:
            k_fused_step<128><<<grid, kThreads, FSmem<128>::kBytes, stream>>>(p->tmR, p->tmRst, p->tmChiH, p->tmChiL, p->tmFH, p->tmFL, args);
            break;
        case 64:
            k_fused_step<64><<<grid, kThreads, FSmem<64>::kBytes, stream>>>(p->tmR, p->tmRst, p->tmChiH, p->tmChiL, p->tmFH, p->tmFL, args);
            break;
        default:
            return report(SFP_ENOTSUP, "unsupported fused-step length");
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report(SFP_ECUDA, cudaGetErrorString(e));
    return SFP_OK;
}

int fused_tile(const FusedPlan* p) { return p->cpt; }

size_t fused_bytes(const FusedPlan* p) { return p ? (size_t)6 * p->M * p->M * sizeof(float) : 0; }

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
    for (float* t : p->tab)
        if (t) cudaFree(t);
    delete p;
}

}  // namespace sfp
