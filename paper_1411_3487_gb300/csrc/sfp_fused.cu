// sfp_fused.cu -- mode-space steps (Sec. 4) for tiles of up to 40 chains of
// the SFP_FP32 and SFP_MIXED_BF16 paths, M = 64, 128, 256 or 512 beads,
// n_steps per launch.
//
// The 128 TMEM lanes hold a tile's chain-axis rows: lane quarter q (rows
// 32 q .. 32 q + 31) holds chains q cpq .. q cpq + cpq - 1 of the tile
// (cpq <= 10 chains per quarter), chain k of the quarter in rows 32 q + 3 k +
// alpha; the rest of a quarter is padding.  A chain's three axes therefore sit
// in three lanes of one warp, so |u_n| and the shear term take warp shuffles
// instead of a trip through shared memory.  Bead / mode indices are TMEM
// columns.  Fewer chains per tile give more CTAs on small batches: the MMA
// time of a tile is fixed by its 128 rows, the noise and force work is not.
// Per step and tile:
//   inverse  (Eq. e5)   D_u[j][n]   = sum_p R[j][p] chi[n][p]            (bonds)
//   force    (Eq. e11)  v_n = u_n (1/|u_n| - (1 - 2 nu)),  v_0 = 0
//   noise    (Eq. b5)   z_n ~ N(0,1), Philox keyed by (seed, job, step, n)
//   forward  (Eqs. c4, e11, d6, f2)
//            D_inc[j][p] = sum_n v[j][n] h_p chi[n][p] + sum_n z[j][n] w_p phi[n][p]
//                        = h_p DeltaH_p + w_p Z_p
//   update   (Eqs. d3, btum)  R_p += -(1 - e^{-zeta_p dtau}) R_p + D_inc_p
//                             (+ shear g_p R^y_p on the x rows); p = 0 feeds the
//                             FP64 centre of mass.
// DeltaH is never formed on its own: Eq. e11 makes it chi^T v, so the
// bead-space stencil of the staged path is not needed, and h_p, w_p are folded
// into one stacked table so a single accumulator holds the whole increment.
//
// Both contractions run on the tcgen05 tensor cores as three passes
// (A_hi B_lo + A_lo B_hi + A_hi B_hi, FP32 accumulate in TMEM): TF32 parts
// (kind::tf32) for SFP_FP32, BF16 parts (kind::f16) for SFP_MIXED_BF16.
// Roles (640 threads):
//   warp 0       TMA producer: R tiles and chi hi/lo (inverse), F hi/lo (forward)
//   warp 1       TMEM allocation; one thread issues every MMA and commit
//   warps 2..9   compute: split the R tiles into hi/lo, read D_u (two warps per
//                lane quarter) and write the force blocks, epilogue from D_inc
//   warps 10..19 noise: Philox / Box-Muller normals written as the noise
//                blocks; the most arithmetic of a step, on warps of their own
//                so that it runs beside the R split and the force
// Block order (K blocks of 32; sched_decode): the inverse blocks first, with
// half of the noise blocks between them, then the force blocks with the other
// half.  The noise half of the forward contraction does not depend on the
// state; only the force blocks wait for the bond vectors.
// Chains never interact, so a CTA runs all n_steps of its tile without any
// grid-wide synchronisation: TMEM stays allocated, the tables stream again
// from L2, and the state goes through global memory (L2) between steps.
//
// M = 512 (k_fused_pair): D_u and D_inc would take 1024 TMEM columns, twice an SM's
// 512, so a cluster of two CTAs shares each tile.  CTA h (cluster rank) holds
// bonds and modes 256 h .. 256 h + 255 (D_u and D_inc halves of 256 columns,
// B operands = those rows of chi and F) and runs all 3 x 16 K blocks of a
// step.  The A operand of every block (R split, force or noise, all 128
// rows) is needed by both: each block has one owner (blocks of schedule index
// i are owned by CTA i & 1), which writes it into its own stage; the MMA
// thread then bulk-copies it into the same stage of the other CTA (completing
// as transaction bytes of that CTA's `full` barrier) as soon as it is written:
// its loop polls the next block to multiply and the next block to send, so
// neither waits for the other.  Force blocks are owned
// by the CTA whose D_u half holds their bonds.  A stage is reused only when
// the MMAs of both CTAs are done with it (`empty` counts two multicast
// commits), and a step's first blocks are written only after both CTAs'
// epilogues of the previous step (`peer_epi`).  Each CTA updates its own mode
// half; rank 0 holds the centre of mass.
// Every wait is bounded (1 s); after a timeout the CTA raises bit 1 of the
// error word and sets its abort flag; from then on every wait of the CTA gives
// up at once, and a role that has given up makes no further arrival, commit
// or copy (arrivals of different blocks could otherwise meet in one phase of a
// barrier and exceed its count).  The CTA frees its TMEM and returns.
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
constexpr int kChains = 40;                  // most chains per tile: 10 per TMEM lane quarter
constexpr int kQuarter = 32 * 128;           // bytes of 32 rows of a 128-byte-swizzled tile
constexpr int kKB = 32;                      // K block: 32 FP32 = one 128-byte swizzle row
constexpr int kComputeWarps = 8;             // R split, residual force, epilogue
constexpr int kNoiseWarps = 10;              // Philox normals of the noise blocks
constexpr int kCompute = 32 * kComputeWarps;  // 256 threads
constexpr int kThreads = 64 + kCompute + 32 * kNoiseWarps;
// A stage's A operand is written by one group, whose warps arrive once each
// (lane 0, after __syncwarp) with weights that add up to the same count.
constexpr int kReadyCount = kComputeWarps * kNoiseWarps;
// Noise warps 10 + 4 t + u share lane quarter (2 + u) & 3: how many there are for
// each u, and so for each quarter q (u = (q + 2) & 3).
__device__ constexpr int kNoiseInQ[4] = {(kNoiseWarps + 3) / 4, (kNoiseWarps + 2) / 4, (kNoiseWarps + 1) / 4,
                                         kNoiseWarps / 4};
static_assert(2 + kComputeWarps == 10 && kComputeWarps == 8, "warp numbering of the quarters");

// Shared memory of one CTA.  A stage holds [R][A hi][A lo][B hi][B lo] for one
// K block of 32: TF32 operands are FP32-sized with a 128-byte swizzle (the R
// tile of an inverse block lands in A hi and is split in place); BF16
// operands are 2 bytes with a 64-byte swizzle, and the FP32 R tile (16 KB)
// either has a staging area R of its own (RS) or lands in A hi + A lo, which
// the compute warps read out in full before they write the hi and lo parts
// over it.  The single-CTA kernel stages R on its own at 64 and 128 beads
// (four stages either way) and in place at 256 beads, where that gives four
// stages of 48 KB instead of three of 64 KB (24.2 -> 23.1 us per step at
// 4096 x 256 bp; with mode-keyed noise, whose steps have no noise blocks,
// three stages stay faster: 24.0 against 24.5 us); the 512-bead kernel splits
// in place.
template <int NB, bool BF, bool MZ = false> constexpr bool kRS = BF && (NB != 256 || MZ);
template <int NB, bool BF, bool RS>
struct FSmem {
    static constexpr int kEl = BF ? 2 : 4;
    static constexpr int kA = kRows * kKB * kEl;          // 16 KB (TF32) / 8 KB (BF16)
    static constexpr int kB = NB * kKB * kEl;             // NB x 128 B / NB x 64 B
    static constexpr int kR = RS ? kRows * kKB * 4 : 0;   // FP32 R staging (BF16, RS)
    static constexpr int kStage = kR + 2 * kA + 2 * kB;
    static_assert(RS || kRows * kKB * 4 <= 2 * kA, "an FP32 R tile fits the A operand region");
    static constexpr int kStages = BF ? ((192 * 1024) / kStage < 4 ? (192 * 1024) / kStage : 4)
                                      : (NB == 256 ? 2 : NB == 128 ? 3 : 4);
    static constexpr int kRT = kRows * kKB * 4;           // an FP32 R block of the epilogue, 16 KB
    static constexpr int kMisc = 5120;   // per-chain keys, steps, shear, stops; tables; barriers
    static constexpr int kBytes = kStages * kStage + kMisc + 1024;
    static_assert(kBytes <= 227 * 1024, "shared memory of one CTA");
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

// Order of the 3 KB blocks of one step (KB = NB / 32 bead blocks, H = KB / 2).
// Inverse blocks I_k (R chi^T into D_u) come first, noise blocks N_j (w phi^T z)
// and force blocks F_k (h chi^T v) accumulate into D_inc.  The noise blocks are
// spread over both phases so that the noise warps draw while the compute warps
// split R (phase 1) or form the force (phase 2):
//   phase 1: I_0 N_0 I_1 | I_2 N_1 I_3 | ... (3 H blocks, ends with I_{KB-1})
//   phase 2: F_0 N_H | F_1 N_{H+1} | ... | F_{H-1} N_{KB-1} | F_H ... F_{KB-1}
// With FILL = F > 0, N_H .. N_{H+F-1} move to the end of phase 1, where they
// keep the tensor pipe busy while the compute warps read the bond vectors out
// (the TF32 kernel's MMAs take twice as long, so there the pipe is the scarcer
// resource; it uses F = 1, measured faster than F = 0 or 2; BF16 uses F = 0;
// the 512-bead kernel, whose phases are twice as long, F = 4 with BF16 (289
// against 295 us per step at F = 0; 1, 2, 3, 5, 6, 8 in between) and F = 1
// with TF32):
//   ... I_{KB-1} N_H .. N_{H+F-1} | F_0 N_{H+F} | ... | F_{H-F-1} N_{KB-1} | F_{H-F} ... F_{KB-1}
template <int KB, int FILL>
__device__ __forceinline__ void sched_decode(int blk, int& kind, int& nb)   // kind: 0 I, 1 N, 2 F
{
    constexpr int H = KB / 2;
    constexpr int P = FILL < H ? FILL : H;   // noise blocks moved into phase 1's tail
    if (blk < 3 * H) {
        const int m = blk / 3, r = blk - 3 * (blk / 3);
        kind = r == 1 ? 1 : 0;
        nb = r == 0 ? 2 * m : r == 1 ? m : 2 * m + 1;
    } else if (blk < 3 * H + P) {
        kind = 1;
        nb = H + (blk - 3 * H);
    } else {
        const int b = blk - 3 * H - P;
        if (b < 2 * (H - P)) {
            kind = (b & 1) ? 1 : 2;
            nb = (b & 1) ? H + P + (b >> 1) : b >> 1;
        } else {
            kind = 2;
            nb = b - (H - P);
        }
    }
}
template <int KB> __device__ __forceinline__ int sched_inv(int k) { return 3 * (k >> 1) + ((k & 1) ? 2 : 0); }
// With mode-keyed noise (MZ) a step has no noise blocks: I_0 .. I_{KB-1}, then F_0 .. F_{KB-1}.
template <int KB, int FILL, bool MZ>
__device__ __forceinline__ void sched_decode_any(int blk, int& kind, int& nb)
{
    if constexpr (MZ) {
        kind = blk < KB ? 0 : 2;
        nb = blk < KB ? blk : blk - KB;
    } else {
        sched_decode<KB, FILL>(blk, kind, nb);
    }
}
template <int KB, int FILL> __device__ __forceinline__ int sched_noise(int j)
{
    constexpr int H = KB / 2, P = FILL < H ? FILL : H;
    return j < H ? 3 * j + 1 : j < H + P ? 3 * H + (j - H) : 3 * H + P + 2 * (j - H - P) + 1;
}
template <int KB, int FILL> __device__ __forceinline__ int sched_force(int k)
{
    constexpr int H = KB / 2, P = FILL < H ? FILL : H;
    return k < H - P ? 3 * H + P + 2 * k : 3 * H + P + 2 * (H - P) + (k - (H - P));
}

// 512 beads: bead block of force block k (schedule index).  CTA h owns the
// force blocks of k = h mod 2, and its D_u half holds bond blocks 8 h .. 8 h + 7.
template <int KBL> __device__ __forceinline__ int force_bonds(int k)
{
    return KBL * (k & 1) + (k >> 1);
}

// Noise of one 32-bead block of a tile (Eq. b5).  The normals of a chain and
// step are numbered k = 3 n + alpha, four per Philox call, so beads
// 32 jb .. 32 jb + 31 are calls 24 jb .. 24 jb + 23 of every chain.  The tile's
// cpt x 24 (chain, call) items are cut into chunks of 32, one item per lane
// (cpt is a multiple of 4, so the chunks are full); chunk h of the noise
// warps' block number qn goes to noise warp (h + qn) mod kNoiseWarps, so that
// the warp holding one chunk more than the others changes from block to block.
// Items of chains past the tile's last chain (a partial tile) are drawn for
// that slot's empty key and written as zeros.
constexpr int kCallsPerBlock = kKB * 3 / 4;                                         // 24
constexpr int kChunksPerWarp = ((kChains * kCallsPerBlock + 31) / 32 + kNoiseWarps - 1) / kNoiseWarps;
static_assert(kChains % 4 == 0 && (4 * kCallsPerBlock) % 32 == 0, "full chunks");

__device__ __forceinline__ int noise_h0(int nw, int qn) { return (nw + kNoiseWarps - qn % kNoiseWarps) % kNoiseWarps; }

// One item: four normals of Philox call `call` of chain slot cl (zeros past the tile's chains).
__device__ __forceinline__ void noise_item(float (&z)[4], int h, int jb, int sp, int lane, int Ct, uint32_t seed,
                                           const uint32_t* s_job, const int64_t* s_step, uint32_t tag = 0u)
{
    const int f = 32 * h + lane;
    const int cl = f / kCallsPerBlock, call = f - kCallsPerBlock * cl;
    Normals<float>::draw4(seed, s_job[cl], s_step[cl] + sp, (uint32_t)(kCallsPerBlock * jb + call), tag, z);
    if (cl >= Ct) z[0] = z[1] = z[2] = z[3] = 0.f;
}

__device__ __forceinline__ void noise_draw(float (&zz)[kChunksPerWarp][4], int nw, int qn, int jb, int sp,
                                           int lane, int cpt, int Ct, uint32_t seed, const uint32_t* s_job,
                                           const int64_t* s_step, uint32_t tag = 0u)
{
    static_assert(kChunksPerWarp == 3, "the draw below handles up to three chunks per warp");
    const int nch = cpt * kCallsPerBlock / 32;
    const int h0 = noise_h0(nw, qn);
    // The warp's first two chunks are drawn in one straight-line block, so that
    // their Philox rounds interleave; the branches are the same for the whole warp.
    if (h0 + kNoiseWarps < nch) {
        noise_item(zz[0], h0, jb, sp, lane, Ct, seed, s_job, s_step, tag);
        noise_item(zz[1], h0 + kNoiseWarps, jb, sp, lane, Ct, seed, s_job, s_step, tag);
        if (h0 + 2 * kNoiseWarps < nch)
            noise_item(zz[2], h0 + 2 * kNoiseWarps, jb, sp, lane, Ct, seed, s_job, s_step, tag);
    } else if (h0 < nch) {
        noise_item(zz[0], h0, jb, sp, lane, Ct, seed, s_job, s_step, tag);
    }
}

// The drawn items as hi / lo parts of the block's A operand: value e of item
// (chain cl, call) is normal k = 4 call + e, i.e. bead k / 3 of the block (the
// column) and axis k % 3 of the chain (row 32 quarter + 3 slot + axis).
template <bool BF>
__device__ __forceinline__ void noise_put(uint8_t* ah, uint8_t* al, const float (&zz)[kChunksPerWarp][4], int nw,
                                          int qn, int lane, int cpt, const int* s_rowb)
{
    const int nch = cpt * kCallsPerBlock / 32;
    const int h0 = noise_h0(nw, qn);
#pragma unroll
    for (int i = 0; i < kChunksPerWarp; ++i) {
        const int h = h0 + kNoiseWarps * i;
        if (h < nch) {
            const int f = 32 * h + lane;
            const int cl = f / kCallsPerBlock, call = f - kCallsPerBlock * cl;
            const int rb = s_rowb[cl];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * call + e, n = k / 3;
                put_hi_lo<BF>(ah, al, rb + (k - 3 * n), n, zz[i][e]);
            }
        }
    }
}

// The step of the 64-, 128- and 256-bead chains: tile `tile` (chains
// tile * cpt ...) through a.n_steps steps on one CTA.  TWO (BF16 only): two
// passes, A_lo B_hi + A_hi B_hi, the tables taken as their BF16 hi part alone
// (SFP_MIXED_BF16_2).  The caller allocates the 2 NB TMEM columns at `tmem`
// and passes the CTA's 1024-byte-aligned dynamic shared memory.  The barriers
// are initialised here, and every arrival on them has landed before the
// function returns (the producer waits for the MMAs' last commits), so a
// persistent kernel may run another tile in the same shared memory.  Returns
// false if a wait gave up.
template <int NB, bool BF, bool TWO, bool MZ = false>
__device__ __forceinline__ bool fused_tile(const CUtensorMap& tmR, const CUtensorMap& tmChiH,
                                           const CUtensorMap& tmChiL, const CUtensorMap& tmFH,
                                           const CUtensorMap& tmFL, const FusedArgs& a, int tile, uint8_t* smem,
                                           uint32_t tmem)
{
    using S = FSmem<NB, BF, kRS<NB, BF, MZ>>;
    constexpr int ST = S::kStages;
    constexpr int KB = NB / kKB;        // inverse K blocks = forward bead blocks
    constexpr int NBLK = MZ ? 2 * KB : 3 * KB;   // blocks of one step, in the order of sched_decode (MZ: sched_mz)
    static_assert(KB % 2 == 0, "the block schedule pairs bead blocks");
    static_assert(ST <= NBLK, "the last ST blocks of a step release every stage");

    uint8_t* stage0 = smem;
    uint8_t* misc = smem + ST * S::kStage;
    uint32_t* s_job = (uint32_t*)misc;
    int64_t* s_step = (int64_t*)(misc + 256);
    double* s_shear = (double*)(misc + 576);
    int64_t* s_stop = (int64_t*)(misc + 896);
    float* s_dm = (float*)(misc + 1216);        // NB <= 256
    float* s_g = (float*)(misc + 2240);
    uint64_t* bars = (uint64_t*)(misc + 3264);
    int* s_rowb = (int*)(misc + 3584);          // first A-operand row of each chain slot
    float* s_w = (float*)(misc + 4096);         // MZ: w_p (Eq. d6; w_0 of the centre of mass), NB <= 256
    uint64_t* full = bars;              // TMA bytes landed                 (1 + tx)
    uint64_t* ready = bars + 4;         // A operand written by one group   (kReadyCount)
    uint64_t* empty = bars + 8;         // MMAs done with the stage         (commit)
    uint64_t* u_done = bars + 12;       // all inverse MMAs done            (commit)
    uint64_t* inc_done = bars + 13;     // all forward MMAs done            (commit)
    uint64_t* epi_done = bars + 15;     // epilogue stored R, stages free   (every worker warp)
    uint32_t* flags = (uint32_t*)(bars + 16);
    volatile int* abort_flag = (volatile int*)(flags + 1);
    int* s_freed = (int*)(flags + 2);   // last block whose stage the producer saw released
    uint64_t* r_blk = bars + 18;        // R column block k reloaded for the epilogue (1 + tx), k < KB
    uint64_t* never = bars + 26;        // nothing arrives here (the stall test)
    uint64_t* z_ready = bars + 27;      // MZ: a step's Z written into buffer b = step & 1 (every noise warp)
    uint64_t* z_free = bars + 29;       // MZ: buffer b read by the step's epilogue (every worker warp)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cpq = a.cpt >> 2;         // chains per TMEM lane quarter (rows 32 q + 3 k + axis)
    const int c0 = tile * a.cpt;
    const int Ct = min(a.cpt, a.C - c0);
    const uint32_t rblock = 4u * 3u * (uint32_t)cpq * 128u;   // bytes of one R column block

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&ready[s], kReadyCount);
            mbar_init(&empty[s], 1);
        }
        mbar_init(u_done, 1);
        mbar_init(inc_done, 1);
        for (int k = 0; k < KB; ++k) mbar_init(&r_blk[k], 1);
        mbar_init(epi_done, kComputeWarps + kNoiseWarps);
        mbar_init(never, 1);
        if constexpr (MZ) {
            for (int b2 = 0; b2 < 2; ++b2) {
                mbar_init(&z_ready[b2], kNoiseWarps);
                mbar_init(&z_free[b2], kComputeWarps + kNoiseWarps);
            }
        }
        *abort_flag = 0;
        *s_freed = -1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmR)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmChiH)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmChiL)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmFH)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmFL)) : "memory");
    }
    for (int p = threadIdx.x; p < NB; p += kThreads) {
        s_dm[p] = a.dm[p];
        s_g[p] = a.g[p];
        if constexpr (MZ) s_w[p] = a.w[p];
    }
    for (int i = threadIdx.x; i < kChains; i += kThreads) {
        const bool live = i < Ct;
        s_job[i] = live ? a.job[c0 + i] : 0u;
        s_step[i] = live ? a.step[c0 + i] : 0;
        s_stop[i] = (live && a.stop) ? a.stop[c0 + i] : INT64_MAX;
        s_shear[i] = live ? a.shear[c0 + i] : 0.0;
        s_rowb[i] = i < a.cpt ? 32 * (i / cpq) + 3 * (i % cpq) : 0;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t t_u = tmem, t_inc = tmem + NB;
    const bool has_shear = __syncthreads_or(threadIdx.x < Ct && s_shear[threadIdx.x] != 0.0) != 0;

    // Epilogue of step sp (R += -dm R + D_inc (+ shear), Eqs. d3, btum) on the R
    // tile that the producer reloads into the stage memory (KB column blocks of
    // [128 rows][32], swizzled, each with its own barrier), in place.  The
    // compute and noise warps of lane quarter q share it: worker w of nw takes
    // the quarter's rows of column blocks w, w + nw, ... and TMA-stores each
    // (block, quarter) box as soon as it is done.  Worker 0 (a compute warp)
    // holds the centre of mass, which column block 0 updates.
    auto epilogue = [&](int sp, int q, int w, int nw, bool& ok, bool& finite, double& cm_x, double& cm_y,
                        double& cm_z) {
        const int row = 32 * q + lane;
        const int kq = lane / 3, ax = lane - 3 * (lane / 3);
        const bool inrow = kq < cpq;
        const int cl = inrow ? cpq * q + kq : 0;
        const bool live = inrow && cl < Ct;
        ok = ok && mbar_wait(inc_done, sp & 1, a.err, abort_flag);
        // MZ: the step's mode noise Z (written one step ahead by the noise warps)
        const float* zrow = nullptr;
        if constexpr (MZ) {
            ok = ok && mbar_wait(&z_ready[sp & 1], (sp >> 1) & 1, a.err, abort_flag);
            zrow = a.zbuf + ((size_t)(sp & 1) * a.C * 3 + (size_t)3 * (c0 + cl) + ax) * NB;
        }
        fence_after();
        // a chain whose step counter has reached its stop step stays as it is
        const bool adv = live && s_step[cl] + sp < s_stop[cl];
#pragma unroll 1
        for (int kb = w; kb < KB; kb += nw) {
            ok = ok && mbar_wait(&r_blk[kb], sp & 1, a.err, abort_flag);
            uint8_t* blk = stage0 + kb * S::kRT;
#pragma unroll 1
            for (int kin = 0; kin < kKB; kin += 16) {
                const int p0 = kb * kKB + kin;
                float d[16], r[16];
                if constexpr (MZ) {
                    // D_inc = h_p DeltaH_p; the noise term w_p Z_p (Eq. d6) is added here in FP32
                    float z[16];
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        const float4 x = live ? *reinterpret_cast<const float4*>(zrow + p0 + 4 * k4)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                        z[4 * k4] = x.x; z[4 * k4 + 1] = x.y; z[4 * k4 + 2] = x.z; z[4 * k4 + 3] = x.w;
                    }
                    tmem_ld16(t_inc + ((uint32_t)(32 * q) << 16) + (uint32_t)p0, d);
#pragma unroll
                    for (int i = 0; i < 16; ++i) d[i] = fmaf(s_w[p0 + i], z[i], d[i]);
                } else {
                    tmem_ld16(t_inc + ((uint32_t)(32 * q) << 16) + (uint32_t)p0, d);
                }
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    const float4 x = *reinterpret_cast<const float4*>(blk + swz(row, kin + 4 * k4));
                    r[4 * k4] = x.x; r[4 * k4 + 1] = x.y; r[4 * k4 + 2] = x.z; r[4 * k4 + 3] = x.w;
                }
                float o[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) o[i] = adv ? r[i] + fmaf(-s_dm[p0 + i], r[i], d[i]) : r[i];
                if (has_shear) {
                    // start-of-step R^y of this chain: the next lane's row (axis 1)
                    const float sh = (float)s_shear[cl];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float ry = __shfl_down_sync(0xffffffffu, r[i], 1);
                        if (adv && ax == 0) o[i] += sh * s_g[p0 + i] * ry;
                    }
                }
                if (p0 == 0) {
                    // centre of mass in FP64 (p = 0 of Eq. d3 with zeta_0 = 0), kept in
                    // registers for the whole launch
                    const float d1 = __shfl_down_sync(0xffffffffu, d[0], 1);
                    const float d2 = __shfl_down_sync(0xffffffffu, d[0], 2);
                    if (adv && ax == 0) {
                        const double ycm = cm_y;
                        cm_x += (double)d[0] * a.inv_sqrtM + s_shear[cl] * a.dtau * ycm;
                        cm_y += (double)d1 * a.inv_sqrtM;
                        cm_z += (double)d2 * a.inv_sqrtM;
                    }
                    o[0] = 0.f;
                }
                if (live) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) finite = finite && isfinite(o[i]);
                }
                if (inrow) {
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4)
                        *reinterpret_cast<float4*>(blk + swz(row, kin + 4 * k4)) =
                            make_float4(o[4 * k4], o[4 * k4 + 1], o[4 * k4 + 2], o[4 * k4 + 3]);
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0 && ok) {
                tma_store_2d(&tmR, blk + q * kQuarter, kb * kKB, 3 * (c0 + q * cpq));
                tma_store_commit();
            }
        }
        // R is in global memory and this warp's stage rows are free again; D_inc
        // has been read before the next step's MMAs write it
        if (lane == 0 && ok) tma_store_wait();
        fence_before();
        __syncwarp();
        if (lane == 0 && ok) mbar_arrive(epi_done);
        if constexpr (MZ) {
            if (lane == 0 && ok) mbar_arrive(&z_free[sp & 1]);   // this warp is done with Z of step sp
        }
    };

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
                st_release_smem(s_freed, gb);   // block gb may be written into stage s
                uint8_t* st = stage0 + s * S::kStage;
                uint8_t* bh = st + S::kR + 2 * S::kA;
                uint8_t* bl = bh + S::kB;
                int kind, nb;
                sched_decode_any<KB, BF ? 0 : 1, MZ>(blk, kind, nb);
                if (kind == 0) {
                    // inverse: the R tile (FP32, one box per lane quarter) and chi
                    mbar_expect_tx(&full[s], rblock + 2 * S::kB);
                    tma_load_2d(bh, &tmChiH, &full[s], nb * kKB, 0);
                    tma_load_2d(bl, &tmChiL, &full[s], nb * kKB, 0);
                    for (int q = 0; q < 4; ++q)
                        tma_load_2d(st + q * kQuarter, &tmR, &full[s], nb * kKB, 3 * (c0 + q * cpq));
                } else {
                    // noise block nb: rows w_p phi (t = 1); force block nb: rows h_p chi (t = 0)
                    const bool noise = kind == 1;
                    mbar_expect_tx(&full[s], 2 * S::kB);
                    tma_load_2d(bh, &tmFH, &full[s], nb * kKB, noise ? NB : 0);
                    tma_load_2d(bl, &tmFL, &full[s], nb * kKB, noise ? NB : 0);
                }
            }
            // reload the R tile (KB column blocks of [128 rows][32]) into the stage
            // memory for the epilogue: column block k as soon as every stage its
            // bytes overlap has seen the last MMA of this step (the last ST blocks
            // release the stages in turn), not only after the last MMA of all
            unsigned freed = 0;
            int k = 0;
            for (int j = NBLK - ST; j < NBLK && ok; ++j) {
                const int gl = sp * NBLK + j, sl = gl % ST;
                if (!mbar_wait(&empty[sl], (gl / ST) & 1, a.err, abort_flag)) { ok = false; break; }
                freed |= 1u << sl;
                for (; k < KB; ++k) {
                    const int s_lo = k * S::kRT / S::kStage, s_hi = ((k + 1) * S::kRT - 1) / S::kStage;
                    bool all = true;
                    for (int t = s_lo; t <= s_hi; ++t) all = all && ((freed >> t) & 1u);
                    if (!all) break;
                    mbar_expect_tx(&r_blk[k], rblock);
                    for (int q = 0; q < 4; ++q)
                        tma_load_2d(stage0 + k * S::kRT + q * kQuarter, &tmR, &r_blk[k], k * kKB, 3 * (c0 + q * cpq));
                }
            }
          }
          // the MMAs' commits of the last block of each stage have arrived, so
          // nothing lands on these barriers after the tile (see above)
          const int G = a.n_steps * NBLK;
          for (int s = 0; s < ST && s < G && ok; ++s) {
              const int gl = s + ST * ((G - 1 - s) / ST);
              ok = mbar_wait(&empty[s], (gl / ST) & 1, a.err, abort_flag);
          }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = BF ? idesc_bf16(kRows, NB) : idesc_tf32(kRows, NB);
            bool ok = true;
            // stall test: this wait runs out after its limit, raises the timeout bit
            // and the abort flag, and every other wait of the CTA then gives up
            if (a.stall_test) ok = mbar_wait(never, 0, a.err, abort_flag);
            for (int sp = 0; sp < a.n_steps; ++sp) {
            for (int blk = 0; blk < NBLK; ++blk) {
                const int gb = sp * NBLK + blk;
                const int s = gb % ST;
                const uint32_t ph = (gb / ST) & 1;
                int kind, nb;
                sched_decode_any<KB, BF ? 0 : 1, MZ>(blk, kind, nb);
                ok = ok && mbar_wait(&full[s], ph, a.err, abort_flag);
                ok = ok && mbar_wait(&ready[s], ph, a.err, abort_flag);
                if (ok) {
                    fence_after();
                    const uint32_t st = smem_u32(stage0 + s * S::kStage);
                    const uint32_t a_hi = st + S::kR, a_lo = a_hi + S::kA, b_hi = a_lo + S::kA, b_lo = b_hi + S::kB;
                    const uint32_t d = kind == 0 ? t_u : t_inc;
                    // first inverse block, first forward (noise, or force with MZ) block
                    const bool first = MZ ? (blk == 0 || blk == KB) : blk <= 1;
                    if constexpr (BF) {
#pragma unroll
                        for (int kk = 0; kk < kKB / 16; ++kk) {
                            const uint32_t off = kk * 32;   // 16 BF16 = 32 bytes along K
                            if constexpr (TWO) {
                                mma_bf16(d, sdesc64(a_lo + off), sdesc64(b_hi + off), idesc, (first && kk == 0) ? 0u : 1u);
                            } else {
                                mma_bf16(d, sdesc64(a_hi + off), sdesc64(b_lo + off), idesc, (first && kk == 0) ? 0u : 1u);
                                mma_bf16(d, sdesc64(a_lo + off), sdesc64(b_hi + off), idesc, 1u);
                            }
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
                if (ok) {
                    mma_commit(&empty[s]);
                    if (blk == (MZ ? KB - 1 : sched_inv<KB>(KB - 1))) mma_commit(u_done);
                }
            }
            if (ok) mma_commit(inc_done);
            }
        }
    } else if (MZ && warp >= 2 + kComputeWarps) {
        // ---------------- noise warps, mode-keyed noise: the normals Z of step
        // sp + 1 (Philox tag 2, normal 3 p + alpha of call (3 p + alpha) / 4,
        // 32-mode blocks of 24 calls per chain) drawn during step sp into buffer
        // (sp + 1) & 1 of a.zbuf ([2][3 C][M], FP32), then this warp's share of
        // step sp's epilogue.  A buffer is written again only after the epilogue
        // two steps back has read it (z_free).
        const int nw = warp - 2 - kComputeWarps;
        bool ok = true, finite = true;
        double cm_unused[3];
        const int eq = warp & 3, et = (warp - 2 - kComputeWarps) / 4;   // epilogue quarter, worker 2 + et
        const int nch = a.cpt * kCallsPerBlock / 32;
        const int h0 = noise_h0(nw, 0);
        auto draw_step = [&](int sp) {
            const int b2 = sp & 1;
            if (sp >= 2) ok = ok && mbar_wait(&z_free[b2], ((sp >> 1) - 1) & 1, a.err, abort_flag);
            float* zb = a.zbuf + (size_t)b2 * a.C * 3 * NB;
#pragma unroll 1
            for (int j = 0; j < KB; ++j) {
                float zz[kChunksPerWarp][4];
                noise_draw(zz, nw, 0, j, sp, lane, a.cpt, Ct, a.seed, s_job, s_step, 2u);
#pragma unroll
                for (int i = 0; i < kChunksPerWarp; ++i) {
                    const int h = h0 + kNoiseWarps * i;
                    if (h >= nch || !ok) continue;
                    const int f = 32 * h + lane;
                    const int cl = f / kCallsPerBlock, call = kCallsPerBlock * j + (f - kCallsPerBlock * cl);
                    if (cl >= Ct) continue;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int k = 4 * call + e, pm = k / 3;
                        zb[(size_t)(3 * (c0 + cl) + (k - 3 * pm)) * NB + pm] = zz[i][e];
                    }
                }
            }
            __syncwarp();
            if (lane == 0 && ok) mbar_arrive(&z_ready[b2]);
        };
        draw_step(0);
#pragma unroll 1
        for (int sp = 0; sp < a.n_steps; ++sp) {
            if (sp + 1 < a.n_steps) draw_step(sp + 1);
            epilogue(sp, eq, 2 + et, 2 + kNoiseInQ[(eq + 2) & 3], ok, finite, cm_unused[0], cm_unused[1], cm_unused[2]);
        }
        if (!finite) atomicOr(a.err, 1);
    } else if (warp >= 2 + kComputeWarps) {
        // ---------------- noise warps: Philox normals of noise block j (Eq. b5),
        // drawn into registers (noise_draw), then written as hi / lo operands once
        // the stage is free (noise_put).
        const int nw = warp - 2 - kComputeWarps;
        auto draw = [&](int qn, float (&zz)[kChunksPerWarp][4]) {
            const int sp = qn / KB;
            noise_draw(zz, nw, qn, qn - sp * KB, sp, lane, a.cpt, Ct, a.seed, s_job, s_step);
        };
        // Noise blocks in sequence qn = KB step + j.  Block qn is drawn into `cur`
        // right after block qn - 1 is written, then written as soon as its stage
        // is free.  Nothing more is drawn ahead: a warp that draws block qn + 1
        // while it waits for the stage of block qn writes block qn late whenever
        // the stage frees during that draw, and the MMAs wait for it (measured
        // 4% slower per step).
        bool ok = true, finite = true;
        double cm_unused[3];
        const int eq = warp & 3, et = (warp - 2 - kComputeWarps) / 4;   // epilogue quarter, worker 2 + et
        const int nq = a.n_steps * KB;
        float cur[kChunksPerWarp][4];
        draw(0, cur);
#pragma unroll 1
        for (int qn = 0; qn < nq; ++qn) {
            const int sp = qn / KB, j = qn - sp * KB;
            const int blk = sp * NBLK + sched_noise<KB, BF ? 0 : 1>(j), s = blk % ST;
            // Consecutive noise blocks may lie more than ST blocks apart, where a
            // parity wait on the stage's barrier is ambiguous: wait instead until
            // the producer has seen the stage released for this block (which it
            // does in block order, after the previous step's epilogue).
            ok = ok && count_wait(s_freed, blk, a.err, abort_flag);
            if (ok) {
                uint8_t* ah = stage0 + s * S::kStage + S::kR;
                uint8_t* al = ah + S::kA;
                noise_put<BF>(ah, al, cur, nw, qn, lane, a.cpt, s_rowb);
                fence_proxy_async();
            }
            __syncwarp();
            if (lane == 0 && ok) mbar_arrive_cnt(&ready[s], kReadyCount / kNoiseWarps);
            // after its last noise block, the step's epilogue (this warp's share)
            if (j == KB - 1)
                epilogue(sp, eq, 2 + et, 2 + kNoiseInQ[(eq + 2) & 3], ok, finite, cm_unused[0], cm_unused[1],
                         cm_unused[2]);
            if (qn + 1 < nq) draw(qn + 1, cur);
        }
        if (!finite) atomicOr(a.err, 1);
    } else {
        // ---------------- compute warps 2..9: two per TMEM lane quarter q; lane
        // 3 k + axis of quarter q is axis `axis` of the quarter's chain k.
        const int cw = warp - 2;            // 0..7
        const int ct = threadIdx.x - 64;    // 0..255
        const int q = warp & 3;             // TMEM lane quarter this warp may access
        const int half = cw >> 2;           // which 16 of a block's 32 columns
        const int row = 32 * q + lane;
        const int kq = lane / 3, ax = lane - 3 * (lane / 3);
        const bool inrow = kq < cpq;        // the row belongs to a chain slot of the tile
        const int cl = inrow ? cpq * q + kq : 0;   // chain of the tile
        const bool live = inrow && cl < Ct;
        const int src0 = lane - ax;         // lane of axis 0 of this chain
        // the chain's FP64 centre of mass, on its axis-0 lane of a first-half warp
        const bool own_cm = half == 0 && live && ax == 0;
        double cm_x = 0.0, cm_y = 0.0, cm_z = 0.0;
        if (own_cm) {
            const double* cm = a.com + 3 * (size_t)(c0 + cl);
            cm_x = cm[0];
            cm_y = cm[1];
            cm_z = cm[2];
        }
        bool ok = true;
        bool finite = true;
        auto arrive = [&](int s) {
            __syncwarp();
            if (lane == 0 && ok) mbar_arrive_cnt(&ready[s], kReadyCount / kComputeWarps);
        };
#pragma unroll 1
        for (int sp = 0; sp < a.n_steps; ++sp) {
        const int g0 = sp * NBLK;                     // global index of this step's first block
        // (1) split the R tile of each inverse block into hi / lo operands
#pragma unroll 1
        for (int nb = 0; nb < KB; ++nb) {
            const int blk = g0 + (MZ ? nb : sched_inv<KB>(nb)), s = blk % ST;
            const uint32_t ph = (blk / ST) & 1;
            // The stage's previous use may be a noise block these warps never
            // waited for, so a parity wait alone could be two phases ahead; the
            // producer's release counter first (that use is consumed) makes it exact.
            ok = ok && count_wait(s_freed, blk, a.err, abort_flag);
            ok = ok && mbar_wait(&full[s], ph, a.err, abort_flag);
            if (BF && !S::kR) {
                // in place: every compute thread reads its values, the compute warps
                // meet (all of them, whether or not a wait gave up), then the hi / lo
                // parts go over the FP32 tile
                uint8_t* base = stage0 + s * S::kStage;
                float xv[kRows * 4 / kCompute][8];
#pragma unroll
                for (int e = 0; e < kRows * 4 / kCompute; ++e) {
                    const int t = ct + kCompute * e;
                    const int r = t >> 2, c = t & 3;
                    if (ok && (r & 31) < 3 * cpq) {
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {
                            const float4 x = *reinterpret_cast<const float4*>(base + swz(r, 8 * c + 4 * h2));
                            xv[e][4 * h2] = x.x; xv[e][4 * h2 + 1] = x.y; xv[e][4 * h2 + 2] = x.z; xv[e][4 * h2 + 3] = x.w;
                        }
                    }
                }
                __syncwarp();
                asm volatile("bar.sync 1, %0;" ::"n"(kCompute) : "memory");
#pragma unroll
                for (int e = 0; e < kRows * 4 / kCompute; ++e) {
                    const int t = ct + kCompute * e;
                    const int r = t >> 2, c = t & 3;
                    if (ok && (r & 31) < 3 * cpq) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const uint16_t h0 = bf16_rn(xv[e][2 * i]), h1 = bf16_rn(xv[e][2 * i + 1]);
                            hw[i] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                            lw[i] = (uint32_t)bf16_rn(xv[e][2 * i] - bf16_f(h0)) |
                                    ((uint32_t)bf16_rn(xv[e][2 * i + 1] - bf16_f(h1)) << 16);
                        }
                        const uint32_t o = swz_bf(r, 8 * c);
                        *reinterpret_cast<uint4*>(base + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(base + S::kA + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
                if (ok) fence_proxy_async();
            } else if (ok && BF) {
                // row t/4, BF16 chunk t%4 (8 values) from the FP32 staging tile
                const uint8_t* r32 = stage0 + s * S::kStage;
                uint8_t* ah = stage0 + s * S::kStage + S::kR;
                uint8_t* al = ah + S::kA;
#pragma unroll
                for (int e = 0; e < kRows * 4 / kCompute; ++e) {
                    const int t = ct + kCompute * e;
                    const int r = t >> 2, c = t & 3;
                    if ((r & 31) >= 3 * cpq) continue;   // padding rows of a lane quarter
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
                }
                fence_proxy_async();
            } else if (ok) {
                float4* ah = (float4*)(stage0 + s * S::kStage);
                float4* al = (float4*)(stage0 + s * S::kStage + S::kA);
#pragma unroll
                for (int i = 0; i < S::kA / 16 / kCompute; ++i) {
                    const int e = ct + kCompute * i;
                    if (((e >> 3) & 31) >= 3 * cpq) continue;   // padding rows of a lane quarter
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
            arrive(s);
        }

        // (2) per bead block nb: bond vectors from D_u -> residual force v (Eq. e11),
        //     |u_n| from the chain's three rows by warp shuffles
        ok = ok && mbar_wait(u_done, sp & 1, a.err, abort_flag);
        fence_after();
#pragma unroll 1
        for (int nb = 0; nb < KB; ++nb) {
            const int col = nb * kKB + 16 * half;       // first bead of this warp's 16
            float v[16];
            tmem_ld16(t_u + ((uint32_t)(32 * q) << 16) + (uint32_t)col, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float sq = v[i] * v[i];
                const float t = sq + __shfl_down_sync(0xffffffffu, sq, 1) + __shfl_down_sync(0xffffffffu, sq, 2);
                const float fac = __shfl_sync(0xffffffffu, rsqrtf(t) - a.c12nu, src0);
                v[i] = (live && col + i >= 1) ? v[i] * fac : 0.f;
            }
            const int blk = g0 + (MZ ? KB + nb : sched_force<KB, BF ? 0 : 1>(nb)), s = blk % ST;
            const uint32_t ph = (blk / ST) & 1;
            ok = ok && mbar_wait(&empty[s], ph ^ 1, a.err, abort_flag);
            if (ok && inrow) {
                uint8_t* ah = stage0 + s * S::kStage + S::kR;
                uint8_t* al = ah + S::kA;
                if constexpr (BF) {
#pragma unroll
                    for (int h8 = 0; h8 < 2; ++h8) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float x0 = v[8 * h8 + 2 * i], x1 = v[8 * h8 + 2 * i + 1];
                            const uint16_t h0 = bf16_rn(x0), h1 = bf16_rn(x1);
                            hw[i] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                            lw[i] = (uint32_t)bf16_rn(x0 - bf16_f(h0)) | ((uint32_t)bf16_rn(x1 - bf16_f(h1)) << 16);
                        }
                        const uint32_t o = swz_bf(row, 16 * half + 8 * h8);
                        *reinterpret_cast<uint4*>(ah + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(al + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                } else {
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        float4 h, l;
                        h.x = tf32_rna(v[4 * k4]);     l.x = tf32_rna(v[4 * k4] - h.x);
                        h.y = tf32_rna(v[4 * k4 + 1]); l.y = tf32_rna(v[4 * k4 + 1] - h.y);
                        h.z = tf32_rna(v[4 * k4 + 2]); l.z = tf32_rna(v[4 * k4 + 2] - h.z);
                        h.w = tf32_rna(v[4 * k4 + 3]); l.w = tf32_rna(v[4 * k4 + 3] - h.w);
                        const uint32_t o = swz(row, 16 * half + 4 * k4);
                        *reinterpret_cast<float4*>(ah + o) = h;
                        *reinterpret_cast<float4*>(al + o) = l;
                    }
                }
            }
            if (ok) fence_proxy_async();
            arrive(s);
        }

        // (3) epilogue, shared with the noise warps of this lane quarter
        epilogue(sp, q, half, 2 + kNoiseInQ[(q + 2) & 3], ok, finite, cm_x, cm_y, cm_z);
        }   // steps
        if (ok && own_cm) {
            double* cm = a.com + 3 * (size_t)(c0 + cl);
            cm[0] = cm_x;
            cm[1] = cm_y;
            cm[2] = cm_z;
        }
        if (ok && half == 0 && live && ax == 0)
            a.step[c0 + cl] = max(s_step[cl], min(s_step[cl] + (int64_t)a.n_steps, s_stop[cl]));
        if (!finite) atomicOr(a.err, 1);
    }
    fence_before();
    __syncthreads();
    return *abort_flag == 0;
}

// TMEM columns for the 2 NB of a tile (warp 1 allocates into *slot).
template <uint32_t kCols>
__device__ __forceinline__ void tmem_alloc(uint32_t* slot)
{
    if ((threadIdx.x >> 5) == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(slot)), "r"(kCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
}
template <uint32_t kCols>
__device__ __forceinline__ void tmem_free(uint32_t tmem)
{
    if ((threadIdx.x >> 5) == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

// One tile per CTA (a launch of one length group).
template <int NB, bool BF, bool TWO = false, bool MZ = false>
__global__ void __launch_bounds__(kThreads, 1)
k_fused_step(const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmChiH,
             const __grid_constant__ CUtensorMap tmChiL, const __grid_constant__ CUtensorMap tmFH,
             const __grid_constant__ CUtensorMap tmFL, const FusedArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t s_tmem;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    tmem_alloc<2 * NB>(&s_tmem);
    const uint32_t tmem = s_tmem;
    fused_tile<NB, BF, TWO, MZ>(tmR, tmChiH, tmChiL, tmFH, tmFL, a, blockIdx.x, smem, tmem);
    tmem_free<2 * NB>(tmem);
}


// The 512-bead step: tile `tile` on a cluster of two CTAs, CTA h (its rank)
// holding bonds and modes 256 h .. 256 h + 255 (see the file's header).  The
// caller launches clusters of two and allocates the 512 TMEM columns at `tmem`;
// the tile starts and ends with a cluster barrier.  Returns false if a wait
// gave up.
template <bool BF, bool TWO>
__device__ __forceinline__ bool pair_tile(const CUtensorMap& tmR, const CUtensorMap& tmChiH,
                                          const CUtensorMap& tmChiL, const CUtensorMap& tmFH,
                                          const CUtensorMap& tmFL, const FusedArgs& a, int tile, uint8_t* smem,
                                          uint32_t tmem)
{
    constexpr int NB = 256;             // TMEM columns of each half (D_u, D_inc) of this CTA
    using S = FSmem<NB, BF, false>;
    constexpr int ST = S::kStages;
    constexpr int KBL = NB / kKB;       // column blocks of this CTA (epilogue; owned blocks of each kind)
    constexpr int KB = 2 * KBL;         // inverse K blocks = forward bead blocks = M / 32
    constexpr int MB = KB * kKB;        // beads M
    constexpr int NBLK = 3 * KB;        // blocks of one step, in the order of sched_decode
    constexpr int FILL = BF ? 4 : 1;   // noise blocks in phase 1's tail (measured: BF16 4, TF32 1)
    static_assert(KB % 2 == 0, "the block schedule pairs bead blocks");

    uint8_t* stage0 = smem;
    uint8_t* misc = smem + ST * S::kStage;
    uint32_t* s_job = (uint32_t*)misc;
    int64_t* s_step = (int64_t*)(misc + 256);
    double* s_shear = (double*)(misc + 576);
    int64_t* s_stop = (int64_t*)(misc + 896);
    float* s_dm = (float*)(misc + 1216);        // NB <= 256
    float* s_g = (float*)(misc + 2240);
    uint64_t* bars = (uint64_t*)(misc + 3264);
    int* s_rowb = (int*)(misc + 3584);          // first A-operand row of each chain slot
    uint64_t* full = bars;              // TMA bytes landed                 (1 + tx)
    uint64_t* ready = bars + 4;         // A operand written by one group   (kReadyCount)
    uint64_t* empty = bars + 8;         // MMAs done with the stage         (commit)
    uint64_t* u_done = bars + 12;       // all inverse MMAs done            (commit)
    uint64_t* inc_done = bars + 13;     // all forward MMAs done            (commit)
    uint64_t* epi_done = bars + 15;     // epilogue stored R, stages free   (every worker warp)
    uint32_t* flags = (uint32_t*)(bars + 16);
    volatile int* abort_flag = (volatile int*)(flags + 1);
    int* s_freed = (int*)(flags + 2);   // last block whose stage the producer saw released
    uint64_t* r_blk = bars + 18;        // R column block k reloaded for the epilogue (1 + tx), k < KBL
    uint64_t* never = bars + 26;        // nothing arrives here (the stall test)
    uint64_t* both_done = bars + 27;    // the MMAs of both CTAs done with the step (2 commits)
    uint64_t* peer_epi = bars + 28;     // the other CTA's epilogue done (its producer arrives)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cpq = a.cpt >> 2;         // chains per TMEM lane quarter (rows 32 q + 3 k + axis)
    const uint32_t rank = cluster_rank();   // this CTA's bead / mode half
    const int col0 = (int)rank * NB;    // first bond and mode of this CTA's TMEM columns
    const int c0 = tile * a.cpt;
    const int Ct = min(a.cpt, a.C - c0);
    const uint32_t rblock = 4u * 3u * (uint32_t)cpq * 128u;   // bytes of one R column block

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&ready[s], kReadyCount);
            mbar_init(&empty[s], 2);      // both CTAs' MMAs
        }
        mbar_init(u_done, 1);
        mbar_init(inc_done, 1);
        for (int k = 0; k < KBL; ++k) mbar_init(&r_blk[k], 1);
        mbar_init(epi_done, kComputeWarps + kNoiseWarps);
        mbar_init(never, 1);
        mbar_init(both_done, 2);
        mbar_init(peer_epi, 1);
        *abort_flag = 0;
        *s_freed = -1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmR)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmChiH)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmChiL)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmFH)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmFL)) : "memory");
    }
    for (int p = threadIdx.x; p < NB; p += blockDim.x) {
        s_dm[p] = a.dm[col0 + p];
        s_g[p] = a.g[col0 + p];
    }
    for (int i = threadIdx.x; i < kChains; i += blockDim.x) {
        const bool live = i < Ct;
        s_job[i] = live ? a.job[c0 + i] : 0u;
        s_step[i] = live ? a.step[c0 + i] : 0;
        s_stop[i] = (live && a.stop) ? a.stop[c0 + i] : INT64_MAX;
        s_shear[i] = live ? a.shear[c0 + i] : 0.0;
        s_rowb[i] = i < a.cpt ? 32 * (i / cpq) + 3 * (i % cpq) : 0;
    }
    fence_before();
    cluster_sync();                     // both CTAs' barriers are initialised
    fence_after();
    const uint32_t t_u = tmem, t_inc = tmem + NB;
    const bool has_shear = __syncthreads_or(threadIdx.x < Ct && s_shear[threadIdx.x] != 0.0) != 0;

    // Epilogue of step sp (R += -dm R + D_inc (+ shear), Eqs. d3, btum) on the R
    // tile that the producer reloads into the stage memory (KBL column blocks of
    // [128 rows][32], swizzled, each with its own barrier; modes col0 + ...), in place.  The
    // compute and noise warps of lane quarter q share it: worker w of nw takes
    // the quarter's rows of column blocks w, w + nw, ... and TMA-stores each
    // (block, quarter) box as soon as it is done.  Worker 0 (a compute warp)
    // holds the centre of mass, which column block 0 updates.
    auto epilogue = [&](int sp, int q, int w, int nw, bool& ok, bool& finite, double& cm_x, double& cm_y,
                        double& cm_z) {
        const int row = 32 * q + lane;
        const int kq = lane / 3, ax = lane - 3 * (lane / 3);
        const bool inrow = kq < cpq;
        const int cl = inrow ? cpq * q + kq : 0;
        const bool live = inrow && cl < Ct;
        ok = ok && mbar_wait(inc_done, sp & 1, a.err, abort_flag);
        fence_after();
        // a chain whose step counter has reached its stop step stays as it is
        const bool adv = live && s_step[cl] + sp < s_stop[cl];
#pragma unroll 1
        for (int kb = w; kb < KBL; kb += nw) {
            ok = ok && mbar_wait(&r_blk[kb], sp & 1, a.err, abort_flag);
            uint8_t* blk = stage0 + kb * S::kRT;
#pragma unroll 1
            for (int kin = 0; kin < kKB; kin += 16) {
                const int p0 = kb * kKB + kin;
                float d[16], r[16];
                tmem_ld16(t_inc + ((uint32_t)(32 * q) << 16) + (uint32_t)p0, d);
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {
                    const float4 x = *reinterpret_cast<const float4*>(blk + swz(row, kin + 4 * k4));
                    r[4 * k4] = x.x; r[4 * k4 + 1] = x.y; r[4 * k4 + 2] = x.z; r[4 * k4 + 3] = x.w;
                }
                float o[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) o[i] = adv ? r[i] + fmaf(-s_dm[p0 + i], r[i], d[i]) : r[i];
                if (has_shear) {
                    // start-of-step R^y of this chain: the next lane's row (axis 1)
                    const float sh = (float)s_shear[cl];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float ry = __shfl_down_sync(0xffffffffu, r[i], 1);
                        if (adv && ax == 0) o[i] += sh * s_g[p0 + i] * ry;
                    }
                }
                if (col0 + p0 == 0) {
                    // centre of mass in FP64 (p = 0 of Eq. d3 with zeta_0 = 0), kept in
                    // registers for the whole launch
                    const float d1 = __shfl_down_sync(0xffffffffu, d[0], 1);
                    const float d2 = __shfl_down_sync(0xffffffffu, d[0], 2);
                    if (adv && ax == 0) {
                        const double ycm = cm_y;
                        cm_x += (double)d[0] * a.inv_sqrtM + s_shear[cl] * a.dtau * ycm;
                        cm_y += (double)d1 * a.inv_sqrtM;
                        cm_z += (double)d2 * a.inv_sqrtM;
                    }
                    o[0] = 0.f;
                }
                if (live) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) finite = finite && isfinite(o[i]);
                }
                if (inrow) {
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4)
                        *reinterpret_cast<float4*>(blk + swz(row, kin + 4 * k4)) =
                            make_float4(o[4 * k4], o[4 * k4 + 1], o[4 * k4 + 2], o[4 * k4 + 3]);
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0 && ok) {
                tma_store_2d(&tmR, blk + q * kQuarter, col0 + kb * kKB, 3 * (c0 + q * cpq));
                tma_store_commit();
            }
        }
        // R is in global memory and this warp's stage rows are free again; D_inc
        // has been read before the next step's MMAs write it
        if (lane == 0 && ok) tma_store_wait();
        fence_before();
        __syncwarp();
        if (lane == 0 && ok) mbar_arrive(epi_done);
    };

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
          bool ok = true;
          for (int sp = 0; sp < a.n_steps && ok; ++sp) {
            if (sp > 0) {
                // the previous step's epilogue used the stage memory and stored R
                if (!mbar_wait(epi_done, (sp - 1) & 1, a.err, abort_flag)) break;
                // ... and so did the other CTA's, into whose stages this CTA copies
                mbar_arrive_remote(mapa(smem_u32(peer_epi), rank ^ 1u));
                if (!mbar_wait_cl(peer_epi, (sp - 1) & 1, a.err, abort_flag)) break;
            }
            for (int blk = 0; blk < NBLK; ++blk) {
                const int gb = sp * NBLK + blk;
                const int s = gb % ST;
                const uint32_t ph = (gb / ST) & 1;
                if (!mbar_wait_cl(&empty[s], ph ^ 1, a.err, abort_flag)) { ok = false; break; }
                st_release_smem(s_freed, gb);   // block gb may be written into stage s
                uint8_t* st = stage0 + s * S::kStage;
                uint8_t* bh = st + S::kR + 2 * S::kA;
                uint8_t* bl = bh + S::kB;
                int kind, nb;
                sched_decode<KB, FILL>(blk, kind, nb);
                // a block of the other CTA arrives with its A operand copied in
                const bool own = (uint32_t)(nb & 1) == rank;
                const uint32_t a_in = own ? 0u : 2u * S::kA;
                if (kind == 0) {
                    // inverse: the R tile (FP32, one box per lane quarter) and chi rows of the bond half
                    mbar_expect_tx(&full[s], (own ? rblock : 0u) + 2 * S::kB + a_in);
                    tma_load_2d(bh, &tmChiH, &full[s], nb * kKB, col0);
                    tma_load_2d(bl, &tmChiL, &full[s], nb * kKB, col0);
                    if (own)
                        for (int q = 0; q < 4; ++q)
                            tma_load_2d(st + q * kQuarter, &tmR, &full[s], nb * kKB, 3 * (c0 + q * cpq));
                } else {
                    // noise block nb: rows w_p phi (t = 1); force block nb: rows h_p chi (t = 0)
                    const bool noise = kind == 1;
                    const int x = (noise ? nb : force_bonds<KBL>(nb)) * kKB;
                    mbar_expect_tx(&full[s], 2 * S::kB + a_in);
                    tma_load_2d(bh, &tmFH, &full[s], x, (noise ? MB : 0) + col0);
                    tma_load_2d(bl, &tmFL, &full[s], x, (noise ? MB : 0) + col0);
                }
                if (!own) mbar_arrive_cnt(&ready[s], kReadyCount);   // no local writer
            }
            // every stage is free once the forward MMAs (of both CTAs) are done:
            // reload the R tile (KBL column blocks of [128 rows][32]) there for the epilogue
            if (ok && mbar_wait(inc_done, sp & 1, a.err, abort_flag) &&
                mbar_wait_cl(both_done, sp & 1, a.err, abort_flag)) {
                for (int k = 0; k < KBL; ++k) {
                    mbar_expect_tx(&r_blk[k], rblock);
                    for (int q = 0; q < 4; ++q)
                        tma_load_2d(stage0 + k * S::kRT + q * kQuarter, &tmR, &r_blk[k], col0 + k * kKB,
                                    3 * (c0 + q * cpq));
                }
            } else {
                ok = false;
            }
          }
          // the other CTA's commits of the last block in each stage have arrived
          const int G = a.n_steps * NBLK;
          for (int s = 0; s < ST && s < G && ok; ++s) {
              const int gl = s + ST * ((G - 1 - s) / ST);
              ok = mbar_wait_cl(&empty[s], (gl / ST) & 1, a.err, abort_flag);
          }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = BF ? idesc_bf16(kRows, NB) : idesc_tf32(kRows, NB);
            bool ok = true;
            // stall test: this wait runs out after its limit, raises the timeout bit
            // and the abort flag, and every other wait of the CTA then gives up
            if (a.stall_test) ok = mbar_wait(never, 0, a.err, abort_flag);
            // the MMAs of block gb (its operands are in stage gb % ST) and the commits after them
            auto issue = [&](int gb) {
                const int blk = gb % NBLK, s = gb % ST;
                int kind, nb;
                sched_decode<KB, FILL>(blk, kind, nb);
                fence_after();
                const uint32_t st = smem_u32(stage0 + s * S::kStage);
                const uint32_t a_hi = st + S::kR, a_lo = a_hi + S::kA, b_hi = a_lo + S::kA, b_lo = b_hi + S::kB;
                const uint32_t d = kind == 0 ? t_u : t_inc;
                const bool first = blk <= 1;       // first inverse block, first noise block
                if constexpr (BF) {
#pragma unroll
                    for (int kk = 0; kk < kKB / 16; ++kk) {
                        const uint32_t off = kk * 32;   // 16 BF16 = 32 bytes along K
                        if constexpr (TWO) {
                            mma_bf16(d, sdesc64(a_lo + off), sdesc64(b_hi + off), idesc, (first && kk == 0) ? 0u : 1u);
                        } else {
                            mma_bf16(d, sdesc64(a_hi + off), sdesc64(b_lo + off), idesc, (first && kk == 0) ? 0u : 1u);
                            mma_bf16(d, sdesc64(a_lo + off), sdesc64(b_hi + off), idesc, 1u);
                        }
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
                mma_commit_mc(&empty[s], 3);   // both CTAs' stage s
                if (blk == sched_inv<KB>(KB - 1)) mma_commit(u_done);
                if (blk == NBLK - 1) {
                    mma_commit(inc_done);
                    mma_commit_mc(both_done, 3);
                }
            };
            const int G = a.n_steps * NBLK;
            {
                // Two streams of work, polled in turn: the MMAs of every block in
                // order, and the copy of each block this CTA owns (its A operand,
                // hi and lo) into the same stage of the other CTA as soon as its
                // writers are done.  A copy waits for the release counter first
                // (the stage's previous uses may be the other CTA's blocks), which
                // makes the `ready` parity exact.
                const uint32_t peer_stage0 = mapa(smem_u32(stage0), rank ^ 1u);
                const uint32_t peer_full = mapa(smem_u32(full), rank ^ 1u);
                auto next_own = [&](int g) {
                    for (; g < G; ++g) {
                        int kind, nb;
                        sched_decode<KB, FILL>(g % NBLK, kind, nb);
                        if ((uint32_t)(nb & 1) == rank) break;
                    }
                    return g;
                };
                int mb = 0, cb = next_own(0);
                uint64_t t0 = globaltimer();
                while (ok && (mb < G || cb < G)) {
                    bool moved = false;
                    if (cb < G) {
                        const int s = cb % ST;
                        if (ld_acquire_smem(s_freed) >= cb && mbar_test_wait(&ready[s], (cb / ST) & 1)) {
                            const uint32_t off = (uint32_t)(s * S::kStage + S::kR);
                            bulk_copy_to_peer(peer_stage0 + off, stage0 + off, 2u * S::kA, peer_full + 8u * (uint32_t)s);
                            cb = next_own(cb + 1);
                            moved = true;
                        }
                    }
                    if (mb < G) {
                        const int s = mb % ST;
                        const uint32_t ph = (mb / ST) & 1;
                        if (mbar_test_wait(&full[s], ph) && mbar_test_wait(&ready[s], ph)) {
                            issue(mb++);
                            moved = true;
                        }
                    }
                    if (moved) {
                        t0 = globaltimer();
                    } else if (*abort_flag) {
                        ok = false;
                    } else if (globaltimer() - t0 > kTimeoutNs) {
                        atomicOr(a.err, 2);
                        *abort_flag = 1;
                        ok = false;
                    } else {
                        __nanosleep(20);
                    }
                }
                if (!ok) {
                    // after a timeout: let copies already issued to the other CTA land
                    const uint64_t t1 = globaltimer();
                    while (globaltimer() - t1 < 1000000ull) __nanosleep(1000);
                }
            }
        }
    } else if (warp >= 2 + kComputeWarps) {
        // ---------------- noise warps: Philox normals of noise block j (Eq. b5),
        // drawn into registers (noise_draw), then written as hi / lo operands once
        // the stage is free (noise_put); this CTA draws the blocks j = 2 i + rank.
        const int nw = warp - 2 - kComputeWarps;
        auto draw = [&](int qn, float (&zz)[kChunksPerWarp][4]) {
            const int sp = qn / KBL;
            noise_draw(zz, nw, qn, 2 * (qn - sp * KBL) + (int)rank, sp, lane, a.cpt, Ct, a.seed, s_job, s_step);
        };
        // Noise blocks in sequence qn = KBL step + i.  Block qn is drawn into `cur`
        // right after block qn - 1 is written, then written as soon as its stage
        // is free (nothing more drawn ahead, as in the single-CTA kernel).
        bool ok = true, finite = true;
        double cm_unused[3];
        const int eq = warp & 3, et = (warp - 2 - kComputeWarps) / 4;   // epilogue quarter, worker 2 + et
        const int nq = a.n_steps * KBL;
        float cur[kChunksPerWarp][4];
        draw(0, cur);
#pragma unroll 1
        for (int qn = 0; qn < nq; ++qn) {
            const int sp = qn / KBL, ib = qn - sp * KBL;
            const int j = 2 * ib + (int)rank;
            const int blk = sp * NBLK + sched_noise<KB, FILL>(j), s = blk % ST;
            // Consecutive noise blocks may lie more than ST blocks apart, where a
            // parity wait on the stage's barrier is ambiguous: wait instead until
            // the producer has seen the stage released for this block (which it
            // does in block order, after the previous step's epilogue).
            ok = ok && count_wait(s_freed, blk, a.err, abort_flag);
            if (ok) {
                uint8_t* ah = stage0 + s * S::kStage + S::kR;
                uint8_t* al = ah + S::kA;
                noise_put<BF>(ah, al, cur, nw, qn, lane, a.cpt, s_rowb);
                fence_proxy_async();
            }
            __syncwarp();
            if (lane == 0 && ok) mbar_arrive_cnt(&ready[s], kReadyCount / kNoiseWarps);
            // after its last noise block, the step's epilogue (this warp's share)
            if (ib == KBL - 1)
                epilogue(sp, eq, 2 + et, 2 + kNoiseInQ[(eq + 2) & 3], ok, finite, cm_unused[0], cm_unused[1],
                         cm_unused[2]);
            if (qn + 1 < nq) draw(qn + 1, cur);
        }
        if (!finite) atomicOr(a.err, 1);
    } else {
        // ---------------- compute warps 2..9: two per TMEM lane quarter q; lane
        // 3 k + axis of quarter q is axis `axis` of the quarter's chain k.
        const int cw = warp - 2;            // 0..7
        const int ct = threadIdx.x - 64;    // 0..255
        const int q = warp & 3;             // TMEM lane quarter this warp may access
        const int half = cw >> 2;           // which 16 of a block's 32 columns
        const int row = 32 * q + lane;
        const int kq = lane / 3, ax = lane - 3 * (lane / 3);
        const bool inrow = kq < cpq;        // the row belongs to a chain slot of the tile
        const int cl = inrow ? cpq * q + kq : 0;   // chain of the tile
        const bool live = inrow && cl < Ct;
        const int src0 = lane - ax;         // lane of axis 0 of this chain
        // the chain's FP64 centre of mass, on its axis-0 lane of a first-half warp
        // (of rank 0, which holds mode 0)
        const bool own_cm = half == 0 && live && ax == 0 && rank == 0;
        double cm_x = 0.0, cm_y = 0.0, cm_z = 0.0;
        if (own_cm) {
            const double* cm = a.com + 3 * (size_t)(c0 + cl);
            cm_x = cm[0];
            cm_y = cm[1];
            cm_z = cm[2];
        }
        bool ok = true;
        bool finite = true;
        auto arrive = [&](int s) {
            __syncwarp();
            if (lane == 0 && ok) mbar_arrive_cnt(&ready[s], kReadyCount / kComputeWarps);
        };
#pragma unroll 1
        for (int sp = 0; sp < a.n_steps; ++sp) {
        const int g0 = sp * NBLK;                     // global index of this step's first block
        // (1) split the R tile of each inverse block of this CTA (nb = 2 i + rank)
        //     into hi / lo operands
#pragma unroll 1
        for (int ib = 0; ib < KBL; ++ib) {
            const int nb = 2 * ib + (int)rank;
            const int blk = g0 + sched_inv<KB>(nb), s = blk % ST;
            const uint32_t ph = (blk / ST) & 1;
            // The stage's previous uses may be blocks these warps never waited for
            // (noise blocks, or the other CTA's blocks), so a parity wait alone
            // could be two phases ahead; the producer's release counter first
            // (the stage's previous use is consumed) makes it exact.
            ok = ok && count_wait(s_freed, blk, a.err, abort_flag);
            ok = ok && mbar_wait(&full[s], ph, a.err, abort_flag);
            if constexpr (BF) {
                // row t/4, BF16 chunk t%4 (8 values) of the FP32 tile in A hi + A lo:
                // every compute thread reads its values, the eight compute warps
                // meet (named barrier 1, always taken by all of them), then the hi
                // and lo parts overwrite the tile
                uint8_t* base = stage0 + s * S::kStage;
                float xv[kRows * 4 / kCompute][8];
#pragma unroll
                for (int e = 0; e < kRows * 4 / kCompute; ++e) {
                    const int t = ct + kCompute * e;
                    const int r = t >> 2, c = t & 3;
                    if (ok && (r & 31) < 3 * cpq) {   // padding rows of a lane quarter stay as they are
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {
                            const float4 x = *reinterpret_cast<const float4*>(base + swz(r, 8 * c + 4 * h2));
                            xv[e][4 * h2] = x.x; xv[e][4 * h2 + 1] = x.y; xv[e][4 * h2 + 2] = x.z; xv[e][4 * h2 + 3] = x.w;
                        }
                    }
                }
                __syncwarp();
                asm volatile("bar.sync 1, %0;" ::"n"(kCompute) : "memory");
#pragma unroll
                for (int e = 0; e < kRows * 4 / kCompute; ++e) {
                    const int t = ct + kCompute * e;
                    const int r = t >> 2, c = t & 3;
                    if (ok && (r & 31) < 3 * cpq) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const uint16_t h0 = bf16_rn(xv[e][2 * i]), h1 = bf16_rn(xv[e][2 * i + 1]);
                            hw[i] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                            lw[i] = (uint32_t)bf16_rn(xv[e][2 * i] - bf16_f(h0)) |
                                    ((uint32_t)bf16_rn(xv[e][2 * i + 1] - bf16_f(h1)) << 16);
                        }
                        const uint32_t o = swz_bf(r, 8 * c);
                        *reinterpret_cast<uint4*>(base + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(base + S::kA + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
                if (ok) fence_proxy_async();
            } else if (ok) {
                float4* ah = (float4*)(stage0 + s * S::kStage);
                float4* al = (float4*)(stage0 + s * S::kStage + S::kA);
#pragma unroll
                for (int i = 0; i < S::kA / 16 / kCompute; ++i) {
                    const int e = ct + kCompute * i;
                    if (((e >> 3) & 31) >= 3 * cpq) continue;   // padding rows of a lane quarter
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
            arrive(s);
        }

        // (2) per bead block of this CTA's D_u: bond vectors -> residual force v
        //     (Eq. e11), |u_n| from the chain's three rows by warp shuffles; the
        //     force block's schedule index is k (bond block 8 rank + ib)
        ok = ok && mbar_wait(u_done, sp & 1, a.err, abort_flag);
        fence_after();
#pragma unroll 1
        for (int ib = 0; ib < KBL; ++ib) {
            const int k = 2 * ib + (int)rank;
            const int col = ib * kKB + 16 * half;       // first bond (TMEM column) of this warp's 16
            float v[16];
            tmem_ld16(t_u + ((uint32_t)(32 * q) << 16) + (uint32_t)col, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float sq = v[i] * v[i];
                const float t = sq + __shfl_down_sync(0xffffffffu, sq, 1) + __shfl_down_sync(0xffffffffu, sq, 2);
                const float fac = __shfl_sync(0xffffffffu, rsqrtf(t) - a.c12nu, src0);
                v[i] = (live && col0 + col + i >= 1) ? v[i] * fac : 0.f;
            }
            const int blk = g0 + sched_force<KB, FILL>(k), s = blk % ST;
            // as for the split, the release counter instead of a parity wait (it
            // also covers the other CTA's MMAs, which `empty` counts)
            ok = ok && count_wait(s_freed, blk, a.err, abort_flag);
            if (ok && inrow) {
                uint8_t* ah = stage0 + s * S::kStage + S::kR;
                uint8_t* al = ah + S::kA;
                if constexpr (BF) {
#pragma unroll
                    for (int h8 = 0; h8 < 2; ++h8) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float x0 = v[8 * h8 + 2 * i], x1 = v[8 * h8 + 2 * i + 1];
                            const uint16_t h0 = bf16_rn(x0), h1 = bf16_rn(x1);
                            hw[i] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                            lw[i] = (uint32_t)bf16_rn(x0 - bf16_f(h0)) | ((uint32_t)bf16_rn(x1 - bf16_f(h1)) << 16);
                        }
                        const uint32_t o = swz_bf(row, 16 * half + 8 * h8);
                        *reinterpret_cast<uint4*>(ah + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4*>(al + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                } else {
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        float4 h, l;
                        h.x = tf32_rna(v[4 * k4]);     l.x = tf32_rna(v[4 * k4] - h.x);
                        h.y = tf32_rna(v[4 * k4 + 1]); l.y = tf32_rna(v[4 * k4 + 1] - h.y);
                        h.z = tf32_rna(v[4 * k4 + 2]); l.z = tf32_rna(v[4 * k4 + 2] - h.z);
                        h.w = tf32_rna(v[4 * k4 + 3]); l.w = tf32_rna(v[4 * k4 + 3] - h.w);
                        const uint32_t o = swz(row, 16 * half + 4 * k4);
                        *reinterpret_cast<float4*>(ah + o) = h;
                        *reinterpret_cast<float4*>(al + o) = l;
                    }
                }
            }
            if (ok) fence_proxy_async();
            arrive(s);
        }

        // (3) epilogue, shared with the noise warps of this lane quarter
        epilogue(sp, q, half, 2 + kNoiseInQ[(q + 2) & 3], ok, finite, cm_x, cm_y, cm_z);
        }   // steps
        if (ok && own_cm) {
            double* cm = a.com + 3 * (size_t)(c0 + cl);
            cm[0] = cm_x;
            cm[1] = cm_y;
            cm[2] = cm_z;
            a.step[c0 + cl] = max(s_step[cl], min(s_step[cl] + (int64_t)a.n_steps, s_stop[cl]));
        }
        if (!finite) atomicOr(a.err, 1);
    }
    fence_before();
    // neither CTA leaves while the other may still copy into or arrive on its shared memory
    __syncwarp();
    cluster_sync();
    return *abort_flag == 0;
}

// After a pair tile gave up, the other CTA may have issued a copy into this
// CTA's stages just before the cluster barrier: let it land before leaving.
__device__ __forceinline__ void pair_abort_grace()
{
    if (threadIdx.x == 32) {
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 1000000ull) __nanosleep(1000);
    }
}

// One 512-bead tile per cluster of two CTAs (a launch of one length group).
template <bool BF, bool TWO = false>
__global__ void __launch_bounds__(kThreads, 1)
k_fused_pair(const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmChiH,
             const __grid_constant__ CUtensorMap tmChiL, const __grid_constant__ CUtensorMap tmFH,
             const __grid_constant__ CUtensorMap tmFL, const FusedArgs a)
{
    if (cluster_size() != 2u) {
        // every access to the other CTA assumes a cluster of two
        if (threadIdx.x == 0) atomicOr(a.err, 4);
        return;
    }
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t s_tmem;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    tmem_alloc<512>(&s_tmem);
    const uint32_t tmem = s_tmem;
    const bool ok = pair_tile<BF, TWO>(tmR, tmChiH, tmChiL, tmFH, tmFL, a, (int)(blockIdx.x >> 1), smem, tmem);
    tmem_free<512>(tmem);
    if (!ok) pair_abort_grace();
}



// All length groups of a batch on the fused step (at most one group each of
// 64, 128, 256 and 512 beads) in one launch of clusters of two CTAs: the first
// clusters each run a 512-bead tile together (pair_tile), every later cluster
// two tiles of the other lengths, one per CTA (fused_tile), the 256-bead tiles
// first, then 128, then 64.  Clusters start in index order as SMs free up, so
// the longest tiles start first and the short ones fill the tail.
struct GroupSlot {
    CUtensorMap tmR, tmChiH, tmChiL, tmFH, tmFL;
    FusedArgs a;
    int tiles;      // 0: the slot is unused
};
struct GroupedArgs {
    GroupSlot g[4];     // 512, 256, 128, 64 beads
    int* err;
};

// A tile of one slot as a call of its own (not inlined), so that each length's
// body gets its own register allocation.
template <int NB, bool BF, bool TWO>
__device__ __noinline__ bool grouped_tile(const GroupSlot& g, int tile, uint8_t* smem, uint32_t tmem)
{
    return fused_tile<NB, BF, TWO>(g.tmR, g.tmChiH, g.tmChiL, g.tmFH, g.tmFL, g.a, tile, smem, tmem);
}
template <bool BF, bool TWO>
__device__ __noinline__ bool grouped_pair(const GroupSlot& g, int tile, uint8_t* smem, uint32_t tmem)
{
    return pair_tile<BF, TWO>(g.tmR, g.tmChiH, g.tmChiL, g.tmFH, g.tmFL, g.a, tile, smem, tmem);
}

template <bool BF, bool TWO>
__global__ void __launch_bounds__(kThreads, 1)
k_fused_grouped(const __grid_constant__ GroupedArgs P)
{
    if (cluster_size() != 2u) {
        if (threadIdx.x == 0) atomicOr(P.err, 4);
        return;
    }
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t s_tmem;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    tmem_alloc<512>(&s_tmem);
    const uint32_t tmem = s_tmem;
    const int k = (int)(blockIdx.x >> 1);
    const int np = P.g[0].tiles;
    bool ok = true;
    if (k < np) {
        ok = grouped_pair<BF, TWO>(P.g[0], k, smem, tmem);
    } else {
        const int item = 2 * (k - np) + (int)cluster_rank();
        const int n1 = P.g[1].tiles, n2 = n1 + P.g[2].tiles, n3 = n2 + P.g[3].tiles;
        if (item < n1) ok = grouped_tile<256, BF, TWO>(P.g[1], item, smem, tmem);
        else if (item < n2) ok = grouped_tile<128, BF, TWO>(P.g[2], item - n1, smem, tmem);
        else if (item < n3) ok = grouped_tile<64, BF, TWO>(P.g[3], item - n2, smem, tmem);
    }
    fence_before();
    __syncthreads();
    tmem_free<512>(tmem);
    if (!ok && k < np) pair_abort_grace();
}

}  // namespace

struct FusedPlan {
    int M = 0, C = 0, cpt = kChains;
    bool bf16 = false, two = false;
    void* tab[4] = {nullptr, nullptr, nullptr, nullptr};    // chi_hi, chi_lo, F_hi, F_lo (TF32 or BF16)
    float* R = nullptr;
    float* w32 = nullptr;       // w_p with w_0 (FP32), for the mode-keyed epilogue
    float* zbuf = nullptr;      // mode-keyed noise of two steps [2][C][3][M]
    bool mz = false;            // mode-keyed noise on
    CUtensorMap tmR, tmChiH, tmChiL, tmFH, tmFL;
};

// Chains per tile: a multiple of 4 (one share per TMEM lane quarter), 4..kChains.
static int round_tile(int cpt) { return std::min(kChains, std::max(4, (cpt + 3) / 4 * 4)); }

bool fused_supported(int M) { return M == 64 || M == 128 || M == 256 || M == 512; }

// Dynamic shared memory of the grouped kernel: that of its largest tile.
static int grouped_smem(bool bf16)
{
    return bf16 ? std::max({FSmem<256, true, true>::kBytes, FSmem<128, true, true>::kBytes, FSmem<64, true, true>::kBytes,
                            FSmem<256, true, false>::kBytes})
                : std::max({FSmem<256, false, false>::kBytes, FSmem<128, false, false>::kBytes,
                            FSmem<64, false, false>::kBytes});
}

template <int NB, bool BF, bool TWO = false, bool MZ = false>
static cudaError_t set_smem()
{
    return cudaFuncSetAttribute(k_fused_step<NB, BF, TWO, MZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                FSmem<NB, BF, kRS<NB, BF, MZ>>::kBytes);
}
template <bool BF, bool TWO = false>
static cudaError_t set_smem_pair()
{
    return cudaFuncSetAttribute(k_fused_pair<BF, TWO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                FSmem<256, BF, false>::kBytes);
}

int fused_create(FusedPlan** out, int M, int C, const double* chi, const double* phi, const double* h,
                 const double* w, float* R, cudaStream_t stream, bool bf16, bool two)
{
    *out = nullptr;
    if (!fused_supported(M)) return report(SFP_ENOTSUP, "the fused step needs M in {64, 128, 256, 512}");
    FusedPlan* p = new FusedPlan();
    p->M = M;
    p->C = C;
    p->R = R;
    p->bf16 = bf16;
    p->two = bf16 && two;
    // the fewest waves of tiles of at most 40 chains (a 512-bead tile takes two
    // SMs), then the chains spread evenly over the tiles of those waves: chains
    // per tile = ceil(C / (units x waves)) rounded up to a multiple of 4
    // (fused_set_tile changes it)
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 148;
    const int units = M == 512 ? sms / 2 : sms;
    const int waves = std::max(1, (C + units * kChains - 1) / (units * kChains));
    p->cpt = round_tile((C + units * waves - 1) / (units * waves));
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
                hb[i] = bf16_round_host((float)src[t][i]);
                lb[i] = bf16_round_host((float)(src[t][i] - (double)bf16_to_float_host(hb[i])));
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
    // one box per lane quarter of the tile, 3 cpt / 4 rows: a tile never writes
    // the next tile's chains
    if ((rc = make_map_2d(&p->tmR, R, 3 * C, M, 3 * (p->cpt / 4)))) {
        fused_destroy(p);
        return rc;
    }
    // B operand boxes: the rows of one CTA's TMEM half (all M, or 256 of 512)
    const int bx = std::min(M, 256);
    if (bf16)
        rc = make_map_bf16(&p->tmChiH, p->tab[0], M, M, bx) ? -1 : make_map_bf16(&p->tmChiL, p->tab[1], M, M, bx) ? -1 :
             make_map_bf16(&p->tmFH, p->tab[2], 2 * M, M, bx) ? -1 : make_map_bf16(&p->tmFL, p->tab[3], 2 * M, M, bx);
    else
        rc = make_map_2d(&p->tmChiH, (const float*)p->tab[0], M, M, bx) ? -1 :
             make_map_2d(&p->tmChiL, (const float*)p->tab[1], M, M, bx) ? -1 :
             make_map_2d(&p->tmFH, (const float*)p->tab[2], 2 * M, M, bx) ? -1 :
             make_map_2d(&p->tmFL, (const float*)p->tab[3], 2 * M, M, bx);
    if (rc) {
        fused_destroy(p);
        return SFP_ECUDA;
    }
    cudaError_t e;
    if (p->two)
        e = M == 512 ? set_smem_pair<true, true>() : M == 256 ? set_smem<256, true, true>() :
            M == 128 ? set_smem<128, true, true>() : set_smem<64, true, true>();
    else if (bf16)
        e = M == 512 ? set_smem_pair<true>() : M == 256 ? set_smem<256, true>() :
            M == 128 ? set_smem<128, true>() : set_smem<64, true>();
    else
        e = M == 512 ? set_smem_pair<false>() : M == 256 ? set_smem<256, false>() :
            M == 128 ? set_smem<128, false>() : set_smem<64, false>();
    if (e == cudaSuccess && !p->two && M <= 256)
        e = bf16 ? (M == 256 ? set_smem<256, true, false, true>() : M == 128 ? set_smem<128, true, false, true>()
                                                                          : set_smem<64, true, false, true>())
                 : (M == 256 ? set_smem<256, false, false, true>() : M == 128 ? set_smem<128, false, false, true>()
                                                                             : set_smem<64, false, false, true>());
    if (e == cudaSuccess) {
        // w_p with w_0 (the centre of mass) in FP32, for the mode-keyed epilogue
        std::vector<float> wf(M);
        for (int q = 0; q < M; ++q) wf[q] = (float)w[q];
        e = cudaMalloc((void**)&p->w32, (size_t)M * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->w32, wf.data(), (size_t)M * sizeof(float), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(p->two ? k_fused_grouped<true, true> : bf16 ? k_fused_grouped<true, false>
                                                                             : k_fused_grouped<false, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, grouped_smem(bf16));
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
    if (args.C < 1 || args.C > p->C) return report(SFP_EINVAL, "fused step: chain count outside the plan");
    const dim3 grid((unsigned)((args.C + p->cpt - 1) / p->cpt));   // the first args.C chains
    FusedArgs a = args;
    a.zbuf = p->zbuf;
    a.w = p->w32;
    if (p->mz && (p->two || p->M > 256)) return report(SFP_ENOTSUP, "mode-keyed noise: M <= 256, three passes");
#define SFP_FUSED_LAUNCH(NBV, BFV)                                                                   \
    if (p->mz)                                                                                       \
        k_fused_step<NBV, BFV, false, true><<<grid, kThreads, FSmem<NBV, BFV, kRS<NBV, BFV, true>>::kBytes, stream>>>( \
            p->tmR, p->tmChiH, p->tmChiL, p->tmFH, p->tmFL, a);                                      \
    else if (p->two)                                                                                 \
        k_fused_step<NBV, BFV, BFV><<<grid, kThreads, FSmem<NBV, BFV, kRS<NBV, BFV>>::kBytes, stream>>>(         \
            p->tmR, p->tmChiH, p->tmChiL, p->tmFH, p->tmFL, a);                                      \
    else                                                                                             \
        k_fused_step<NBV, BFV><<<grid, kThreads, FSmem<NBV, BFV, kRS<NBV, BFV>>::kBytes, stream>>>(              \
            p->tmR, p->tmChiH, p->tmChiL, p->tmFH, p->tmFL, a)
    cudaError_t e = cudaSuccess;
    switch (p->M * 2 + (p->bf16 ? 1 : 0)) {
        case 1024:
        case 1025: {
            // two CTAs (a cluster) per tile
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(2u * grid.x);
            cfg.blockDim = dim3(kThreads);
            cfg.dynamicSmemBytes = p->bf16 ? FSmem<256, true, false>::kBytes : FSmem<256, false, false>::kBytes;
            cfg.stream = stream;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 2;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            e = p->two ? cudaLaunchKernelEx(&cfg, k_fused_pair<true, true>, p->tmR, p->tmChiH, p->tmChiL, p->tmFH,
                                            p->tmFL, args)
              : p->bf16 ? cudaLaunchKernelEx(&cfg, k_fused_pair<true>, p->tmR, p->tmChiH, p->tmChiL, p->tmFH,
                                             p->tmFL, args)
                        : cudaLaunchKernelEx(&cfg, k_fused_pair<false>, p->tmR, p->tmChiH, p->tmChiL, p->tmFH,
                                             p->tmFL, args);
            break;
        }
        case 512: SFP_FUSED_LAUNCH(256, false); break;
        case 513: SFP_FUSED_LAUNCH(256, true); break;
        case 256: SFP_FUSED_LAUNCH(128, false); break;
        case 257: SFP_FUSED_LAUNCH(128, true); break;
        case 128: SFP_FUSED_LAUNCH(64, false); break;
        case 129: SFP_FUSED_LAUNCH(64, true); break;
        default: return report(SFP_ENOTSUP, "unsupported fused-step length");
    }
#undef SFP_FUSED_LAUNCH
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return report(SFP_ECUDA, cudaGetErrorString(e));
    return SFP_OK;
}

bool fused_groupable(const FusedPlan* p) { return p != nullptr; }

int fused_step_grouped(FusedPlan* const* plans, const FusedArgs* args, int n, cudaStream_t stream)
{
    if (n < 1 || n > 4) return report(SFP_EINVAL, "grouped step: 1 to 4 plans");
    GroupedArgs P;
    std::memset(&P, 0, sizeof P);
    const bool bf = plans[0]->bf16, two = plans[0]->two;
    for (int i = 0; i < n; ++i) {
        const FusedPlan* p = plans[i];
        const int slot = p->M == 512 ? 0 : p->M == 256 ? 1 : p->M == 128 ? 2 : p->M == 64 ? 3 : -1;
        if (slot < 0 || P.g[slot].tiles || p->bf16 != bf || p->two != two || args[i].cpt != p->cpt ||
            args[i].n_steps != args[0].n_steps)
            return report(SFP_EINVAL, "grouped step: one plan each of 64, 128, 256, 512 beads, one arithmetic");
        GroupSlot& g = P.g[slot];
        g.tmR = p->tmR; g.tmChiH = p->tmChiH; g.tmChiL = p->tmChiL; g.tmFH = p->tmFH; g.tmFL = p->tmFL;
        g.a = args[i];
        if (args[i].C < 1 || args[i].C > p->C) return report(SFP_EINVAL, "grouped step: chain count outside the plan");
        g.tiles = (args[i].C + p->cpt - 1) / p->cpt;
    }
    P.err = args[0].err;
    const int small = P.g[1].tiles + P.g[2].tiles + P.g[3].tiles;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2u * (unsigned)(P.g[0].tiles + (small + 1) / 2));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = grouped_smem(bf);
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = two ? cudaLaunchKernelEx(&cfg, k_fused_grouped<true, true>, P)
                        : bf ? cudaLaunchKernelEx(&cfg, k_fused_grouped<true, false>, P)
                             : cudaLaunchKernelEx(&cfg, k_fused_grouped<false, false>, P);
    if (e != cudaSuccess) return report(SFP_ECUDA, cudaGetErrorString(e));
    return SFP_OK;
}

int fused_tile(const FusedPlan* p) { return p->cpt; }

int fused_ctas_per_tile(const FusedPlan* p) { return p->M == 512 ? 2 : 1; }

size_t fused_bytes(const FusedPlan* p)
{
    if (!p) return 0;
    return (size_t)6 * p->M * p->M * (p->bf16 ? 2 : 4) + (size_t)p->M * sizeof(float) +
           (p->zbuf ? (size_t)2 * p->C * 3 * p->M * sizeof(float) : 0);
}

int fused_set_tile(FusedPlan* p, int cpt)
{
    if (cpt < 1 || cpt > kChains) return report(SFP_EINVAL, "chains per tile must be 1..40");
    cpt = round_tile(cpt);
    CUtensorMap m;
    const int rc = make_map_2d(&m, p->R, 3 * p->C, p->M, 3 * (cpt / 4));
    if (rc) return rc;
    p->tmR = m;
    p->cpt = cpt;
    return SFP_OK;
}

bool fused_mode_noise_supported(int M) { return M == 64 || M == 128 || M == 256; }

int fused_set_mode_noise(FusedPlan* p, bool on)
{
    if (on && (!fused_mode_noise_supported(p->M) || p->two))
        return report(SFP_ENOTSUP, "mode-keyed noise on the fused step: 64, 128 or 256 beads, three passes");
    if (on && !p->zbuf) {
        const size_t bytes = (size_t)2 * p->C * 3 * p->M * sizeof(float);
        if (cudaMalloc((void**)&p->zbuf, bytes) != cudaSuccess) return report(SFP_ENOMEM, "mode-noise buffer allocation failed");
    }
    p->mz = on;
    return SFP_OK;
}

void fused_destroy(FusedPlan* p)
{
    if (!p) return;
    for (void* t : p->tab)
        if (t) cudaFree(t);
    if (p->w32) cudaFree(p->w32);
    if (p->zbuf) cudaFree(p->zbuf);
    delete p;
}

}  // namespace sfp
